// rrg_adjoint.cu -- discrete adjoint of the robust RG objective.
//
// g(kappa) = min over scenarios k and steps j = 0..H of the slack
// s_j^k = h(x_j^k, v) - y_min, v = v_prev + kappa (r - v_prev) (Eq. 2), with
// x_{j+1} = RK4(x_j, v) + d_j^k (Eq. 4): the admissibility test of Alg. 3
// is g >= 0 (without the steady-state part).  Its derivative at the argmin
// (k*, j*) (a subgradient where the argmin is not unique) is obtained by the
// reverse (adjoint) sweep of the RK4 recursion of trajectory k* from j* back
// to 0:
//   forward  adjoint_forward_kernel: one thread per (kappa, scenario), full
//            horizon, with the rollouts' binary32/binary64 step, the state
//            saved every `checkpoint` steps, per-lane min and argmin;
//   argmin   adjoint_argmin_kernel: per kappa, the first (k, then j)
//            attaining the min;
//   reverse  adjoint_reverse_kernel: the checkpoint segments before j* are
//            recomputed in parallel (one thread each), storing every step's
//            state and RK4 stage points; one thread then sweeps them
//            backwards with the vector-Jacobian products of the FC3
//            right-hand side; the adjoints of the folded constants are
//            mapped to the 27 model parameters, to x_t and (through the
//            setpoint) to kappa.
#include <cfloat>
#include <cmath>

#include "rrg_device.cuh"
#include "rrg_internal.h"
#include "rrg_lane.cuh"

namespace rrg {

namespace {

// Adjoints of the constants the right-hand side and output read.
template <typename T>
struct ConstAdj {
  T a_w, a_p, k_sm, k_ca, e, C_cp, C_m, k_v, K_p, RT_Vca, RT_Vsm, inv_J, inv_p_atm;
  T W_o2, V0, y_scale;
};

// The elementary functions of the reverse sweep.  binary32: MUFU forms
// (__powf, __logf, approximate reciprocal), relative errors of a few 1e-7,
// far inside what a binary32 gradient carries anyway; binary64: x^e through
// the handle's series (pow_m1_series falls back to pow outside [1, 2] or for
// another exponent), log and IEEE division.
template <typename T> struct VjpMath;
template <>
struct VjpMath<float> {
  static __device__ __forceinline__ float pw(float x, float e, const PowSeries*) { return __powf(x, e); }
  static __device__ __forceinline__ float ln(float x) { return __logf(x); }
  static __device__ __forceinline__ float inv(float x) { return __fdividef(1.0f, x); }
};
template <>
struct VjpMath<double> {
  static __device__ __forceinline__ double pw(double x, double e, const PowSeries* S) {
    return pow_m1_series(S, x, e) + 1.0;
  }
  static __device__ __forceinline__ double ln(double x) { return log(x); }
  static __device__ __forceinline__ double inv(double x) { return 1.0 / x; }
};

// Vector-Jacobian product of fc3_rhs at q with output adjoint (b_ca, b_w,
// b_sm): adds J^T b to (qb_ca, qb_w, qb_sm) and the constants' adjoints to g.
template <typename T>
__device__ void fc3_rhs_vjp(const Fc3K<T>& K, const CandK<T>& C, T q_ca, T w, T q_sm, T b_ca,
                            T b_w, T b_sm, T& qb_ca, T& qb_w, T& qb_sm, ConstAdj<T>& g) {
  // forward intermediates (as in fc3_rhs)
  const T W_cp = K.a_w * w - K.a_p * q_sm;
  const T W_sm = K.k_sm * (q_sm - q_ca);
  const T W_ca = K.k_ca * q_ca;
  const T Pi = T(1) + q_sm * K.inv_p_atm;
  const T Pe = VjpMath<T>::pw(Pi, K.e, K.pws);
  const T pr = Pe - T(1);
  const T inv_w = VjpMath<T>::inv(w);
  const T tau_cp = K.C_cp * pr * W_cp * inv_w;
  const T v_cm = C.V0 - K.K_p * W_cp;
  const T tau_cm = K.C_m * (v_cm - K.k_v * w);
  // d_ca = RT_Vca (W_sm - W_ca - W_o2)
  g.RT_Vca += b_ca * (W_sm - W_ca - C.W_o2);
  T Wsm_b = K.RT_Vca * b_ca;
  const T Wca_b = -K.RT_Vca * b_ca;
  g.W_o2 += -K.RT_Vca * b_ca;
  // d_w = (tau_cm - tau_cp) inv_J
  g.inv_J += b_w * (tau_cm - tau_cp);
  const T tcm_b = K.inv_J * b_w, tcp_b = -K.inv_J * b_w;
  // d_sm = RT_Vsm (W_cp - W_sm)
  g.RT_Vsm += b_sm * (W_cp - W_sm);
  T Wcp_b = K.RT_Vsm * b_sm;
  Wsm_b += -K.RT_Vsm * b_sm;
  // tau_cm = C_m (v_cm - k_v w)
  g.C_m += tcm_b * (v_cm - K.k_v * w);
  const T vcm_b = K.C_m * tcm_b;
  T w_b = -K.C_m * K.k_v * tcm_b;
  g.k_v += -K.C_m * w * tcm_b;
  // v_cm = V0 - K_p W_cp
  g.V0 += vcm_b;
  g.K_p += -W_cp * vcm_b;
  Wcp_b += -K.K_p * vcm_b;
  // tau_cp = C_cp pr W_cp / w
  g.C_cp += tcp_b * pr * W_cp * inv_w;
  const T pr_b = tcp_b * K.C_cp * W_cp * inv_w;
  Wcp_b += tcp_b * K.C_cp * pr * inv_w;
  w_b += -tcp_b * tau_cp * inv_w;
  // pr = Pi^e - 1
  g.e += pr_b * Pe * VjpMath<T>::ln(Pi);
  const T Pi_b = pr_b * K.e * Pe * VjpMath<T>::inv(Pi);
  // Pi = 1 + q_sm inv_p_atm
  T qsm_b = Pi_b * K.inv_p_atm;
  g.inv_p_atm += Pi_b * q_sm;
  // W_ca = k_ca q_ca
  g.k_ca += Wca_b * q_ca;
  T qca_b = K.k_ca * Wca_b;
  // W_sm = k_sm (q_sm - q_ca)
  g.k_sm += Wsm_b * (q_sm - q_ca);
  qsm_b += K.k_sm * Wsm_b;
  qca_b += -K.k_sm * Wsm_b;
  // W_cp = a_w w - a_p q_sm
  g.a_w += Wcp_b * w;
  g.a_p += -Wcp_b * q_sm;
  w_b += K.a_w * Wcp_b;
  qsm_b += -K.a_p * Wcp_b;
  qb_ca += qca_b;
  qb_w += w_b;
  qb_sm += qsm_b;
}

// The RK4 stage points of one step from x: y2 = x + dt/2 k1, y3 = x + dt/2 k2,
// y4 = x + dt k3 (k_i the right-hand side at the previous stage point);
// y[0..2] = y2, y[3..5] = y3, y[6..8] = y4.  They do not depend on the adjoint.
template <typename T>
__device__ __forceinline__ void rk4_stage_points(const Fc3K<T>& K, const CandK<T>& C, T dt, T q_ca, T w,
                                                 T q_sm, T* y) {
  const T h2 = T(0.5) * dt;
  T a, b, c;
  fc3_rhs<T>(K, C, q_ca, w, q_sm, a, b, c);
  y[0] = q_ca + h2 * a; y[1] = w + h2 * b; y[2] = q_sm + h2 * c;
  fc3_rhs<T>(K, C, y[0], y[1], y[2], a, b, c);
  y[3] = q_ca + h2 * a; y[4] = w + h2 * b; y[5] = q_sm + h2 * c;
  fc3_rhs<T>(K, C, y[3], y[4], y[5], a, b, c);
  y[6] = q_ca + dt * a; y[7] = w + dt * b; y[8] = q_sm + dt * c;
}

// Adjoint of one RK4 step q+ = q + dt/6 (k1 + 2 k2 + 2 k3 + k4) (+ d) at state
// q with stage points y (rk4_stage_points): given the adjoint (l0, l1, l2) of
// q+, overwrites it with the adjoint of q; the constants' adjoints accumulate
// into g.
template <typename T>
__device__ void rk4_step_vjp_at(const Fc3K<T>& K, const CandK<T>& C, T dt, T q_ca, T w, T q_sm,
                                const T* y, T& l0, T& l1, T& l2, ConstAdj<T>& g) {
  const T h2 = T(0.5) * dt, h6 = dt / T(6);
  T q0 = l0, q1 = l1, q2 = l2;                  // identity part
  T k1_0 = h6 * l0, k1_1 = h6 * l1, k1_2 = h6 * l2;
  T k2_0 = T(2) * h6 * l0, k2_1 = T(2) * h6 * l1, k2_2 = T(2) * h6 * l2;
  T k3_0 = T(2) * h6 * l0, k3_1 = T(2) * h6 * l1, k3_2 = T(2) * h6 * l2;
  const T k4_0 = h6 * l0, k4_1 = h6 * l1, k4_2 = h6 * l2;
  T y0 = 0, y1 = 0, y2 = 0;
  fc3_rhs_vjp<T>(K, C, y[6], y[7], y[8], k4_0, k4_1, k4_2, y0, y1, y2, g);
  q0 += y0; q1 += y1; q2 += y2;
  k3_0 += dt * y0; k3_1 += dt * y1; k3_2 += dt * y2;
  y0 = y1 = y2 = 0;
  fc3_rhs_vjp<T>(K, C, y[3], y[4], y[5], k3_0, k3_1, k3_2, y0, y1, y2, g);
  q0 += y0; q1 += y1; q2 += y2;
  k2_0 += h2 * y0; k2_1 += h2 * y1; k2_2 += h2 * y2;
  y0 = y1 = y2 = 0;
  fc3_rhs_vjp<T>(K, C, y[0], y[1], y[2], k2_0, k2_1, k2_2, y0, y1, y2, g);
  q0 += y0; q1 += y1; q2 += y2;
  k1_0 += h2 * y0; k1_1 += h2 * y1; k1_2 += h2 * y2;
  y0 = y1 = y2 = 0;
  fc3_rhs_vjp<T>(K, C, q_ca, w, q_sm, k1_0, k1_1, k1_2, y0, y1, y2, g);
  l0 = q0 + y0;
  l1 = q1 + y1;
  l2 = q2 + y2;
}

// Parameters of scenario k: theta, or theta_p m_p^k under parametric
// uncertainty (multipliers of scenario pair 0).
__device__ __forceinline__ void scenario_params(const Launch& L, int k, double* Pk) {
  for (int p = 0; p < RRG_NPARAM; ++p)
    Pk[p] = L.pmul ? __dmul_rn(L.params[p], L.pmul[static_cast<size_t>(k) * RRG_NPARAM + p])
                   : L.params[p];
}

template <typename T>
__device__ __forceinline__ Fc3K<T> konst(const double* Pk) {
  Fc3K<double> k64;
  Fc3K<float> k32;
  fold_constants(Pk, &k64, &k32);
  if constexpr (sizeof(T) == 8) return k64;
  else return k32;
}

template <typename T>
__device__ CandK<T> cand_of(const double* P, double I) {
  const double W_o2 = P[P_M_O2] * P[P_N_CELL] * I / (4.0 * P[P_FARADAY]);
  CandK<T> C;
  C.W_o2 = static_cast<T>(W_o2);
  C.V0 = static_cast<T>(P[P_C0] + P[P_C1] * I + P[P_C2] * I * I +
                        P[P_K_P] * P[P_LAM_REF] * W_o2 / P[P_X_O2]);
  C.y_scale = static_cast<T>(P[P_X_O2] * P[P_K_SM] / W_o2);
  return C;
}

// Register slots of the forward pass's disturbance prefetch ring.

constexpr int kFwdRing = 8;

// The launch's rollout constants in precision T.
template <typename T> __device__ __forceinline__ RhsU<T> launch_u(const Launch& L);
template <> __device__ __forceinline__ RhsU<float> launch_u<float>(const Launch& L) { return L.u32; }
template <> __device__ __forceinline__ RhsU<double> launch_u<double>(const Launch& L) { return L.u64; }
template <typename T> __device__ __forceinline__ RhsC<T> launch_c(const Launch& L, int i);
template <> __device__ __forceinline__ RhsC<float> launch_c<float>(const Launch& L, int i) { return L.cand_c32[i]; }
template <> __device__ __forceinline__ RhsC<double> launch_c<double>(const Launch& L, int i) { return L.cand_c64[i]; }

// Forward: one thread per (candidate slot i = blockIdx.y, scenario k), full
// horizon, with the rollouts' arithmetic (deviation coordinates about the
// candidate's reference point, the multiplied-out right-hand side, the
// slot's constants from the candidate set-up; under parametric uncertainty
// the scenario's own model): the state x_j is saved in gauge coordinates at
// j = 0, C, 2C, ... (j < H) into ckpt[((i N + k) nseg + c) 3 + .], and the
// lane's min slack and the first step attaining it go to lane_min / lane_arg
// [i N + k].  DT: the disturbance array's type (the stored binary32 copy for
// binary32 gradients when the handle draws one, else the binary64 values
// rounded to T).  The disturbances pass through a ring of kFwdRing register
// slots: step j takes slot j % kFwdRing and refills it with step j +
// kFwdRing's values (steps past the horizon re-read the last one), so each
// load has kFwdRing steps to arrive.
template <typename T, typename DT>
__global__ void __launch_bounds__(128)
adjoint_forward_kernel(const Launch L, const DT* __restrict__ d, int checkpoint,
                       double* __restrict__ ckpt, double* __restrict__ lane_min,
                       int* __restrict__ lane_arg) {
  const int i = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = L.N, H = L.H;
  if (k >= N) return;
  RhsU<T> K = launch_u<T>(L);
  RhsC<T> C = launch_c<T>(L, i);
  double p_atm = L.params[P_P_ATM];
  if (L.pmul != nullptr)
    p_atm = scenario_model<T>(L.params, L.pmul + static_cast<size_t>(k) * RRG_NPARAM, L.cand_v[i],
                              L.k64.pws, L.y_min, K, C);
  T z_ca, z_w, z_sm, w_abs;
  start_state<T>(C, L.st->x, p_atm, z_ca, z_w, z_sm, w_abs);
  const double r_ca = static_cast<double>(C.r_ca), r_w = static_cast<double>(C.r_w),
               r_sm = static_cast<double>(C.r_sm);
  const StepC<T> S = step_consts<T>(K, static_cast<T>(L.dt));
  const int nseg = H / checkpoint + 1;
  const size_t HN = static_cast<size_t>(H) * N;
  double* ck = ckpt + (static_cast<size_t>(i) * N + k) * nseg * 3;
  T smin = C.y_scale * (z_sm - z_ca) + C.s_off;
  int arg = 0;
  int next_ck = 0;  // the next step whose state is saved
  if constexpr (sizeof(T) == 4 && sizeof(DT) == 4) {
    // binary32 from the stored binary32 array: the rollouts' shared-memory
    // ring, one asynchronous copy per lane, component and step, RRG_RING_DEPTH
    // steps ahead (a warp running its chain alone issues its steps in order,
    // and the register ring's loads and index arithmetic sit between them)
    constexpr int D = RRG_RING_DEPTH;
    __shared__ float sring[D * 3 * 128];
    const int bd = blockDim.x;
    float* my = sring + threadIdx.x;
    const DT* pf = d + k;  // the next step to fetch
#pragma unroll 1
    for (int u = 0; u < D; ++u) {
      if (u < H) {
        cp_async4(my + (3 * u) * bd, pf);
        cp_async4(my + (3 * u + 1) * bd, pf + HN);
        cp_async4(my + (3 * u + 2) * bd, pf + 2 * HN);
      }
      cp_async_commit();
      pf += N;
    }
    int slot = 0;
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
      cp_async_wait<D - 1>();
      float* e = my + (3 * slot) * bd;
      const float e0 = e[0], e1 = e[bd], e2 = e[2 * bd];
      if (j == next_ck) {
        double* c = ck + (j / checkpoint) * 3;
        c[0] = static_cast<double>(z_ca) + r_ca;
        c[1] = static_cast<double>(z_w) + r_w;
        c[2] = static_cast<double>(z_sm) + r_sm;
        next_ck += checkpoint;
      }
      rk4_step_fast<T>(K, C, S, z_ca, z_w, z_sm, w_abs, e0, e1, e2);
      // the slot is free once its values are in registers: step j + D
      if (j + D < H) {
        cp_async4(e, pf);
        cp_async4(e + bd, pf + HN);
        cp_async4(e + 2 * bd, pf + 2 * HN);
      }
      cp_async_commit();
      pf += N;
      slot = (slot + 1) & (D - 1);
      const T s = C.y_scale * (z_sm - z_ca) + C.s_off;
      if (s < smin) { smin = s; arg = j + 1; }
    }
    cp_async_wait<0>();  // nothing in flight into the ring when the lane ends
    lane_min[static_cast<size_t>(i) * N + k] = static_cast<double>(smin);
    lane_arg[static_cast<size_t>(i) * N + k] = arg;
    return;
  }
  auto at = [&](int j) { return static_cast<size_t>(j < H ? j : H - 1) * N + k; };
  T ring[kFwdRing][3];
#pragma unroll
  for (int u = 0; u < kFwdRing; ++u) {
    const size_t o = at(u);
    ring[u][0] = static_cast<T>(d[o]);
    ring[u][1] = static_cast<T>(d[HN + o]);
    ring[u][2] = static_cast<T>(d[2 * HN + o]);
  }
  for (int j0 = 0; j0 < H; j0 += kFwdRing) {
#pragma unroll
    for (int u = 0; u < kFwdRing; ++u) {
      const int j = j0 + u;
      if (j >= H) break;
      const T e0 = ring[u][0], e1 = ring[u][1], e2 = ring[u][2];
      const size_t o = at(j + kFwdRing);
      ring[u][0] = static_cast<T>(d[o]);
      ring[u][1] = static_cast<T>(d[HN + o]);
      ring[u][2] = static_cast<T>(d[2 * HN + o]);
      if (j == next_ck) {
        double* c = ck + (j / checkpoint) * 3;
        c[0] = static_cast<double>(z_ca) + r_ca;
        c[1] = static_cast<double>(z_w) + r_w;
        c[2] = static_cast<double>(z_sm) + r_sm;
        next_ck += checkpoint;
      }
      rk4_step_fast<T>(K, C, S, z_ca, z_w, z_sm, w_abs, e0, e1, e2);
      const T s = C.y_scale * (z_sm - z_ca) + C.s_off;
      if (s < smin) { smin = s; arg = j + 1; }
    }
  }
  lane_min[static_cast<size_t>(i) * N + k] = static_cast<double>(smin);
  lane_arg[static_cast<size_t>(i) * N + k] = arg;
}

// Slot i = blockIdx.x: the first (k, then j) attaining the min of the
// slot's lanes; out[i * kOutStride + 0] = g, [1], [2] = k*, j* (as long long).
constexpr int kOutStride = kAdjOutStride;

// The argmin of slot i by the whole block (blockDim a power of two, at most
// the shared arrays' size): the smallest lane minimum, and among equal ones
// the smallest k, which the reduction order cannot change; written to
// o[0..2] by thread 0, visible to the block after its closing barrier.
__device__ void block_argmin(const double* __restrict__ lm, const int* __restrict__ la, int N, double* o,
                             double* sv, int* sk) {
  double best = INFINITY;
  int bk = 0x7fffffff;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const double s = lm[k];
    if (s < best || (s == best && k < bk)) { best = s; bk = k; }
  }
  sv[threadIdx.x] = best;
  sk[threadIdx.x] = bk;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double s = sv[threadIdx.x + w];
      const int kk = sk[threadIdx.x + w];
      if (s < sv[threadIdx.x] || (s == sv[threadIdx.x] && kk < sk[threadIdx.x])) {
        sv[threadIdx.x] = s;
        sk[threadIdx.x] = kk;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    long long kj[2] = {sk[0], (sk[0] >= 0 && sk[0] < N) ? la[sk[0]] : 0};
    o[0] = sv[0];
    memcpy(o + 1, kj, sizeof kj);
  }
  __syncthreads();
}

__global__ void adjoint_argmin_kernel(const double* __restrict__ lane_min,
                                      const int* __restrict__ lane_arg, int N, double* out) {
  __shared__ double sv[256];
  __shared__ int sk[256];
  const int i = blockIdx.x;
  block_argmin(lane_min + static_cast<size_t>(i) * N, lane_arg + static_cast<size_t>(i) * N, N,
               out + static_cast<size_t>(i) * kOutStride, sv, sk);
}

// Values stored per step of the recomputed trajectory: x_j and the three
// stage points of step j.
constexpr int kSegVals = 12;
constexpr int kRevThreads = 128;

// Reverse sweep of trajectory k* from j* to 0, then the chain rule from the
// folded constants to the model parameters and kappa.  One block:
//   phase 1, all threads: the checkpoint segments before j* are recomputed
//     in parallel, one segment per thread, storing for each step j its state
//     and stage points in seg[j * kSegVals ...], and x_{j*} after the last one;
//   phase 2, thread 0: the adjoint recursion from j* down to 0 over the
//     stored steps (the only serial part), each step's values loaded one step
//     ahead.
// seg: scratch of (j* + 1) * kSegVals values (at most (H + 1) * kSegVals).
// out[0] = dg/dkappa, out[1..3] = dg/dx_t, out[4..4+NPARAM) = dg/dtheta.
template <typename T, typename DT>
__global__ void __launch_bounds__(kRevThreads)
adjoint_reverse_kernel(const Launch L, const DT* __restrict__ d,
                       int checkpoint, const double* __restrict__ ckpt, T* __restrict__ seg_all,
                       double* __restrict__ out_all, int slot0, const double* __restrict__ lane_min,
                       const int* __restrict__ lane_arg) {
  const int i = slot0 + static_cast<int>(blockIdx.x);  // candidate slot
  const int N = L.N, H = L.H;
  // the inputs of the candidate set-up the forward pass ran on
  const double v_prev = L.st->v_prev, r = L.st->r;
  double* o = out_all + static_cast<size_t>(i) * kOutStride;
  if (lane_min != nullptr) {
    // the argmin first, by this block (one launch fewer than a separate pass)
    __shared__ double sv[kRevThreads];
    __shared__ int sk[kRevThreads];
    block_argmin(lane_min + static_cast<size_t>(i) * N, lane_arg + static_cast<size_t>(i) * N, N, o, sv, sk);
  }
  long long kj[2];
  memcpy(kj, o + 1, sizeof kj);
  double* out = o + 3;
  T* seg = seg_all + static_cast<size_t>(i) * (H + 1) * kSegVals;
  const double kappa = L.cand_kappa[i];
  const double v = governed(v_prev, r, kappa);
  if (kj[0] < 0 || kj[0] >= N || kj[1] < 0 || kj[1] > H) {  // no argmin: same for every thread
    if (threadIdx.x < 4 + RRG_NPARAM) out[threadIdx.x] = NAN;
    return;
  }
  const int k = static_cast<int>(kj[0]), jstar = static_cast<int>(kj[1]);
  double P[RRG_NPARAM];
  scenario_params(L, k, P);
  Fc3K<T> K = konst<T>(P);
  if (sizeof(T) == 8) K.pws = L.k64.pws;  // the series of the model's exponent (checked per call)
  const CandK<T> C = cand_of<T>(P, v);
  const T dt = static_cast<T>(L.dt);
  const int nseg = H / checkpoint + 1;
  const size_t HN = static_cast<size_t>(H) * N;
  const double* ck = ckpt + (static_cast<size_t>(i) * N + k) * nseg * 3;
  // phase 1: segment c covers steps c * checkpoint .. min((c + 1) * checkpoint, j*) - 1
  const int nc = jstar > 0 ? (jstar - 1) / checkpoint + 1 : 0;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const int j0 = c * checkpoint;
    const int j1 = (j0 + checkpoint < jstar) ? j0 + checkpoint : jstar;
    T a = static_cast<T>(ck[c * 3]), b = static_cast<T>(ck[c * 3 + 1]), e = static_cast<T>(ck[c * 3 + 2]);
    for (int j = j0; j < j1; ++j) {
      T* sj = seg + static_cast<size_t>(j) * kSegVals;
      sj[0] = a; sj[1] = b; sj[2] = e;
      rk4_stage_points<T>(K, C, dt, a, b, e, sj + 3);
      const size_t o = static_cast<size_t>(j) * N + k;
      rk4_step<T>(K, C, dt, a, b, e);
      a += static_cast<T>(d[o]);
      b += static_cast<T>(d[HN + o]);
      e += static_cast<T>(d[2 * HN + o]);
    }
    if (j1 == jstar) {
      T* sj = seg + static_cast<size_t>(jstar) * kSegVals;
      sj[0] = a; sj[1] = b; sj[2] = e;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  ConstAdj<T> g{};
  // output at j*: s = y_scale (q_sm - q_ca) - y_min (x_0 is checkpoint 0)
  T q_ca, q_sm;
  if (jstar == 0) {
    q_ca = static_cast<T>(ck[0]);
    q_sm = static_cast<T>(ck[2]);
  } else {
    q_ca = seg[static_cast<size_t>(jstar) * kSegVals];
    q_sm = seg[static_cast<size_t>(jstar) * kSegVals + 2];
  }
  g.y_scale += q_sm - q_ca;
  T l0 = -C.y_scale, l1 = T(0), l2 = C.y_scale;
  // phase 2: backwards over the stored steps
  if (jstar > 0) {
    T cur[kSegVals];
#pragma unroll
    for (int u = 0; u < kSegVals; ++u) cur[u] = seg[static_cast<size_t>(jstar - 1) * kSegVals + u];
    for (int j = jstar - 1; j >= 0; --j) {
      T nxt[kSegVals];
      const int jn = j > 0 ? j - 1 : 0;
#pragma unroll
      for (int u = 0; u < kSegVals; ++u) nxt[u] = seg[static_cast<size_t>(jn) * kSegVals + u];
      rk4_step_vjp_at<T>(K, C, dt, cur[0], cur[1], cur[2], cur + 3, l0, l1, l2, g);
#pragma unroll
      for (int u = 0; u < kSegVals; ++u) cur[u] = nxt[u];
    }
  }
  // chain rule to the parameter vector (binary64)
  double th[RRG_NPARAM];
  for (int i = 0; i < RRG_NPARAM; ++i) th[i] = 0.0;
  const double I = v;
  const double W_o2 = P[P_M_O2] * P[P_N_CELL] * I / (4.0 * P[P_FARADAY]);
  const double y_scale = P[P_X_O2] * P[P_K_SM] / W_o2;
  const double lam = P[P_LAM_REF], xo2 = P[P_X_O2], Kp = P[P_K_P];
  const double gamma = P[P_GAMMA];
  th[P_A_W] += g.a_w;
  th[P_A_P] += g.a_p;
  th[P_K_SM] += g.k_sm + static_cast<double>(g.y_scale) * y_scale / P[P_K_SM];
  th[P_K_CA] += g.k_ca;
  th[P_GAMMA] += static_cast<double>(g.e) / (gamma * gamma);
  {
    const double Ccp = P[P_C_P] * P[P_T_ATM] / P[P_ETA_CP], gc = g.C_cp;
    th[P_C_P] += gc * P[P_T_ATM] / P[P_ETA_CP];
    th[P_T_ATM] += gc * P[P_C_P] / P[P_ETA_CP];
    th[P_ETA_CP] += -gc * Ccp / P[P_ETA_CP];
  }
  {
    const double Cm = P[P_ETA_CM] * P[P_K_T] / P[P_R_CM], gc = g.C_m;
    th[P_ETA_CM] += gc * P[P_K_T] / P[P_R_CM];
    th[P_K_T] += gc * P[P_ETA_CM] / P[P_R_CM];
    th[P_R_CM] += -gc * Cm / P[P_R_CM];
  }
  th[P_K_V] += g.k_v;
  th[P_K_P] += g.K_p;
  {
    const double RTa = P[P_R_A] * P[P_T_ST] / P[P_V_CA], RTs = P[P_R_A] * P[P_T_ST] / P[P_V_SM];
    const double ga = g.RT_Vca, gs = g.RT_Vsm;
    th[P_R_A] += ga * P[P_T_ST] / P[P_V_CA] + gs * P[P_T_ST] / P[P_V_SM];
    th[P_T_ST] += ga * P[P_R_A] / P[P_V_CA] + gs * P[P_R_A] / P[P_V_SM];
    th[P_V_CA] += -ga * RTa / P[P_V_CA];
    th[P_V_SM] += -gs * RTs / P[P_V_SM];
  }
  th[P_J_CP] += -static_cast<double>(g.inv_J) / (P[P_J_CP] * P[P_J_CP]);
  // p_atm: through 1/p_atm and through q_0 = x_t - p_atm (pressures)
  th[P_P_ATM] += -static_cast<double>(g.inv_p_atm) / (P[P_P_ATM] * P[P_P_ATM]) -
                 static_cast<double>(l0) - static_cast<double>(l2);
  // candidate constants
  const double gV0 = g.V0, gy = g.y_scale;
  const double gW = static_cast<double>(g.W_o2) + gV0 * Kp * lam / xo2 - gy * y_scale / W_o2;
  th[P_M_O2] += gW * W_o2 / P[P_M_O2];
  th[P_N_CELL] += gW * W_o2 / P[P_N_CELL];
  th[P_FARADAY] += -gW * W_o2 / P[P_FARADAY];
  th[P_C0] += gV0;
  th[P_C1] += gV0 * I;
  th[P_C2] += gV0 * I * I;
  th[P_K_P] += gV0 * lam * W_o2 / xo2;
  th[P_LAM_REF] += gV0 * Kp * W_o2 / xo2;
  th[P_X_O2] += -gV0 * Kp * lam * W_o2 / (xo2 * xo2) + gy * y_scale / xo2;
  const double dI = gW * W_o2 / I + gV0 * (P[P_C1] + 2.0 * P[P_C2] * I);
  out[0] = dI * (r - v_prev);
  out[1] = l0;
  out[2] = l1;
  out[3] = l2;
  // theta'_p = theta_p m_p^{k*}: back to the nominal parameters
  for (int i = 0; i < RRG_NPARAM; ++i)
    out[4 + i] = L.pmul ? th[i] * L.pmul[static_cast<size_t>(k) * RRG_NPARAM + i] : th[i];
}

}  // namespace

// Host side.  launch_adjoint_forward enqueues the forward pass and the
// argmin for the m candidate slots the last candidate set-up prepared
// (kappas in cand_kappa); launch_adjoint_reverse the reverse sweeps of slots
// slot0 .. slot0 + count - 1 on the states the forward pass saved.
// ckpt: m N (H / checkpoint + 1) 3 doubles; lane_min / lane_arg: m N each;
// seg: m (H + 1) 12 values of T; d_out: m kOutStride doubles (per slot: g,
// k*, j*, then dg/dkappa, dg/dx_t, dg/dtheta).  fwd_begin / fwd_end (either
// may be null): events around the forward kernel.  The binary32 gradient
// reads the stored binary32 disturbances when the handle draws them (the
// values its binary32 rollouts use), otherwise the binary64 array (filled by
// the caller) rounded to binary32.
namespace {
bool reads32(const Launch& L, bool fp64) { return !fp64 && L.precision != RRG_FP64 && !L.scen_gen; }
}  // namespace

cudaError_t launch_adjoint_forward(const Launch& L, bool fp64, int m, int checkpoint, double* ckpt,
                                   double* lane_min, int* lane_arg, double* d_out,
                                   cudaEvent_t fwd_begin, cudaEvent_t fwd_end, bool argmin) {
  // one warp per block until blocks of 128 threads would fill every SM:
  // each scenario is one dependent chain, so spreading them over SMs costs
  // nothing
  if (L.sms <= 0 || m < 1) return cudaErrorInvalidConfiguration;
  const long long lanes = static_cast<long long>(L.N) * m;
  const int threads = (lanes >= 128LL * L.sms) ? 128 : 32;
  const dim3 grid((L.N + threads - 1) / threads, m);
  if (fwd_begin) {
    const cudaError_t er = cudaEventRecord(fwd_begin, L.stream);
    if (er != cudaSuccess) return er;
  }
  if (fp64)
    adjoint_forward_kernel<double, double><<<grid, threads, 0, L.stream>>>(L, L.d64, checkpoint, ckpt,
                                                                           lane_min, lane_arg);
  else if (reads32(L, fp64))
    adjoint_forward_kernel<float, float><<<grid, threads, 0, L.stream>>>(L, L.d32, checkpoint, ckpt,
                                                                         lane_min, lane_arg);
  else
    adjoint_forward_kernel<float, double><<<grid, threads, 0, L.stream>>>(L, L.d64, checkpoint, ckpt,
                                                                          lane_min, lane_arg);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (fwd_end) {
    e = cudaEventRecord(fwd_end, L.stream);
    if (e != cudaSuccess) return e;
  }
  if (argmin) adjoint_argmin_kernel<<<m, 256, 0, L.stream>>>(lane_min, lane_arg, L.N, d_out);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_reverse(const Launch& L, bool fp64, int slot0, int count, int checkpoint,
                                   const double* ckpt, void* seg, double* d_out, const double* lane_min,
                                   const int* lane_arg) {
  if (count < 1 || slot0 < 0) return cudaErrorInvalidConfiguration;
  if (fp64)
    adjoint_reverse_kernel<double, double><<<count, kRevThreads, 0, L.stream>>>(
        L, L.d64, checkpoint, ckpt, static_cast<double*>(seg), d_out, slot0, lane_min, lane_arg);
  else if (reads32(L, fp64))
    adjoint_reverse_kernel<float, float><<<count, kRevThreads, 0, L.stream>>>(
        L, L.d32, checkpoint, ckpt, static_cast<float*>(seg), d_out, slot0, lane_min, lane_arg);
  else
    adjoint_reverse_kernel<float, double><<<count, kRevThreads, 0, L.stream>>>(
        L, L.d64, checkpoint, ckpt, static_cast<float*>(seg), d_out, slot0, lane_min, lane_arg);
  return cudaGetLastError();
}

}  // namespace rrg
