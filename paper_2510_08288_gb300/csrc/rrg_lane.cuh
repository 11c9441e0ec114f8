// rrg_lane.cuh -- device code shared by the single-problem kernels
// (rrg_kernels.cu) and the batched kernels (rrg_batch.cu): the trajectory
// loop with its constraint check, the binary64 re-run from Philox counters,
// the equilibrium solve of the steady-state check, per-scenario model
// constants and the k-section grids.
#pragma once

#include <cfloat>
#include <cmath>

#include "rrg_device.cuh"
#include "rrg_internal.h"

namespace rrg {

template <typename T> __device__ __forceinline__ T max_finite();
template <> __device__ __forceinline__ float max_finite<float>() { return FLT_MAX; }
template <> __device__ __forceinline__ double max_finite<double>() { return DBL_MAX; }
template <typename T> __device__ __forceinline__ T inf_v();
template <> __device__ __forceinline__ float inf_v<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double inf_v<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

// ---------------------------------------------------------------------------
// Equilibrium manifold (Sec. II-A).  At rest the cathode balance fixes the
// cathode gauge pressure from the air flow W, the orifice fixes the supply
// manifold pressure and the compressor map the speed, leaving the shaft
// torque balance g(W) = 0, with g decreasing in W and g(W_o2) > 0.  The root
// lies close to the controller's target flow W_ref = lam_ref W_o2 / x_O2, so
// a secant iteration started there converges in a handful of binary64
// evaluations; every iterate is kept inside a sign-change bracket and a
// step that leaves it is replaced by bisection.
template <typename T>
__device__ __forceinline__ T eq_torque(const Fc3K<T>& K, const CandK<T>& C, T inv_k_ca, T inv_k_sm, T a_p,
                       T inv_a_w, T W, T q[3]) {
  q[0] = (W - C.W_o2) * inv_k_ca;
  q[2] = q[0] + W * inv_k_sm;
  q[1] = (W + a_p * q[2]) * inv_a_w;
  T a, b, c;
  fc3_rhs<T>(K, C, q[0], q[1], q[2], a, b, c);
  return b;
}

template <typename T> __device__ __forceinline__ T eq_tol();
template <> __device__ __forceinline__ double eq_tol<double>() { return 1e-15; }
// binary32: the screen only needs y_ss to about 1e-5 (it defers to binary64
// within 1e-4 of the threshold); a tighter stop can stall on rounding noise
// and run every iteration.
template <> __device__ __forceinline__ float eq_tol<float>() { return 1e-6f; }

// Returns 0 and the gauge state q, output *y_ss at the equilibrium, or < 0.
template <typename T>
__device__ __forceinline__ int equilibrium_from(const Fc3K<T>& K, const double* __restrict__ P,
                                                const CandK<double>& Cd, T q[3], T* y_ss) {
  CandK<T> C;
  C.W_o2 = static_cast<T>(Cd.W_o2);
  C.V0 = static_cast<T>(Cd.V0);
  C.y_scale = static_cast<T>(Cd.y_scale);
  // reciprocals in the solve's own precision (binary32 divisions in the
  // binary32 screen, none of GB300's slow binary64 ones)
  const T ikca = T(1) / K.k_ca, iksm = T(1) / K.k_sm;
  const T a_p = K.a_p, iaw = T(1) / K.a_w;
  const T big = static_cast<T>(1e30);
  T lo = C.W_o2;
  if (!(eq_torque<T>(K, C, ikca, iksm, a_p, iaw, lo, q) > T(0))) return -2;
  T hi = big;
  // two starting points around the target flow
  T x0 = static_cast<T>(P[P_LAM_REF] * Cd.W_o2 / P[P_X_O2]);
  T g0 = eq_torque<T>(K, C, ikca, iksm, a_p, iaw, x0, q);
  if (g0 > T(0)) lo = x0; else hi = x0;
  T x1 = x0 * (g0 > T(0) ? T(1.001) : T(0.999));
  T g1 = eq_torque<T>(K, C, ikca, iksm, a_p, iaw, x1, q);
  if (g1 > T(0)) { if (x1 > lo) lo = x1; } else if (x1 < hi) hi = x1;
  // make sure the bracket is closed before bisection can be needed
  for (int it = 0; it < 60 && hi == big; ++it) {
    const T xt = T(2) * lo;
    if (eq_torque<T>(K, C, ikca, iksm, a_p, iaw, xt, q) > T(0)) lo = xt; else hi = xt;
  }
  if (hi == big) return -2;
  T W = x1;
  for (int it = 0; it < 100; ++it) {
    T x2 = x1 - g1 * (x1 - x0) / (g1 - g0);
    if (!(x2 > lo && x2 < hi)) x2 = T(0.5) * (lo + hi);
    const T g2 = eq_torque<T>(K, C, ikca, iksm, a_p, iaw, x2, q);
    W = x2;
    if (g2 == T(0)) break;
    if (g2 > T(0)) lo = x2; else hi = x2;
    if (fabs(x2 - x1) <= eq_tol<T>() * x2 || hi - lo <= T(0.4) * eq_tol<T>() * hi) break;
    x0 = x1; g0 = g1;
    x1 = x2; g1 = g2;
  }
  eq_torque<T>(K, C, ikca, iksm, a_p, iaw, W, q);
  *y_ss = fc3_output<T>(C, q[0], q[2]);
  return 0;
}

// The same from the setpoint I alone.
template <typename T>
__device__ __forceinline__ int equilibrium_dev(const Fc3K<T>& K, const double* __restrict__ P,
                                               double I, T q[3], T* y_ss) {
  if (!(I > 0.0) || !(I <= DBL_MAX)) return -1;
  return equilibrium_from<T>(K, P, cand_consts(P, I), q, y_ss);
}

// Candidate set-up shared by the single-problem and batched searches: the
// binary32 equilibrium of setpoint v (Sec. II-A) is the reference point of
// the rollouts' deviation coordinates (0 when it cannot be found), the
// candidate's rollout constants are folded about it, and, when ss_check is
// set, the steady-state check of Eq. 3 (y_ss(v) >= thr_ss) is decided by it
// unless y_ss lands within 1e-4 of the threshold (its error is ~1e-6), in
// which case a binary64 solve decides.  Returns the check's outcome (1 when
// off).
__device__ __forceinline__ int candidate_setup(const Fc3K<double>& k64, const Fc3K<float>& k32,
                                               const double* __restrict__ P, double v, int ss_check,
                                               double thr_ss, double y_min, RhsC<double>* c64,
                                               RhsC<float>* c32) {
  const CandK<double> C = cand_consts(P, v);
  float q32[3] = {0.0f, 0.0f, 0.0f}, y32 = 0.0f;
  const bool v_ok = v > 0.0 && v <= DBL_MAX;
  const int rc32 = v_ok ? equilibrium_from<float>(k32, P, C, q32, &y32) : -1;
  double q_r[3] = {0.0, 0.0, 0.0};
  if (rc32 == 0 && fabsf(q32[0]) <= FLT_MAX && fabsf(q32[1]) <= FLT_MAX && fabsf(q32[2]) <= FLT_MAX) {
    q_r[0] = q32[0];
    q_r[1] = q32[1];
    q_r[2] = q32[2];
  }
  fold_rhs_cand(k64, C, q_r, y_min, c64, c32);
  if (!ss_check) return 1;
  if (rc32 == 0 && fabs(static_cast<double>(y32) - thr_ss) > 1e-4 * (1.0 + fabs(thr_ss)))
    return static_cast<double>(y32) >= thr_ss;
  double q[3], y_ss = 0.0;
  return v_ok && equilibrium_from<double>(k64, P, C, q, &y_ss) == 0 && y_ss >= thr_ss;
}

// Start of a trajectory: the deviation z = q - q_r of the absolute state x
// (pressures measured from p_atm), formed in binary64 and rounded once, and
// the absolute speed w_r + z_w that rk4_step_fast carries next to it.
template <typename T>
__device__ __forceinline__ void start_state(const RhsC<T>& C, const double* x, double p_atm, T& z_ca,
                                            T& z_w, T& z_sm, T& w_abs) {
  z_ca = static_cast<T>((x[0] - p_atm) - static_cast<double>(C.r_ca));
  z_w = static_cast<T>(x[1] - static_cast<double>(C.r_w));
  z_sm = static_cast<T>((x[2] - p_atm) - static_cast<double>(C.r_sm));
  w_abs = C.r_w + z_w;
}

// ---------------------------------------------------------------------------
// One trajectory: x_0 = x_t, x_{j+1} = RK4(x_j, v) + d_j, slack s_j =
// h(x_j, v) - y_min at j = 0..H; a non-finite state or output counts as
// s = -inf.  Stops when s < thr (thr = -inf: never) and, checked once per
// block of PF steps, when *dead is set.  Returns min_j s_j; *steps
// receives the RK4 steps done.
//
// The disturbances of step j are loaded PF steps ahead into a small
// register ring, so the L2 latency of the three loads (larger than one RK4
// step on a two-die GB300) overlaps the arithmetic of the steps in between.
// The candidate's dead flag is read at the start of a block and used at its
// end, for the same reason.
// Depth 16 in binary32 (measured on GB300: the closed-loop update ran 24 %
// faster than with 8, and the 65,536-scenario sweep was unchanged), 8 in
// binary64 (16 would spill the binary64 state and ring).
#ifndef RRG_PREFETCH
#define RRG_PREFETCH 16
#endif
#ifndef RRG_PREFETCH64
#define RRG_PREFETCH64 8
#endif
template <typename T> struct PrefetchDepth { static constexpr int value = RRG_PREFETCH; };
template <> struct PrefetchDepth<double> { static constexpr int value = RRG_PREFETCH64; };

// The slack y_j - y_min of the deviation state (y_min is folded into s_off).
template <typename T>
__device__ __forceinline__ T checked_slack(const RhsC<T>& C, T q_ca, T w, T q_sm) {
  const T s = C.y_scale * (q_sm - q_ca) + C.s_off;
  const bool fin = fabs(q_ca) <= max_finite<T>() && fabs(w) <= max_finite<T>() &&
                   fabs(q_sm) <= max_finite<T>() && fabs(s) <= max_finite<T>();
  return fin ? s : -inf_v<T>();
}

// a b + c rounded once; never simplified (x 0 + c is NaN for x = inf or NaN).
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Lane outcome of run_lane.
enum LaneEnd : int { LANE_REACHED_END = 0, LANE_VIOLATED = 1, LANE_STOPPED = 2 };

// Steps j0+1..j_end of one trajectory, from the state (q_ca, w, q_sm) at
// step j0 (updated in place); with j0 = 0 the output at step 0 is checked
// first (for j0 > 0 it was checked by the run that stopped there).  smin_in
// is the min slack so far.
//
// *jlast (in/out) bounds the last step whose slack was below `band`: it is
// raised to the end of each block of steps that had one (so it may overshoot
// the step by less than PF).  The binary64 recheck of a binary32 lane needs
// only steps 0..*jlast: every later step had a binary32 slack of at least the
// band, which the band's error bound makes non-negative in binary64.
// band = -inf tracks nothing.
template <typename T, int PF = PrefetchDepth<T>::value>
__device__ __forceinline__ T run_lane(const RhsU<T>& K, const RhsC<T>& C,
                                      const T* __restrict__ d, int k, int N, int H, int j0,
                                      int j_end, T& q_ca, T& w, T& q_sm, T& w_abs, T smin_in, T dt,
                                      T thr, const volatile int32_t* dead, unsigned* steps,
                                      int* end, T band, int* jlast) {
  T smin = smin_in;
  int j = j0;
  int jl = *jlast;
  int how = LANE_REACHED_END;
  bool go = j < j_end;
  if (j0 == 0) {
    const T s0 = checked_slack<T>(C, q_ca, w, q_sm);
    smin = fmin(smin, s0);
    if (s0 < band) jl = 0;
    if (s0 < thr) {
      how = LANE_VIOLATED;
      go = false;
    }
  }
  const StepC<T> S = step_consts<T>(K, dt);
  if (go) {
    const size_t HN = static_cast<size_t>(H) * N;
    T r0[PF], r1[PF], r2[PF];
    const T* pf = d + static_cast<size_t>(j0) * N + k;  // next step to prefetch
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      if (j0 + u < j_end) {
        r0[u] = __ldg(pf);
        r1[u] = __ldg(pf + HN);
        r2[u] = __ldg(pf + 2 * HN);
      } else {
        r0[u] = r1[u] = r2[u] = T(0);
      }
      pf += N;
    }
    bool stop = false;
    // Whole blocks of PF steps (PF = prefetch depth) run without a per-step exit branch: the
    // running min is tested once per block.  A lane that violates inside a
    // block runs to the block's end; that only lowers its min slack, so no
    // decision changes.  The last, partial block steps one at a time.
    //
    // Finiteness is also settled once per block: nf = sum of s_j 0 stays 0
    // while every slack is finite and turns NaN (for good) at the first that
    // is not; a non-finite state component is tested at the block's end,
    // since it contaminates every component through the next right-hand side
    // (every derivative reads W_cp or s) and NaN and inf never return to a
    // finite value through +, -, x and / by a finite or NaN operand.  Either
    // makes the lane's min slack -inf, as a per-step test would.
    while (!stop && j + PF <= j_end) {
      const int dead_now = dead != nullptr ? *dead : 0;
      T nf = T(0), bmin = inf_v<T>();
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const T e0 = r0[u], e1 = r1[u], e2 = r2[u];
        if (j + PF < j_end) {
          r0[u] = __ldg(pf);
          r1[u] = __ldg(pf + HN);
          r2[u] = __ldg(pf + 2 * HN);
        }
        pf += N;
        rk4_step_fast<T>(K, C, S, q_ca, w, q_sm, w_abs, e0, e1, e2);
        ++j;
        const T s = C.y_scale * (q_sm - q_ca) + C.s_off;
        bmin = fmin(bmin, s);
        nf = fma_rn(s, T(0), nf);
      }
      nf = fma_rn(q_ca, T(0), fma_rn(w, T(0), fma_rn(q_sm, T(0), nf)));
      if (nf != nf) bmin = -inf_v<T>();
      smin = fmin(smin, bmin);
      if (bmin < band) jl = j;
      if (smin < thr) {
        how = LANE_VIOLATED;
        stop = true;
      } else if (dead_now != 0 && j < j_end) {
        how = LANE_STOPPED;
        stop = true;
      }
    }
    const T* dp = d + static_cast<size_t>(j) * N + k;
    while (!stop && j < j_end) {
      const T e0 = __ldg(dp), e1 = __ldg(dp + HN), e2 = __ldg(dp + 2 * HN);
      dp += N;
      rk4_step_fast<T>(K, C, S, q_ca, w, q_sm, w_abs, e0, e1, e2);
      ++j;
      const T s = checked_slack<T>(C, q_ca, w, q_sm);
      smin = fmin(smin, s);
      if (s < band) jl = j;
      if (s < thr) {
        how = LANE_VIOLATED;
        stop = true;
      }
    }
  }
  *steps = static_cast<unsigned>(j - j0);
  *end = how;
  *jlast = jl;
  return smin;
}

// ---------------------------------------------------------------------------
// Two trajectories of one scenario k -- candidates A and B, the same
// disturbances -- in one thread: each step's three disturbance loads, the
// ring's addressing and the loop's bookkeeping serve both, and the two step
// chains are independent work for the scheduler.  Same arithmetic as
// run_lane for each trajectory: the decisions, and the min slack of a
// trajectory that does not violate, equal run_lane's bit for bit (a
// violating one may be integrated a little longer, so its min slack, an upper
// bound either way, can come out lower).
//
// From step 0 (its slack checked first: a violation there runs nothing in
// pair) over whole blocks of PF steps while
// neither candidate has been stopped: a trajectory that violates keeps being
// integrated with its partner (its min slack only falls, so no decision
// changes) and, when dead_X is given, marks its candidate dead at once, so
// the stop reaches every lane together at a block end (read at the block's
// start, as in run_lane) instead of splitting the warp.  Without dead flags
// (no candidate-level exit) a lane leaves the pair when either trajectory
// has violated.  The survivor then finishes alone in run_lane from the
// step reached; the last, partial block too.  z_X[4] = (q_ca, w, q_sm,
// w_abs) in and out; smin, steps, end, jlast per trajectory as run_lane's.
// Returns the steps both trajectories ran together.
template <typename T, int PF = PrefetchDepth<T>::value>
__device__ __forceinline__ int run_lane_pair(const RhsU<T>& K, const RhsC<T>& CA, const RhsC<T>& CB,
                                              const T* __restrict__ d, int k, int N, int H, int j_end,
                                              T* za, T* zb, T dt, T thr, T band,
                                              volatile int32_t* deadA, volatile int32_t* deadB,
                                              T* smin, unsigned* steps, int* end, int* jlast) {
  smin[0] = checked_slack<T>(CA, za[0], za[1], za[2]);
  smin[1] = checked_slack<T>(CB, zb[0], zb[1], zb[2]);
  jlast[0] = smin[0] < band ? 0 : -1;
  jlast[1] = smin[1] < band ? 0 : -1;
  int how[2] = {smin[0] < thr ? LANE_VIOLATED : LANE_REACHED_END,
                smin[1] < thr ? LANE_VIOLATED : LANE_REACHED_END};
  if (how[0] == LANE_VIOLATED && deadA != nullptr) *deadA = 1;
  if (how[1] == LANE_VIOLATED && deadB != nullptr) *deadB = 1;
  const bool cand_stop = deadA != nullptr;
  int j = 0;
  const StepC<T> S = step_consts<T>(K, dt);
  bool pair = how[0] == LANE_REACHED_END && how[1] == LANE_REACHED_END;
  bool stopA = false, stopB = false;  // candidate stopped (dead flag) while not violated
  if (pair && j + PF <= j_end) {
    const size_t HN = static_cast<size_t>(H) * N;
    T r0[PF], r1[PF], r2[PF];
    const T* pf = d + k;
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      r0[u] = __ldg(pf);
      r1[u] = __ldg(pf + HN);
      r2[u] = __ldg(pf + 2 * HN);
      pf += N;
    }
    while (pair && j + PF <= j_end) {
      const int dA = cand_stop ? *deadA : 0, dB = cand_stop ? *deadB : 0;
      T nfa = T(0), nfb = T(0), ba = inf_v<T>(), bb = inf_v<T>();
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const T e0 = r0[u], e1 = r1[u], e2 = r2[u];
        if (j + PF < j_end) {
          r0[u] = __ldg(pf);
          r1[u] = __ldg(pf + HN);
          r2[u] = __ldg(pf + 2 * HN);
        }
        pf += N;
        rk4_step_fast<T>(K, CA, S, za[0], za[1], za[2], za[3], e0, e1, e2);
        rk4_step_fast<T>(K, CB, S, zb[0], zb[1], zb[2], zb[3], e0, e1, e2);
        ++j;
        const T sa = CA.y_scale * (za[2] - za[0]) + CA.s_off;
        const T sb = CB.y_scale * (zb[2] - zb[0]) + CB.s_off;
        ba = fmin(ba, sa);
        bb = fmin(bb, sb);
        nfa = fma_rn(sa, T(0), nfa);
        nfb = fma_rn(sb, T(0), nfb);
      }
      nfa = fma_rn(za[0], T(0), fma_rn(za[1], T(0), fma_rn(za[2], T(0), nfa)));
      nfb = fma_rn(zb[0], T(0), fma_rn(zb[1], T(0), fma_rn(zb[2], T(0), nfb)));
      if (nfa != nfa) ba = -inf_v<T>();
      if (nfb != nfb) bb = -inf_v<T>();
      smin[0] = fmin(smin[0], ba);
      smin[1] = fmin(smin[1], bb);
      if (ba < band) jlast[0] = j;
      if (bb < band) jlast[1] = j;
      if (how[0] == LANE_REACHED_END && smin[0] < thr) {
        how[0] = LANE_VIOLATED;
        if (cand_stop) *deadA = 1;
      }
      if (how[1] == LANE_REACHED_END && smin[1] < thr) {
        how[1] = LANE_VIOLATED;
        if (cand_stop) *deadB = 1;
      }
      if (cand_stop) {
        // a candidate's stop comes to every lane at once: from the flag
        stopA = dA != 0 && j < j_end;
        stopB = dB != 0 && j < j_end;
        pair = !stopA && !stopB;
        if (how[0] == LANE_VIOLATED && how[1] == LANE_VIOLATED) pair = false;
      } else {
        pair = how[0] == LANE_REACHED_END && how[1] == LANE_REACHED_END;
      }
    }
  }
  unsigned extra[2] = {0u, 0u};
  // each trajectory still running finishes alone
  if (how[0] == LANE_REACHED_END && stopA) how[0] = LANE_STOPPED;
  if (how[1] == LANE_REACHED_END && stopB) how[1] = LANE_STOPPED;
  if (how[0] == LANE_REACHED_END && j < j_end) {
    int e = LANE_REACHED_END;
    smin[0] = run_lane<T, PF>(K, CA, d, k, N, H, j, j_end, za[0], za[1], za[2], za[3], smin[0], dt, thr,
                              deadA, &extra[0], &e, band, &jlast[0]);
    how[0] = e;
  }
  if (how[1] == LANE_REACHED_END && j < j_end) {
    int e = LANE_REACHED_END;
    smin[1] = run_lane<T, PF>(K, CB, d, k, N, H, j, j_end, zb[0], zb[1], zb[2], zb[3], smin[1], dt, thr,
                              deadB, &extra[1], &e, band, &jlast[1]);
    how[1] = e;
  }
  steps[0] = static_cast<unsigned>(j) + extra[0];
  steps[1] = static_cast<unsigned>(j) + extra[1];
  end[0] = how[0];
  end[1] = how[1];
  return j;
}

// ---------------------------------------------------------------------------
// The same trajectory loop with the disturbances staged through a ring of D
// steps in shared memory, filled by cp.async (LDGSTS) D steps ahead.  The
// exit and finiteness tests come every B steps as in run_lane (the candidate's
// dead flag is read at the start of a block and used at the end of the next
// one, since the read queues behind the ring's fills), and the block's body
// is unrolled U steps at a time.  A warp that runs one trajectory alone on
// its scheduler issues its steps in order: the register ring's 16-step
// unrolled body then costs more than the ring's extra instructions, and
// shallower register rings expose the load latency.  Measured on GB300 with
// a single warp and the scenario array in DRAM: 332 cycles per step for the
// register ring at depth 16, 262 for this ring; in the 1,024-scenario closed
// loop the average rollout launch took 70.5 us with D = 32, B = 16, U = 8
// against 78.4 us with the register ring; on another box 69.1 us with
// B = 32 against 70.2 us with B = 16 (U = 16 with B = 16: 78.3, a body too
// large for the instruction cache).  Results equal run_lane's bit for
// bit (same arithmetic in the same order); a lane may run one block longer
// after its candidate died, which changes no decision.
//
// ring: this block's ring, ring[(3 s + c) blockDim.x + threadIdx.x] holds
// component c of the step in slot s; each thread uses only its own column.
#ifndef RRG_RING_DEPTH
#define RRG_RING_DEPTH 32
#endif
#ifndef RRG_RING_UNROLL
#define RRG_RING_UNROLL 8
#endif
#ifndef RRG_RING_BLOCK
#define RRG_RING_BLOCK 32
#endif
static_assert((RRG_RING_DEPTH & (RRG_RING_DEPTH - 1)) == 0, "ring depth: a power of two");
static_assert(RRG_RING_BLOCK % RRG_RING_UNROLL == 0, "block: a multiple of the unroll");

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gmem_src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int D = RRG_RING_DEPTH, int B = RRG_RING_BLOCK, int U = RRG_RING_UNROLL>
__device__ __forceinline__ float run_lane_ring(const RhsU<float>& K, const RhsC<float>& C,
                                               const float* __restrict__ d, int k, int N, int H,
                                               int j0, int j_end, float& q_ca, float& w,
                                               float& q_sm, float& w_abs, float smin_in, float dt,
                                               float thr, const volatile int32_t* dead,
                                               unsigned* steps, int* end, float band, int* jlast,
                                               float* ring) {
  float smin = smin_in;
  int j = j0;
  int jl = *jlast;
  int how = LANE_REACHED_END;
  bool go = j < j_end;
  if (j0 == 0) {
    const float s0 = checked_slack<float>(C, q_ca, w, q_sm);
    smin = fmin(smin, s0);
    if (s0 < band) jl = 0;
    if (s0 < thr) {
      how = LANE_VIOLATED;
      go = false;
    }
  }
  const StepC<float> S = step_consts<float>(K, dt);
  if (go) {
    const size_t HN = static_cast<size_t>(H) * N;
    const int bd = blockDim.x;
    float* my = ring + threadIdx.x;
    const float* pf = d + static_cast<size_t>(j0) * N + k;  // next step to fetch
    // one commit group per step (empty past j_end), so that waiting until at
    // most D - 1 groups are pending means the oldest step has landed
#pragma unroll 1
    for (int u = 0; u < D; ++u) {
      if (j0 + u < j_end) {
        cp_async4(my + (3 * u) * bd, pf);
        cp_async4(my + (3 * u + 1) * bd, pf + HN);
        cp_async4(my + (3 * u + 2) * bd, pf + 2 * HN);
      }
      cp_async_commit();
      pf += N;
    }
    int slot = 0;  // slot of step j
    bool stop = false;
    // the dead flag read at the start of a block is used at the end of the
    // next one: the read queues behind the block's ring fills
    int dead_prev = 0;
    while (!stop && j + B <= j_end) {
      const int dead_now = dead != nullptr ? *dead : 0;
      float nf = 0.0f, bmin = inf_v<float>();
#pragma unroll U
      for (int u = 0; u < B; ++u) {
        cp_async_wait<D - 1>();
        float* e = my + (3 * slot) * bd;
        const float e0 = e[0], e1 = e[bd], e2 = e[2 * bd];
        rk4_step_fast<float>(K, C, S, q_ca, w, q_sm, w_abs, e0, e1, e2);
        // the slot is free once its values are in registers: step j + D
        if (j + D < j_end) {
          cp_async4(e, pf);
          cp_async4(e + bd, pf + HN);
          cp_async4(e + 2 * bd, pf + 2 * HN);
        }
        cp_async_commit();
        pf += N;
        slot = (slot + 1) & (D - 1);
        ++j;
        const float s = C.y_scale * (q_sm - q_ca) + C.s_off;
        bmin = fmin(bmin, s);
        nf = fma_rn(s, 0.0f, nf);
      }
      nf = fma_rn(q_ca, 0.0f, fma_rn(w, 0.0f, fma_rn(q_sm, 0.0f, nf)));
      if (nf != nf) bmin = -inf_v<float>();
      smin = fmin(smin, bmin);
      if (bmin < band) jl = j;
      if (smin < thr) {
        how = LANE_VIOLATED;
        stop = true;
      } else if (dead_prev != 0 && j < j_end) {
        how = LANE_STOPPED;
        stop = true;
      }
      dead_prev = dead_now;
    }
    while (!stop && j < j_end) {
      cp_async_wait<D - 1>();
      float* e = my + (3 * slot) * bd;
      const float e0 = e[0], e1 = e[bd], e2 = e[2 * bd];
      rk4_step_fast<float>(K, C, S, q_ca, w, q_sm, w_abs, e0, e1, e2);
      if (j + D < j_end) {
        cp_async4(e, pf);
        cp_async4(e + bd, pf + HN);
        cp_async4(e + 2 * bd, pf + 2 * HN);
      }
      cp_async_commit();
      pf += N;
      slot = (slot + 1) & (D - 1);
      ++j;
      const float s = checked_slack<float>(C, q_ca, w, q_sm);
      smin = fmin(smin, s);
      if (s < band) jl = j;
      if (s < thr) {
        how = LANE_VIOLATED;
        stop = true;
      }
    }
    cp_async_wait<0>();  // nothing in flight into the ring when the lane ends
  }
  *steps = static_cast<unsigned>(j - j0);
  *end = how;
  *jlast = jl;
  return smin;
}

// ---------------------------------------------------------------------------
// The trajectory loop fed by the Tensor Memory Accelerator.  Each warp owns a
// two-stage ring of T-step chunks in shared memory; a chunk is one
// cp.async.bulk.tensor copy of the box (32 scenarios from the warp's first,
// T steps, 3 components) of the binary32 array [3][H][N], issued by lane 0
// and counted on the stage's mbarrier, so a step reads its three values with
// shared loads at fixed offsets instead of issuing three per-lane
// asynchronous copies, their commit and wait and the address arithmetic.
// Scenarios and steps of a box beyond the array are filled with zeros by the
// copy (the ragged last warp, the last chunk).
//
// The warp walks the chunks together: the copies serve every lane, so a lane
// that has stopped keeps its place, does no arithmetic, and the chunk loop
// ends once no lane runs.  Per trajectory the arithmetic is run_lane's in the
// same order, so the min slack and the decisions equal it bit for bit; the
// exit and finiteness tests come at each whole chunk's end (the last, partial
// chunk steps one at a time with run_lane's per-step test); the candidate's
// dead flag is read at a chunk's start and used at its end, and a lane that
// violates marks `mark` at once.  on = false: the lane only keeps the warp
// company (inactive scenario, or finished in an earlier segment).
//
// Waits are bounded.  A stage whose copy has not landed after kTmaWaitLimit
// polls or kTmaWaitNs of the global timer ends the loop for the whole warp: the call counts one timeout in
// *timeouts and every lane still running reports a violation (min slack
// -inf, so no candidate is accepted on data that did not arrive).  Before
// returning, the warp waits (bounded again) for every copy it issued, so
// nothing lands in shared memory after the block has left.
//
// stages: the warp's 2 * 3 * T * 32 floats (128-byte aligned); bars: its two
// mbarriers.  Called by all 32 lanes of the warp.
#ifndef RRG_TMA_CHUNK
#define RRG_TMA_CHUNK 16
#endif
constexpr int kTmaChunk = RRG_TMA_CHUNK;
constexpr int kTmaStageFloats = 3 * kTmaChunk * 32;
constexpr unsigned kTmaStageBytes = kTmaStageFloats * 4u;
constexpr int kTmaWaitLimit = 1 << 22;          // polls
constexpr unsigned long long kTmaWaitNs = 100000000ull;  // and at most 0.1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
// Makes the initialised barriers visible to the asynchronous proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's (and, after a warp barrier, the warp's) generic-proxy
// shared-memory accesses before the asynchronous proxy's next writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Polls until the phase of the given parity has completed, at most
// kTmaWaitLimit times and kTmaWaitNs of the global timer; false if it has
// not.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int it = 1; it < kTmaWaitLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 0 && global_ns() - t0 > kTmaWaitNs) return false;
  }
  return false;
}
// Chunk copy: box (x = k0, y = j, z = 0) of the tensor map into `dst`,
// completion counted on `bar` (lane 0 only).  tmap == nullptr (the test
// switch RRG_INJECT_TMA_NO_COPY): nothing is issued, so the stage's wait runs
// out.
__device__ __forceinline__ void tma_chunk(const void* tmap, uint32_t dst, uint32_t bar, int k0, int j) {
  if (tmap == nullptr) return;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kTmaStageBytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(k0), "r"(j), "r"(0), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float run_lane_tma(const RhsU<float>& K, const RhsC<float>& C, const void* tmap,
                                              int k0, bool on, int j0, int j_end, float& q_ca, float& w,
                                              float& q_sm, float& w_abs, float smin_in, float dt, float thr,
                                              const volatile int32_t* dead, volatile int32_t* mark,
                                              unsigned* steps, int* end, float band, int* jlast,
                                              float* stages, uint64_t* bars,
                                              unsigned long long* timeouts) {
  constexpr int T = kTmaChunk;
  const int lane = threadIdx.x & 31;
  float smin = smin_in;
  int j = j0;
  int jl = *jlast;
  int how = LANE_REACHED_END;
  bool run = on && j0 < j_end;
  if (on && j0 == 0) {
    const float s0 = checked_slack<float>(C, q_ca, w, q_sm);
    smin = fmin(smin, s0);
    if (s0 < band) jl = 0;
    if (s0 < thr) {
      how = LANE_VIOLATED;
      run = false;
      if (mark != nullptr) *mark = 1;
    }
  }
  const StepC<float> S = step_consts<float>(K, dt);
  const int nchunks = j_end > j0 ? (j_end - j0 + T - 1) / T : 0;
  if (nchunks > 0 && __any_sync(0xffffffffu, run)) {
    const uint32_t st0 = smem_u32(stages), bar0 = smem_u32(bars);
    if (lane == 0) {
      mbar_init(bar0, 1u);
      mbar_init(bar0 + 8u, 1u);
      fence_mbar_init();
    }
    __syncwarp();
    if (lane == 0) {
      tma_chunk(tmap, st0, bar0, k0, j0);
      if (nchunks > 1) tma_chunk(tmap, st0 + kTmaStageBytes, bar0 + 8u, k0, j0 + T);
    }
    int issued = nchunks > 1 ? 2 : 1;  // chunks whose copy was issued
    int waited = 0;                     // chunks whose copy has landed
    bool timed_out = false;
    for (int c = 0; c < nchunks; ++c) {
      const int sg = c & 1;
      const uint32_t bar = bar0 + 8u * static_cast<uint32_t>(sg);
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, static_cast<uint32_t>((c >> 1) & 1)));
      if (!ok) {
        timed_out = true;
        break;
      }
      waited = c + 1;
      const float* e = stages + sg * kTmaStageFloats + lane;
      const int nst = j_end - (j0 + c * T) < T ? j_end - (j0 + c * T) : T;
      const int dead_now = (run && dead != nullptr) ? *dead : 0;
      if (run) {
        if (nst == T) {
          float nf = 0.0f, bmin = inf_v<float>();
#pragma unroll
          for (int u = 0; u < T; ++u) {
            const float e0 = e[u * 32], e1 = e[(T + u) * 32], e2 = e[(2 * T + u) * 32];
            rk4_step_fast<float>(K, C, S, q_ca, w, q_sm, w_abs, e0, e1, e2);
            const float sl = C.y_scale * (q_sm - q_ca) + C.s_off;
            bmin = fmin(bmin, sl);
            nf = fma_rn(sl, 0.0f, nf);
          }
          j += T;
          nf = fma_rn(q_ca, 0.0f, fma_rn(w, 0.0f, fma_rn(q_sm, 0.0f, nf)));
          if (nf != nf) bmin = -inf_v<float>();
          smin = fmin(smin, bmin);
          if (bmin < band) jl = j;
          if (smin < thr) {
            how = LANE_VIOLATED;
            run = false;
            if (mark != nullptr) *mark = 1;
          } else if (dead_now != 0 && j < j_end) {
            how = LANE_STOPPED;
            run = false;
          }
        } else {
          for (int u = 0; u < nst && run; ++u) {
            const float e0 = e[u * 32], e1 = e[(T + u) * 32], e2 = e[(2 * T + u) * 32];
            rk4_step_fast<float>(K, C, S, q_ca, w, q_sm, w_abs, e0, e1, e2);
            ++j;
            const float sl = checked_slack<float>(C, q_ca, w, q_sm);
            smin = fmin(smin, sl);
            if (sl < band) jl = j;
            if (sl < thr) {
              how = LANE_VIOLATED;
              run = false;
              if (mark != nullptr) *mark = 1;
            }
          }
        }
      }
      if (!__any_sync(0xffffffffu, run)) break;
      // every lane is done reading this stage: refill it with chunk c + 2
      __syncwarp();
      if (c + 2 < nchunks) {
        if (lane == 0) {
          fence_proxy_async_smem();
          tma_chunk(tmap, st0 + static_cast<uint32_t>(sg) * kTmaStageBytes, bar, k0, j0 + (c + 2) * T);
        }
        issued = c + 3;
      }
    }
    // nothing may land after the warp leaves: wait for the copies issued and
    // not yet waited for
    bool drained = true;
    for (int c = waited; c < issued; ++c)
      drained = mbar_wait_bounded(bar0 + 8u * static_cast<uint32_t>(c & 1),
                                  static_cast<uint32_t>((c >> 1) & 1)) && drained;
    drained = __all_sync(0xffffffffu, drained);
    if (timed_out || !drained) {
      if (lane == 0) atomicAdd(timeouts, 1ull);
      if (run) {
        smin = -inf_v<float>();
        how = LANE_VIOLATED;
        run = false;
      }
    }
    __syncwarp();
    if (lane == 0 && drained) {
      mbar_inval(bar0);
      mbar_inval(bar0 + 8u);
    }
  }
  *steps = static_cast<unsigned>(j - j0);
  *end = how;
  *jlast = jl;
  return smin;
}

// ---------------------------------------------------------------------------
// Two candidates of one scenario per thread on the TMA ring: the warp's chunk
// copies, waits and shared loads serve both trajectories, whose step chains
// are independent work for the scheduler (run_lane_pair's idea on
// run_lane_tma's ring).  Per trajectory the arithmetic, the chunk-end tests
// and the dead-flag handling are run_lane_tma's, so the decisions and the min
// slack of a trajectory that does not violate equal it bit for bit.  A chunk
// in which both trajectories of a lane run takes one body for both; one that
// has stopped leaves the other to a single-trajectory body.
struct TmaTraj {
  float q_ca, w, q_sm, w_abs;  // deviation state and absolute speed
  float smin;
  int jl, how, j;
  bool run;
};

__device__ __forceinline__ void tma_traj_start(TmaTraj& t, const RhsC<float>& C, bool on, int j0, int j_end,
                                               float thr, float band, volatile int32_t* mark) {
  t.j = j0;
  t.how = LANE_REACHED_END;
  t.run = on && j0 < j_end;
  if (on && j0 == 0) {
    const float s0 = checked_slack<float>(C, t.q_ca, t.w, t.q_sm);
    t.smin = fmin(t.smin, s0);
    if (s0 < band) t.jl = 0;
    if (s0 < thr) {
      t.how = LANE_VIOLATED;
      t.run = false;
      if (mark != nullptr) *mark = 1;
    }
  }
}

// The tests at the end of a whole chunk of T steps (run_lane_tma's).
__device__ __forceinline__ void tma_traj_chunk_end(TmaTraj& t, float bmin, float nf, int T, int j_end, float thr,
                                                   float band, int dead_now, volatile int32_t* mark) {
  t.j += T;
  nf = fma_rn(t.q_ca, 0.0f, fma_rn(t.w, 0.0f, fma_rn(t.q_sm, 0.0f, nf)));
  if (nf != nf) bmin = -inf_v<float>();
  t.smin = fmin(t.smin, bmin);
  if (bmin < band) t.jl = t.j;
  if (t.smin < thr) {
    t.how = LANE_VIOLATED;
    t.run = false;
    if (mark != nullptr) *mark = 1;
  } else if (dead_now != 0 && t.j < j_end) {
    t.how = LANE_STOPPED;
    t.run = false;
  }
}

// A whole chunk for one trajectory (e: the lane's column of the stage).
template <int T>
__device__ __forceinline__ void tma_traj_chunk(TmaTraj& t, const RhsU<float>& K, const RhsC<float>& C,
                                               const StepC<float>& S, const float* e, float& bmin, float& nf) {
#pragma unroll 8
  for (int u = 0; u < T; ++u) {
    const float e0 = e[u * 32], e1 = e[(T + u) * 32], e2 = e[(2 * T + u) * 32];
    rk4_step_fast<float>(K, C, S, t.q_ca, t.w, t.q_sm, t.w_abs, e0, e1, e2);
    const float sl = C.y_scale * (t.q_sm - t.q_ca) + C.s_off;
    bmin = fmin(bmin, sl);
    nf = fma_rn(sl, 0.0f, nf);
  }
}

// A whole chunk for both trajectories, one load of each value for the two.
template <int T>
__device__ __forceinline__ void tma_pair_chunk(TmaTraj& a, TmaTraj& b, const RhsU<float>& K,
                                               const RhsC<float>& CA, const RhsC<float>& CB,
                                               const StepC<float>& S, const float* e, float& bma, float& nfa,
                                               float& bmb, float& nfb) {
#pragma unroll 8
  for (int u = 0; u < T; ++u) {
    const float e0 = e[u * 32], e1 = e[(T + u) * 32], e2 = e[(2 * T + u) * 32];
    rk4_step_fast<float>(K, CA, S, a.q_ca, a.w, a.q_sm, a.w_abs, e0, e1, e2);
    rk4_step_fast<float>(K, CB, S, b.q_ca, b.w, b.q_sm, b.w_abs, e0, e1, e2);
    const float sa = CA.y_scale * (a.q_sm - a.q_ca) + CA.s_off;
    const float sb = CB.y_scale * (b.q_sm - b.q_ca) + CB.s_off;
    bma = fmin(bma, sa);
    bmb = fmin(bmb, sb);
    nfa = fma_rn(sa, 0.0f, nfa);
    nfb = fma_rn(sb, 0.0f, nfb);
  }
}

// The last, partial chunk: step by step with the per-step test (run_lane's).
__device__ __forceinline__ void tma_traj_tail(TmaTraj& t, const RhsU<float>& K, const RhsC<float>& C,
                                              const StepC<float>& S, const float* e, int T, int nst, float thr,
                                              float band, volatile int32_t* mark) {
  for (int u = 0; u < nst && t.run; ++u) {
    const float e0 = e[u * 32], e1 = e[(T + u) * 32], e2 = e[(2 * T + u) * 32];
    rk4_step_fast<float>(K, C, S, t.q_ca, t.w, t.q_sm, t.w_abs, e0, e1, e2);
    ++t.j;
    const float sl = checked_slack<float>(C, t.q_ca, t.w, t.q_sm);
    t.smin = fmin(t.smin, sl);
    if (sl < band) t.jl = t.j;
    if (sl < thr) {
      t.how = LANE_VIOLATED;
      t.run = false;
      if (mark != nullptr) *mark = 1;
    }
  }
}

// The chunk loop of run_lane_tma for two trajectories per lane (a: candidate
// A, b: candidate B; state, smin and jl in, everything out; steps = j - j0).
// dead_X / mark_X: the candidates' flags (nullptr without a candidate-level
// exit).  *paired: steps this lane ran for both trajectories at once.  Called
// by all 32 lanes of the warp.
__device__ __forceinline__ void run_lane_tma_pair(const RhsU<float>& K, const RhsC<float>& CA,
                                                  const RhsC<float>& CB, const void* tmap, int k0, bool onA,
                                                  bool onB, int j0, int j_end, TmaTraj& a, TmaTraj& b, float dt,
                                                  float thr, float band, const volatile int32_t* deadA,
                                                  const volatile int32_t* deadB, volatile int32_t* markA,
                                                  volatile int32_t* markB, float* stages, uint64_t* bars,
                                                  unsigned long long* timeouts, unsigned* paired) {
  constexpr int T = kTmaChunk;
  const int lane = threadIdx.x & 31;
  tma_traj_start(a, CA, onA, j0, j_end, thr, band, markA);
  tma_traj_start(b, CB, onB, j0, j_end, thr, band, markB);
  *paired = 0u;
  const StepC<float> S = step_consts<float>(K, dt);
  const int nchunks = j_end > j0 ? (j_end - j0 + T - 1) / T : 0;
  if (nchunks > 0 && __any_sync(0xffffffffu, a.run || b.run)) {
    const uint32_t st0 = smem_u32(stages), bar0 = smem_u32(bars);
    if (lane == 0) {
      mbar_init(bar0, 1u);
      mbar_init(bar0 + 8u, 1u);
      fence_mbar_init();
    }
    __syncwarp();
    if (lane == 0) {
      tma_chunk(tmap, st0, bar0, k0, j0);
      if (nchunks > 1) tma_chunk(tmap, st0 + kTmaStageBytes, bar0 + 8u, k0, j0 + T);
    }
    int issued = nchunks > 1 ? 2 : 1;
    int waited = 0;
    bool timed_out = false;
    for (int c = 0; c < nchunks; ++c) {
      const int sg = c & 1;
      const uint32_t bar = bar0 + 8u * static_cast<uint32_t>(sg);
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, static_cast<uint32_t>((c >> 1) & 1)));
      if (!ok) {
        timed_out = true;
        break;
      }
      waited = c + 1;
      const float* e = stages + sg * kTmaStageFloats + lane;
      const int nst = j_end - (j0 + c * T) < T ? j_end - (j0 + c * T) : T;
      const int da = (a.run && deadA != nullptr) ? *deadA : 0;
      const int db = (b.run && deadB != nullptr) ? *deadB : 0;
      if (nst == T) {
        float bma = inf_v<float>(), nfa = 0.0f, bmb = inf_v<float>(), nfb = 0.0f;
        if (a.run && b.run) {
          tma_pair_chunk<T>(a, b, K, CA, CB, S, e, bma, nfa, bmb, nfb);
          *paired += 2u * T;
          tma_traj_chunk_end(a, bma, nfa, T, j_end, thr, band, da, markA);
          tma_traj_chunk_end(b, bmb, nfb, T, j_end, thr, band, db, markB);
        } else if (a.run) {
          tma_traj_chunk<T>(a, K, CA, S, e, bma, nfa);
          tma_traj_chunk_end(a, bma, nfa, T, j_end, thr, band, da, markA);
        } else if (b.run) {
          tma_traj_chunk<T>(b, K, CB, S, e, bmb, nfb);
          tma_traj_chunk_end(b, bmb, nfb, T, j_end, thr, band, db, markB);
        }
      } else {
        tma_traj_tail(a, K, CA, S, e, T, nst, thr, band, markA);
        tma_traj_tail(b, K, CB, S, e, T, nst, thr, band, markB);
      }
      if (!__any_sync(0xffffffffu, a.run || b.run)) break;
      // every lane is done reading this stage: refill it with chunk c + 2
      __syncwarp();
      if (c + 2 < nchunks) {
        if (lane == 0) {
          fence_proxy_async_smem();
          tma_chunk(tmap, st0 + static_cast<uint32_t>(sg) * kTmaStageBytes, bar, k0, j0 + (c + 2) * T);
        }
        issued = c + 3;
      }
    }
    bool drained = true;
    for (int c = waited; c < issued; ++c)
      drained = mbar_wait_bounded(bar0 + 8u * static_cast<uint32_t>(c & 1),
                                  static_cast<uint32_t>((c >> 1) & 1)) && drained;
    drained = __all_sync(0xffffffffu, drained);
    if (timed_out || !drained) {
      if (lane == 0) atomicAdd(timeouts, 1ull);
      if (a.run) {
        a.smin = -inf_v<float>();
        a.how = LANE_VIOLATED;
        a.run = false;
      }
      if (b.run) {
        b.smin = -inf_v<float>();
        b.how = LANE_VIOLATED;
        b.run = false;
      }
    }
    __syncwarp();
    if (lane == 0 && drained) {
      mbar_inval(bar0);
      mbar_inval(bar0 + 8u);
    }
  }
}

// Disturbance component of Philox word w with half-range a: the binary32
// copy (top 24 bits, a 2^-23 folded in) or the binary64 value, exactly as the
// sampler stores them.
template <typename T> __device__ __forceinline__ T draw(uint64_t w, double a);
template <> __device__ __forceinline__ float draw<float>(uint64_t w, double a) {
  return uniform_sym32(w, static_cast<float>(a * 0x1.0p-23));
}
template <> __device__ __forceinline__ double draw<double>(uint64_t w, double a) {
  return uniform_sym(w, a);
}

// run_lane with the disturbances drawn from their Philox counters (j, k,
// update, 0) inside the loop instead of read from the stored array: the
// same values, so the same trajectory and decisions.  Same contract as
// run_lane.
template <typename T, int PF = PrefetchDepth<T>::value>
__device__ __forceinline__ T run_lane_gen(const RhsU<T>& K, const RhsC<T>& C, const ScenSrc& src,
                                          int k, int j0, int j_end, T& q_ca, T& w, T& q_sm,
                                          T& w_abs, T smin_in, T dt, T thr,
                                          const volatile int32_t* dead, unsigned* steps, int* end,
                                          T band, int* jlast) {
  T smin = smin_in;
  int j = j0;
  int jl = *jlast;
  int how = LANE_REACHED_END;
  bool go = j < j_end;
  if (j0 == 0) {
    const T s0 = checked_slack<T>(C, q_ca, w, q_sm);
    smin = fmin(smin, s0);
    if (s0 < band) jl = 0;
    if (s0 < thr) {
      how = LANE_VIOLATED;
      go = false;
    }
  }
  bool stop = !go;
  const StepC<T> S = step_consts<T>(K, dt);
  while (!stop && j + PF <= j_end) {
    const int dead_now = dead != nullptr ? *dead : 0;
    T nf = T(0), bmin = inf_v<T>();
#pragma unroll 4
    for (int u = 0; u < PF; ++u) {
      const U64x4 r = philox4x64_10(static_cast<uint64_t>(j), src.base + static_cast<uint64_t>(k), src.update,
                                    0ull, src.seed, 0ull);
      rk4_step_fast<T>(K, C, S, q_ca, w, q_sm, w_abs, draw<T>(r.w[0], src.amp[0]),
                       draw<T>(r.w[1], src.amp[1]), draw<T>(r.w[2], src.amp[2]));
      ++j;
      const T s = C.y_scale * (q_sm - q_ca) + C.s_off;
      bmin = fmin(bmin, s);
      nf = fma_rn(s, T(0), nf);
    }
    nf = fma_rn(q_ca, T(0), fma_rn(w, T(0), fma_rn(q_sm, T(0), nf)));
    if (nf != nf) bmin = -inf_v<T>();
    smin = fmin(smin, bmin);
    if (bmin < band) jl = j;
    if (smin < thr) {
      how = LANE_VIOLATED;
      stop = true;
    } else if (dead_now != 0 && j < j_end) {
      how = LANE_STOPPED;
      stop = true;
    }
  }
  while (!stop && j < j_end) {
    const U64x4 r = philox4x64_10(static_cast<uint64_t>(j), src.base + static_cast<uint64_t>(k), src.update, 0ull,
                                  src.seed, 0ull);
    rk4_step_fast<T>(K, C, S, q_ca, w, q_sm, w_abs, draw<T>(r.w[0], src.amp[0]),
                     draw<T>(r.w[1], src.amp[1]), draw<T>(r.w[2], src.amp[2]));
    ++j;
    const T s = checked_slack<T>(C, q_ca, w, q_sm);
    smin = fmin(smin, s);
    if (s < band) jl = j;
    if (s < thr) {
      how = LANE_VIOLATED;
      stop = true;
    }
  }
  *steps = static_cast<unsigned>(j - j0);
  *end = how;
  *jlast = jl;
  return smin;
}

// Scenario k's model under parametric uncertainty: the parameters theta_p
// m_p^k folded like the nominal ones, and the candidate constants at v about
// the reference point of the nominal candidate constants C comes in with
// (replaced on return).  Returns the scenario's p_atm (the origin of its
// gauge coordinates).
template <typename T>
__device__ __forceinline__ double scenario_model(const double* __restrict__ P,
                                                 const double* __restrict__ m_k, double v,
                                                 const PowSeries* pws, double y_min, RhsU<T>& U,
                                                 RhsC<T>& C) {
  const double q_r[3] = {static_cast<double>(C.r_ca), static_cast<double>(C.r_w),
                         static_cast<double>(C.r_sm)};
  double Pk[RRG_NPARAM];
#pragma unroll
  for (int p = 0; p < RRG_NPARAM; ++p) Pk[p] = __dmul_rn(P[p], m_k[p]);
  Fc3K<double> k64;
  Fc3K<float> k32;
  fold_constants(Pk, &k64, &k32);
  k64.pws = pws;  // used only if the scenario's exponent is the table's
  const CandK<double> c64 = cand_consts(Pk, v);
  RhsU<double> u64;
  RhsU<float> u32;
  RhsC<double> r64;
  RhsC<float> r32;
  fold_rhs(k64, &u64, &u32);
  fold_rhs_cand(k64, c64, q_r, y_min, &r64, &r32);
  if constexpr (sizeof(T) == 8) {
    U = u64;
    C = r64;
  } else {
    U = u32;
    C = r32;
  }
  return Pk[P_P_ATM];
}

// Warp minimum in the lane's own precision (a binary32 lane's value needs no
// binary64 shuffles or compares on GB300's narrow binary64 pipe).
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One binary64 trajectory whose disturbances are regenerated from their
// Philox counters step by step (the pair was sampled in a binary32 mode, so
// its binary64 array was never written).  Same contract as run_lane over
// steps 1..H with early exit at s < thr.
__device__ __forceinline__ double run_lane_philox(const RhsU<double>& K, const RhsC<double>& C,
                                  const ScenSrc& src, int k, int H, double q_ca, double w,
                                  double q_sm, double w_abs, double dt, double thr,
                                  unsigned* steps) {
  double smin = checked_slack<double>(C, q_ca, w, q_sm);
  int j = 0;
  const StepC<double> S = step_consts<double>(K, dt);
  if (!(smin < thr)) {
    while (j < H) {
      const U64x4 r = philox4x64_10(static_cast<uint64_t>(j), src.base + static_cast<uint64_t>(k), src.update,
                                    0ull, src.seed, 0ull);
      rk4_step_fast<double>(K, C, S, q_ca, w, q_sm, w_abs, uniform_sym(r.w[0], src.amp[0]),
                            uniform_sym(r.w[1], src.amp[1]), uniform_sym(r.w[2], src.amp[2]));
      ++j;
      const double s = checked_slack<double>(C, q_ca, w, q_sm);
      smin = fmin(smin, s);
      if (s < thr) break;
    }
  }
  *steps = static_cast<unsigned>(j);
  return smin;
}

// k-section grids (Alg. 3 / Eq. 5 for round 1; M points strictly inside the
// bracket for the later rounds).
__device__ __forceinline__ int grid_points(double* cand_kappa, int M) {
  for (int i = 0; i < M; ++i)
    cand_kappa[i] = __ddiv_rn(static_cast<double>(i), static_cast<double>(M - 1));
  return M;
}

__device__ __forceinline__ int interior_points(double* cand_kappa, int M, double lo, double hi) {
  const double w = __dsub_rn(hi, lo);
  for (int i = 0; i < M; ++i)
    cand_kappa[i] = __dadd_rn(lo, __ddiv_rn(__dmul_rn(w, static_cast<double>(i + 1)),
                                            static_cast<double>(M + 1)));
  return M;
}

// ---------------------------------------------------------------------------
// One step of the simulated plant at setpoint v (Fig. 1): x_{t+1} =
// RK4(x_t, v) + (e_ca, e_w, e_sm), the plant's own draw added after the step
// as in Eq. 4.  Binary64, with the rollouts' multiplied-out right-hand side
// and x^e - 1 series: the plant step sits on the closed loop's critical path,
// and a binary64 pow() costs thousands of cycles on GB300.
__device__ __forceinline__ void plant_step_fast(const Fc3K<double>& K, const RhsU<double>& U,
                                                const double* __restrict__ P, double dt, double v,
                                                const double x[3], double e_ca, double e_w,
                                                double e_sm, double x_next[3]) {
  RhsC<double> c64;
  RhsC<float> c32;
  const double q0[3] = {0.0, 0.0, 0.0};
  fold_rhs_cand(K, cand_consts(P, v), q0, 0.0, &c64, &c32);
  const double p_atm = P[P_P_ATM];
  double q_ca = x[0] - p_atm, w = x[1], q_sm = x[2] - p_atm, w_abs = x[1];
  rk4_step_fast<double>(U, c64, dt, q_ca, w, q_sm, w_abs, e_ca, e_w, e_sm);
  x_next[0] = q_ca + p_atm;
  x_next[1] = w;
  x_next[2] = q_sm + p_atm;
}

}  // namespace rrg
