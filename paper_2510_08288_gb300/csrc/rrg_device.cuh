// rrg_device.cuh -- device-side building blocks of the robust reference
// governor: the FC3 closed-loop right-hand side and output, the RK4 step,
// the Philox4x64-10 scenario generator and order-preserving keys for
// atomic minima.  Included by rrg_kernels.cu only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rrg {

// ---------------------------------------------------------------------------
// Binomial series of x^e - 1 about c = 3/2, for binary64 (GB300's binary64
// pow has a dependent latency of about 5,800 cycles, this about 500): with
// t = x / c - 1, |t| <= 1/3 for x in [1, 2], and
//   x^e - 1 = (c^e - 1) + c^e sum_{n >= 1} binom(e, n) t^n,
// truncated after t^32 (the rest is below 3^-33 c^e / 33 < 1e-17), evaluated by
// Estrin's scheme.  Built on the host for one exponent (make_pow_series);
// another exponent or an x outside [1, 2] takes pow.
struct PowSeries {
  double e;      // the exponent the coefficients are for
  double inv_c;  // 1 / c
  double a[33];  // a[0] = c^e - 1, a[n] = c^e binom(e, n)
};

__device__ __forceinline__ double pow_m1_series(const PowSeries* __restrict__ S, double x,
                                                double e) {
  if (S != nullptr && S->e == e) {
    const double t = fma(x, S->inv_c, -1.0);
    if (fabs(t) <= 1.0 / 3.0) {
      const double* a = S->a;
      const double t2 = t * t, t4 = t2 * t2, t8 = t4 * t4, t16 = t8 * t8, t32 = t16 * t16;
      double p[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) p[i] = fma(a[2 * i + 1], t, a[2 * i]);
#pragma unroll
      for (int i = 0; i < 8; ++i) p[i] = fma(p[2 * i + 1], t2, p[2 * i]);
#pragma unroll
      for (int i = 0; i < 4; ++i) p[i] = fma(p[2 * i + 1], t4, p[2 * i]);
#pragma unroll
      for (int i = 0; i < 2; ++i) p[i] = fma(p[2 * i + 1], t8, p[2 * i]);
      return fma(a[32], t32, fma(p[1], t16, p[0]));
    }
  }
  return pow(x, e) - 1.0;
}

// ---------------------------------------------------------------------------
// FC3 constants.  The state is kept in gauge coordinates
//   q = [p_ca - p_atm, w_cp, p_sm - p_atm]
// so that the pressure differences that set every flow (and the output) are
// formed from numbers of the size of the differences, not of ~1e5 Pa: in
// binary32 this keeps about 3 more significant bits in the slack.  All
// constants are folded once per handle in binary64 and rounded once.
template <typename T>
struct Fc3K {
  T inv_p_atm;   // 1 / p_atm
  T a_w, a_p;    // compressor map W_cp = a_w w - a_p q_sm
  T k_sm, k_ca;  // orifice and outlet coefficients
  T e;           // (gamma - 1) / gamma
  T C_cp;        // c_p T_atm / eta_cp
  T C_m;         // eta_cm k_t / R_cm
  T k_v;         // back-EMF constant
  T K_p;         // controller gain on the air-flow error
  T RT_Vca;      // R_a T_st / V_ca
  T RT_Vsm;      // R_a T_st / V_sm
  T inv_J;       // 1 / J_cp
  const PowSeries* pws;  // binary64 x^e - 1 (device memory; nullptr: pow)
};

// Per-candidate constants (functions of the governed setpoint v = I only).
template <typename T>
struct CandK {
  T W_o2;     // O2 consumed, M_O2 n_cell I / (4 F)
  T V0;       // v_ff(I) + K_p W_ref(I): motor voltage at zero flow error
  T y_scale;  // x_O2 k_sm / W_o2: OER per pascal of p_sm - p_ca
};

// (1 + u)^e - 1, the compressor's isentropic temperature-ratio term: pow in
// binary64, the MUFU-based __powf in binary32.  (A degree-10 Chebyshev
// interpolant evaluated by Estrin's scheme was measured slower on GB300: a
// warp running one trajectory is issue-bound, and the polynomial costs more
// instructions than the two MUFU operations it would replace.)
template <typename T>
__device__ __forceinline__ T pow_e_m1(T e, T u, const PowSeries* S);

template <>
__device__ __forceinline__ double pow_e_m1<double>(double e, double u, const PowSeries* S) {
  return pow_m1_series(S, 1.0 + u, e);
}

template <>
__device__ __forceinline__ float pow_e_m1<float>(float e, float u, const PowSeries*) {
  return __powf(1.0f + u, e) - 1.0f;
}

template <typename T> __device__ __forceinline__ T div_fast(T a, T b);
template <> __device__ __forceinline__ float div_fast<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double div_fast<double>(double a, double b) { return a / b; }

// dq/dt of the FC3 closed loop (mass balances of the cathode and supply
// manifold, torque balance of the compressor shaft under a feed-forward +
// proportional air-flow controller).
template <typename T>
__device__ __forceinline__ void fc3_rhs(const Fc3K<T>& K, const CandK<T>& C,
                                        T q_ca, T w, T q_sm,
                                        T& d_ca, T& d_w, T& d_sm) {
  const T W_cp = K.a_w * w - K.a_p * q_sm;
  const T W_sm = K.k_sm * (q_sm - q_ca);
  const T W_ca = K.k_ca * q_ca;
  const T pr_e = pow_e_m1<T>(K.e, q_sm * K.inv_p_atm, K.pws);
  const T tau_cp = div_fast<T>(K.C_cp * pr_e * W_cp, w);
  const T tau_cm = K.C_m * ((C.V0 - K.K_p * W_cp) - K.k_v * w);
  d_ca = K.RT_Vca * (W_sm - W_ca - C.W_o2);
  d_w = (tau_cm - tau_cp) * K.inv_J;
  d_sm = K.RT_Vsm * (W_cp - W_sm);
}

// Oxygen excess ratio y = h(x, v).
template <typename T>
__device__ __forceinline__ T fc3_output(const CandK<T>& C, T q_ca, T q_sm) {
  return C.y_scale * (q_sm - q_ca);
}

// One classical RK4 step of size dt, in place.
template <typename T>
__device__ __forceinline__ void rk4_step(const Fc3K<T>& K, const CandK<T>& C, T dt,
                                         T& q_ca, T& w, T& q_sm) {
  const T h2 = T(0.5) * dt, h6 = dt / T(6);
  T a1, b1, c1, a2, b2, c2, a3, b3, c3, a4, b4, c4;
  fc3_rhs<T>(K, C, q_ca, w, q_sm, a1, b1, c1);
  fc3_rhs<T>(K, C, q_ca + h2 * a1, w + h2 * b1, q_sm + h2 * c1, a2, b2, c2);
  fc3_rhs<T>(K, C, q_ca + h2 * a2, w + h2 * b2, q_sm + h2 * c2, a3, b3, c3);
  fc3_rhs<T>(K, C, q_ca + dt * a3, w + dt * b3, q_sm + dt * c3, a4, b4, c4);
  q_ca += h6 * ((a1 + a4) + T(2) * (a2 + a3));
  w += h6 * ((b1 + b4) + T(2) * (b2 + b3));
  q_sm += h6 * ((c1 + c4) + T(2) * (c2 + c3));
}

// ---------------------------------------------------------------------------
// The same right-hand side with its constants multiplied out, for the
// rollouts (the equilibrium solve and the adjoint keep the form above), in
// deviation coordinates z = q - q_r about a reference point q_r of the
// candidate (its binary32 equilibrium; 0 gives the gauge form):
//   d_ca = RT_Vca (k_sm (p_sm - p_ca) - k_ca p_ca - W_o2)
//        = a1 z_sm - (a1 + a2) z_ca + c_ca
//   d_sm = RT_Vsm (W_cp - k_sm (p_sm - p_ca))
//        = RT_Vsm a_w z_w - (RT_Vsm a_p + b3) z_sm + b3 z_ca + c_sm
//   d_w  = (C_m (V0 - K_p W_cp - k_v w) - C_cp pr W_cp / w) / J
//        = (e0 - e2 z_w) - W_cp (e1 + e3 pr / w),
//   W_cp = a_w z_w - a_p z_sm + W_r,  w = w_r + z_w
// where c_ca, c_sm (the derivatives at q_r), W_r and e0 are folded in
// binary64 and rounded once.  Near the reference every binary32 term is of
// the size of the deviation, not of the ~1e4 Pa gauge pressures, so the
// state's rounding and the cancellations between the flow terms shrink with
// it (and the terms can be multiplied out without losing digits).  16
// instructions per evaluation in binary32 (3 of them MUFU), as many as the
// gauge form, plus five per step that carry the absolute speed w (see
// rk4_step_fast).
template <typename T>
struct RhsU {      // constants of the model (per scenario under parametric uncertainty)
  T a1, a12;       // RT_Vca k_sm, RT_Vca (k_sm + k_ca)
  T a_w, a_p;      // compressor map
  T b3;            // RT_Vsm k_sm
  T g_w, g_sm;     // RT_Vsm a_w, RT_Vsm a_p + b3
  T inv_p_atm, e;
  T e1, e2, e3;    // C_m K_p / J, C_m k_v / J, C_cp / J
  const PowSeries* pws;  // binary64 x^e - 1 (device memory; nullptr: pow)
};

template <typename T>
struct RhsC {    // constants of the candidate setpoint v (and the scenario's model)
  T c_ca;        // d_ca at q_r: a1 s_r - a2 ca_r - RT_Vca W_o2
  T c_sm;        // d_sm at q_r: RT_Vsm W_r - b3 s_r
  T W_r;         // compressor flow at q_r: a_w w_r - a_p sm_r
  T e0;          // C_m V0 / J - e2 w_r
  T x_r;         // 1 + sm_r / p_atm
  T y_scale;     // x_O2 k_sm / W_o2
  T s_off;       // slack at q_r: y_scale s_r - y_min
  T r_ca, r_w, r_sm;  // q_r (binary32 values, so both precisions share it)
};

// x^e - 1 for the compressor term, x = 1 + q_sm / p_atm formed by the caller.
template <typename T>
__device__ __forceinline__ T pow_m1(T x, T e, const PowSeries* S);
template <>
__device__ __forceinline__ double pow_m1<double>(double x, double e, const PowSeries* S) {
  return pow_m1_series(S, x, e);
}
template <>
__device__ __forceinline__ float pow_m1<float>(float x, float e, const PowSeries*) {
  return __powf(x, e) - 1.0f;
}

// The compressor torque factor f = e1 + e3 pr / w.  binary32: e3 pr is
// formed on the power term's path and the approximate reciprocal of w feeds
// the final multiply-add directly (w arrives last, from the previous stage's
// d_w); binary64: IEEE division.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <typename T> __device__ __forceinline__ T torque_factor(const RhsU<T>& U, T pr, T w);
template <>
__device__ __forceinline__ float torque_factor<float>(const RhsU<float>& U, float pr, float w) {
  return fmaf(U.e3 * pr, rcp_approx(w), U.e1);
}
template <>
__device__ __forceinline__ double torque_factor<double>(const RhsU<double>& U, double pr, double w) {
  return U.e1 + (U.e3 / w) * pr;
}

// x_pw = x_r + z_sm / p_atm and the absolute speed w = w_r + z_w are passed
// in: the caller forms both from the previous stage's derivatives directly
// (x_pw + (h / p_atm) d_sm, w + h d_w), one dependent operation shorter than
// through the stage state.  The terms with z_w, the component that arrives
// last, are added last.
template <typename T>
__device__ __forceinline__ void fc3_rhs_fast(const RhsU<T>& U, const RhsC<T>& C, T z_ca, T z_w,
                                             T z_sm, T w, T x_pw, T& d_ca, T& d_w, T& d_sm) {
  d_ca = U.a1 * z_sm + (C.c_ca - U.a12 * z_ca);
  d_sm = U.g_w * z_w + ((C.c_sm + U.b3 * z_ca) - U.g_sm * z_sm);
  const T W_cp = U.a_w * z_w + (C.W_r - U.a_p * z_sm);
  const T f = torque_factor<T>(U, pow_m1<T>(x_pw, U.e, U.pws), w);
  d_w = (C.e0 - U.e2 * z_w) - W_cp * f;
}

// Step-size constants of rk4_step_fast, formed once per trajectory (the
// division dt / 6 is not left to the compiler to hoist out of the loop).
template <typename T>
struct StepC {
  T dt, h2, h6, g2, g1;  // dt, dt / 2, dt / 6, dt / (2 p_atm), dt / p_atm
};
template <typename T>
__device__ __forceinline__ StepC<T> step_consts(const RhsU<T>& U, T dt) {
  StepC<T> S;
  S.dt = dt;
  S.h2 = T(0.5) * dt;
  S.h6 = dt / T(6);
  S.g2 = S.h2 * U.inv_p_atm;
  S.g1 = dt * U.inv_p_atm;
  return S;
}

// One RK4 step of size dt followed by the disturbance (e_ca, e_w, e_sm) of
// Eq. 4, in place, on the deviation z = (q_ca, w, q_sm) - q_r.  w_abs is the
// absolute compressor speed w_r + w that the torque term divides by: it is
// re-derived from the deviation every step ((p_w + w_r) + h/6 k4 next to
// p_w + h/6 k4), so it never drifts from it by more than a rounding, and the
// stage points form it from the previous stage's d_w in one operation.  (A
// first-order update of one reciprocal per step would not do: in the largest
// FC3 transients w moves by up to 20 % within half a step.)  The update is
// summed as ((z + e) + h/6 (k1 + 2 (k2 + k3))) + h/6 k4, so only one
// operation follows the last stage.
template <typename T>
__device__ __forceinline__ void rk4_step_fast(const RhsU<T>& U, const RhsC<T>& C, const StepC<T>& S,
                                              T& q_ca, T& w, T& q_sm, T& w_abs, T e_ca, T e_w,
                                              T e_sm) {
  const T dt = S.dt, h2 = S.h2, h6 = S.h6, g2 = S.g2, g1 = S.g1;
  const T x1 = q_sm * U.inv_p_atm + C.x_r;
  T a1, b1, c1, a2, b2, c2, a3, b3, c3, a4, b4, c4;
  fc3_rhs_fast<T>(U, C, q_ca, w, q_sm, w_abs, x1, a1, b1, c1);
  fc3_rhs_fast<T>(U, C, q_ca + h2 * a1, w + h2 * b1, q_sm + h2 * c1, w_abs + h2 * b1, x1 + g2 * c1,
                  a2, b2, c2);
  fc3_rhs_fast<T>(U, C, q_ca + h2 * a2, w + h2 * b2, q_sm + h2 * c2, w_abs + h2 * b2, x1 + g2 * c2,
                  a3, b3, c3);
  const T p_ca = (q_ca + e_ca) + h6 * (a1 + T(2) * (a2 + a3));
  const T p_w = (w + e_w) + h6 * (b1 + T(2) * (b2 + b3));
  const T p_sm = (q_sm + e_sm) + h6 * (c1 + T(2) * (c2 + c3));
  const T p_wa = p_w + C.r_w;
  fc3_rhs_fast<T>(U, C, q_ca + dt * a3, w + dt * b3, q_sm + dt * c3, w_abs + dt * b3, x1 + g1 * c3,
                  a4, b4, c4);
  q_ca = p_ca + h6 * a4;
  w = p_w + h6 * b4;
  q_sm = p_sm + h6 * c4;
  w_abs = p_wa + h6 * b4;
}

template <typename T>
__device__ __forceinline__ void rk4_step_fast(const RhsU<T>& U, const RhsC<T>& C, T dt, T& q_ca,
                                              T& w, T& q_sm, T& w_abs, T e_ca, T e_w, T e_sm) {
  rk4_step_fast<T>(U, C, step_consts<T>(U, dt), q_ca, w, q_sm, w_abs, e_ca, e_w, e_sm);
}

// ---------------------------------------------------------------------------
// Philox4x64-10, written from Salmon et al., "Parallel random numbers: as easy
// as 1, 2, 3" (SC'11): per round two 64x64 -> 128-bit products, words
// permuted and xored with the key; the key advances by a Weyl sequence.
struct U64x4 { uint64_t w[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                               uint64_t c3, uint64_t k0, uint64_t k1) {
  constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ull, kM1 = 0xCA5A826395121157ull;
  constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ull, kW1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += kW0; k1 += kW1; }
    const uint64_t hi0 = __umul64hi(kM0, c0), lo0 = kM0 * c0;
    const uint64_t hi1 = __umul64hi(kM1, c2), lo1 = kM1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  U64x4 o;
  o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
  return o;
}

// a (2u - 1) with u the top 53 bits of w scaled to [0, 1).  2u - 1 equals
// t 2^-52 exactly for the integer t = (w >> 11) - 2^52, and a 2^-52 is exact,
// so (a 2^-52) t rounds the same real number once: one conversion and one
// binary64 multiply instead of four operations on GB300's narrow FP64 pipe.
// (For a below 2^-960, a 2^-52 would lose bits to underflow; such tiny
// half-ranges take the four-operation form.)
__device__ __forceinline__ double uniform_sym(uint64_t w, double a) {
  if (a < 0x1.0p-960) {
    const double u = __dmul_rn(static_cast<double>(w >> 11), 0x1.0p-53);
    return __dmul_rn(a, __dsub_rn(__dmul_rn(2.0, u), 1.0));
  }
  const long long t = static_cast<long long>(w >> 11) - (1ll << 52);
  return __dmul_rn(__ll2double_rn(t), __dmul_rn(a, 0x1.0p-52));
}

// a (2u - 1) in binary32 from the top 24 bits of w, with a_scaled = a 2^-23:
// RN32((w >> 40) - 2^23) a 2^-23).  Within a 2^-23 plus one binary32 rounding
// of the binary64 value above, and without binary64 arithmetic.
__device__ __forceinline__ float uniform_sym32(uint64_t w, float a_scaled) {
  const int t = static_cast<int>(w >> 40) - (1 << 23);
  return __fmul_rn(__int2float_rn(t), a_scaled);
}

// ---------------------------------------------------------------------------
// Order-preserving 64-bit key of a double (for atomicMin); NaN must be mapped
// by the caller.
__device__ __forceinline__ unsigned long long dkey(double x) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dunkey(unsigned long long k) {
  return (k >> 63) ? __longlong_as_double(static_cast<long long>(k & 0x7FFFFFFFFFFFFFFFull))
                   : __longlong_as_double(static_cast<long long>(~k));
}

// Eq. 2 evaluated as written, without fused multiply-add.
__device__ __forceinline__ double governed(double v_prev, double r, double kappa) {
  return __dadd_rn(v_prev, __dmul_rn(kappa, __dsub_rn(r, v_prev)));
}

}  // namespace rrg
