// rrg_error.cu -- the binary32 rollouts' error against binary64, per
// trajectory and per step (the quantity the FP32 + FP64-recheck rule of the
// binary32 modes rests on).
//
// The paper reports that single precision had no visible effect on its GPU
// governor (Sec. III-C) and leaves its accuracy open (Sec. V).  Here each
// trajectory (candidate i, scenario k) is integrated twice from the same
// start over the full horizon, with no early exit: once exactly as the
// binary32 rollouts do it (same constants, same right-hand side, the stored
// binary32 disturbances) and once as the binary64 rollouts and the recheck do
// it (binary64 disturbances, read or regenerated from their Philox counters).
// At every step j = 0..H the two slacks s32_j, s64_j are compared.  The
// recheck decides a lane in binary32 only where its slack lies outside the
// band [-eps, eps), so the rule is exact when, at every step, s32_j >= eps
// implies s64_j >= 0 and s32_j < -eps implies s64_j < 0; steps where that
// fails are counted as unsafe.  The rule holds with margin 1 / r when every
// step's error is below r max(eps, |s64_j|): the ratio of each step's error
// to max(eps, |s64_j|) is reported per trajectory (its maximum over j).
#include "rrg_internal.h"
#include "rrg_lane.cuh"

namespace rrg {

namespace {

__device__ __forceinline__ bool finite_d(double x) { return fabs(x) <= DBL_MAX; }

// |s32 - s64| with a non-finite slack on one side only counted as +inf (the
// two sides disagree on whether the state blew up) and on both sides as 0.
__device__ __forceinline__ double step_err(float s32, double s64) {
  const double a = static_cast<double>(s32);
  const bool f32 = finite_d(a), f64 = finite_d(s64);
  if (f32 && f64) return fabs(a - s64);
  return f32 == f64 ? 0.0 : inf_v<double>();
}

// err / max(band, |s64|): below 1 at every step, no step can be decided
// wrongly by the band rule.
__device__ __forceinline__ double step_ratio(double e, double s64, float band) {
  const double den = fmax(static_cast<double>(band), fabs(s64));
  if (!(den > 0.0)) return e > 0.0 ? inf_v<double>() : 0.0;
  return e / den;
}

// The recheck rule at one step: binary32 decides it (outside the band) and
// binary64 disagrees in sign.
__device__ __forceinline__ bool step_unsafe(float s32, double s64, float band) {
  if (s32 >= band) return !(s64 >= 0.0);
  if (s32 < -band) return s64 >= 0.0;
  return false;
}

template <bool PU>
__global__ void __launch_bounds__(128)
slack_error_kernel(const Launch L, float band, double* __restrict__ err, int32_t* __restrict__ j_err,
                   double* __restrict__ smin32, double* __restrict__ smin64,
                   int32_t* __restrict__ unsafe, double* __restrict__ ratio) {
  const int i = blockIdx.y;
  const int N = L.N, H = L.H;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const ScenSrc src = L.st->src[0];
  RhsU<float> K32 = L.u32;
  RhsC<float> C32 = L.cand_c32[i];
  RhsU<double> K64 = L.u64;
  RhsC<double> C64 = L.cand_c64[i];
  double p32 = L.params[P_P_ATM], p64 = p32;
  if constexpr (PU) {
    const double* mk = L.pmul + static_cast<size_t>(k) * RRG_NPARAM;
    p32 = scenario_model<float>(L.params, mk, L.cand_v[i], L.k64.pws, L.y_min, K32, C32);
    p64 = scenario_model<double>(L.params, mk, L.cand_v[i], L.k64.pws, L.y_min, K64, C64);
  }
  // starting states exactly as the rollouts of each precision form them
  float a_ca, a_w, a_sm, a_wa;
  double b_ca, b_w, b_sm, b_wa;
  start_state<float>(C32, L.st->x, p32, a_ca, a_w, a_sm, a_wa);
  start_state<double>(C64, L.st->x, p64, b_ca, b_w, b_sm, b_wa);
  const StepC<float> S32 = step_consts<float>(K32, static_cast<float>(L.dt));
  const StepC<double> S64 = step_consts<double>(K64, L.dt);

  float s32 = checked_slack<float>(C32, a_ca, a_w, a_sm);
  double s64 = checked_slack<double>(C64, b_ca, b_w, b_sm);
  double emax = step_err(s32, s64);
  int jmax = 0;
  float m32 = s32;
  double m64 = s64;
  int bad = step_unsafe(s32, s64, band) ? 1 : 0;
  double rmax = step_ratio(emax, s64, band);

  const size_t HN = static_cast<size_t>(H) * N;
  const bool gen = L.scen_gen != 0;
  const bool have64 = src.d64_valid != 0;
  const float sc0 = static_cast<float>(src.amp[0] * 0x1.0p-23),
              sc1 = static_cast<float>(src.amp[1] * 0x1.0p-23),
              sc2 = static_cast<float>(src.amp[2] * 0x1.0p-23);
  for (int j = 0; j < H; ++j) {
    const size_t q = static_cast<size_t>(j) * N + k;
    float e0, e1, e2;
    double f0, f1, f2;
    if (gen || !have64) {
      const U64x4 r = philox4x64_10(static_cast<uint64_t>(j), src.base + static_cast<uint64_t>(k), src.update,
                                    0ull, src.seed, 0ull);
      f0 = uniform_sym(r.w[0], src.amp[0]);
      f1 = uniform_sym(r.w[1], src.amp[1]);
      f2 = uniform_sym(r.w[2], src.amp[2]);
      if (gen) {
        e0 = uniform_sym32(r.w[0], sc0);
        e1 = uniform_sym32(r.w[1], sc1);
        e2 = uniform_sym32(r.w[2], sc2);
      } else {
        e0 = L.d32[q];
        e1 = L.d32[HN + q];
        e2 = L.d32[2 * HN + q];
      }
    } else {
      f0 = L.d64[q];
      f1 = L.d64[HN + q];
      f2 = L.d64[2 * HN + q];
      e0 = L.d32[q];
      e1 = L.d32[HN + q];
      e2 = L.d32[2 * HN + q];
    }
    rk4_step_fast<float>(K32, C32, S32, a_ca, a_w, a_sm, a_wa, e0, e1, e2);
    rk4_step_fast<double>(K64, C64, S64, b_ca, b_w, b_sm, b_wa, f0, f1, f2);
    s32 = checked_slack<float>(C32, a_ca, a_w, a_sm);
    s64 = checked_slack<double>(C64, b_ca, b_w, b_sm);
    const double e = step_err(s32, s64);
    if (e > emax) {
      emax = e;
      jmax = j + 1;
    }
    m32 = fminf(m32, s32);
    m64 = fmin(m64, s64);
    bad += step_unsafe(s32, s64, band) ? 1 : 0;
    rmax = fmax(rmax, step_ratio(e, s64, band));
  }
  const size_t o = static_cast<size_t>(i) * N + k;
  err[o] = emax;
  if (j_err) j_err[o] = jmax;
  if (smin32) smin32[o] = static_cast<double>(m32);
  if (smin64) smin64[o] = m64;
  if (unsafe) unsafe[o] = bad;
  if (ratio) ratio[o] = rmax;
}

}  // namespace

cudaError_t launch_slack_error(const Launch& L, int m, float band, double* err, int32_t* j_err,
                               double* smin32, double* smin64, int32_t* unsafe, double* ratio) {
  const dim3 grid((L.N + 127) / 128, m);
  if (L.pmul)
    slack_error_kernel<true><<<grid, 128, 0, L.stream>>>(L, band, err, j_err, smin32, smin64, unsafe,
                                                          ratio);
  else
    slack_error_kernel<false><<<grid, 128, 0, L.stream>>>(L, band, err, j_err, smin32, smin64, unsafe,
                                                           ratio);
  return cudaGetLastError();
}

}  // namespace rrg
