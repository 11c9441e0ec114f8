// rrg_kernels.cu -- CUDA kernels of the robust reference governor update.
//
// One RG update (Alg. 3 and the bisection of Alg. 1/2, on the joint
// all-scenario predicate) is a fixed sequence of launches on one stream:
//
//   sample_kernel            d_j^k for all (j, k)            (Sec. II-C)
//   search_begin_kernel      round-1 candidates, v_i (Eq. 2), steady-state
//                            check y_ss(v_i) (Eq. 3)
//   { rollout_kernel<T, SRC> one thread per (candidate i, scenario k): RK4
//                            rollout with the output check at every step and
//                            early exit (Alg. 3 steps 2-3), warp AND / min of
//                            the per-trajectory results into per-candidate
//                            flags and min slack (Eq. 5 reduced on the device)
//     recheck_kernel         binary64 re-run of near-zero-slack trajectories
//     search_next_kernel  }  decide (Alg. 1 / Alg. 3 / k-section), build the
//                            next round's candidates or write the result
//
// Nothing returns to the host between rounds; the whole update can be
// captured in a CUDA graph.
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cudaTypedefs.h>

#include "rrg_device.cuh"
#include "rrg_internal.h"
#include "rrg_lane.cuh"

namespace rrg {

#ifndef RRG_ROLL_THREADS
#define RRG_ROLL_THREADS 128
#endif
constexpr int kRollThreads = RRG_ROLL_THREADS;
constexpr int kSearchThreads = 256;

__global__ void equilibrium_kernel(const double* __restrict__ P, const Fc3K<double> k64,
                                   double v, double* out4, int32_t* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double q[3], y = 0.0;
  const int rc = equilibrium_dev<double>(k64, P, v, q, &y);
  out4[0] = q[0] + P[P_P_ATM];
  out4[1] = q[1];
  out4[2] = q[2] + P[P_P_ATM];
  out4[3] = y;
  *status = rc;
}

cudaError_t launch_equilibrium(const Launch& L, double v, double* d_out4, int32_t* d_status) {
  equilibrium_kernel<<<1, 32, 0, L.stream>>>(L.params, L.k64, v, d_out4, d_status);
  return cudaGetLastError();
}

// One warp integrating `steps` binary32 RK4 steps of the rollout (the same
// right-hand side, constants, slack and finiteness accumulation as the
// trajectory loop, no disturbance) from the equilibrium of v, timed with the
// SM clock: the latency of the trajectory loop's dependent chain, the bound of
// a launch whose lanes each run alone on a scheduler.  out[0] = cycles per
// step, out[1] keeps the lanes' results alive; *status = the equilibrium's.
__global__ void __launch_bounds__(32)
step_latency_kernel(const Launch L, const RhsU<float> U, double v, int steps, double* out,
                    int32_t* status) {
  const CandK<double> Cd = cand_consts(L.params, v);
  RhsC<double> c64;
  RhsC<float> c32;
  float q[3] = {0.0f, 0.0f, 0.0f}, y = 0.0f;
  const int rc = equilibrium_from<float>(L.k32, L.params, Cd, q, &y);
  const double q_r[3] = {q[0], q[1], q[2]};
  fold_rhs_cand(L.k64, Cd, q_r, L.y_min, &c64, &c32);
  // deviation coordinates about the equilibrium, lanes slightly apart
  float q_ca = 1e-3f * static_cast<float>(threadIdx.x), w = 0.0f, q_sm = 0.0f, w_abs = c32.r_w;
  const StepC<float> S = step_consts<float>(U, static_cast<float>(L.dt));
  float smin = inf_v<float>(), nf = 0.0f;
  __syncwarp();
  const long long t0 = clock64();
#pragma unroll 8
  for (int j = 0; j < steps; ++j) {
    rk4_step_fast<float>(U, c32, S, q_ca, w, q_sm, w_abs, 0.0f, 0.0f, 0.0f);
    const float s = c32.y_scale * (q_sm - q_ca) + c32.s_off;
    smin = fminf(smin, s);
    nf = fma_rn(s, 0.0f, nf);
  }
  const long long t1 = clock64();
  float r = smin + nf + q_ca + w + q_sm + w_abs;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  if (threadIdx.x == 0) {
    out[0] = static_cast<double>(t1 - t0) / steps;
    out[1] = r;
    *status = rc;
  }
}

cudaError_t launch_step_latency(const Launch& L, double v, int steps, double* d_out2, int32_t* d_status) {
  step_latency_kernel<<<1, 32, 0, L.stream>>>(L, L.u32, v, steps, d_out2, d_status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Scenario sampling: one thread per (j, k), coalesced over k.
//
// binary64 values: d = a (2u - 1), u = (w >> 11) 2^-53 (bit-exact with the
// definition in rrg.h).  binary32 copy in the binary32 modes: from the top 24
// bits of the same word, d32 = RN32((u24 - 2^23) a 2^-23); it differs from
// the binary64 value by less than a 2^-23 plus one binary32 rounding, far
// inside the binary32 rollout's own error, and needs no binary64 arithmetic
// (GB300's binary64 pipe is narrow).

// Parametric uncertainty: multiplier m_p^k = 1 + rho (2u - 1) of parameter p
// in scenario k for every p set in mask (1 for the rest), u from word p % 4 of
// the Philox block at counter (p / 4, k, update, 2).
constexpr int kParamGroups = (RRG_NPARAM + 3) / 4;

__device__ __forceinline__ void sample_param_group(double* __restrict__ pm, uint64_t k, uint64_t kbase,
                                                   int g, uint64_t upd, uint64_t seed, double rho,
                                                   uint32_t mask) {
  const U64x4 w = philox4x64_10(static_cast<uint64_t>(g), kbase + k, upd, 2ull, seed, 0ull);
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int p = 4 * g + b;
    if (p < RRG_NPARAM)
      pm[k * RRG_NPARAM + p] = ((mask >> p) & 1u) ? __dadd_rn(1.0, uniform_sym(w.w[b], rho)) : 1.0;
  }
}

__global__ void sample_kernel(double* __restrict__ d64, float* __restrict__ d32,
                              double* __restrict__ d64b, float* __restrict__ d32b, int N, int H,
                              uint64_t seed, uint64_t base, const unsigned long long* t_dev,
                              double a0, double a1, double a2, int write64, int gen, SearchState* st,
                              double* __restrict__ pm, double* __restrict__ pmb, double rho,
                              uint32_t mask, uint64_t kbase) {
  const uint64_t upd = base + (t_dev ? *t_dev : 0ull);
  const int pair = (d64b != nullptr && (upd & 1ull)) ? 1 : 0;
  if (pair) {
    d64 = d64b;
    d32 = d32b;
    pm = pmb;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ScenSrc src;
    src.d64_valid = gen ? 0 : write64;
    src.pad = 0;
    src.seed = seed;
    src.update = upd;
    src.base = kbase;
    src.amp[0] = a0;
    src.amp[1] = a1;
    src.amp[2] = a2;
    st->src[pair] = src;
  }
  const size_t HN = static_cast<size_t>(H) * N;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  const float s0 = static_cast<float>(a0 * 0x1.0p-23), s1 = static_cast<float>(a1 * 0x1.0p-23),
              s2 = static_cast<float>(a2 * 0x1.0p-23);
  for (size_t q = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; !gen && q < HN;
       q += stride) {
    const uint64_t j = q / static_cast<uint64_t>(N), k = q - j * static_cast<uint64_t>(N);
    const U64x4 w = philox4x64_10(j, kbase + k, upd, 0ull, seed, 0ull);
    if (write64) {
      d64[q] = uniform_sym(w.w[0], a0);
      d64[HN + q] = uniform_sym(w.w[1], a1);
      d64[2 * HN + q] = uniform_sym(w.w[2], a2);
    } else {
      d32[q] = uniform_sym32(w.w[0], s0);
      d32[HN + q] = uniform_sym32(w.w[1], s1);
      d32[2 * HN + q] = uniform_sym32(w.w[2], s2);
    }
  }
  if (pm != nullptr) {
    const size_t G = static_cast<size_t>(N) * kParamGroups;
    for (size_t q = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < G; q += stride) {
      const uint64_t k = q / kParamGroups;
      sample_param_group(pm, k, kbase, static_cast<int>(q - k * kParamGroups), upd, seed, rho, mask);
    }
  }
}

static int grid_for(size_t n, int threads, int cap) {
  size_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > static_cast<size_t>(cap)) b = cap;
  return static_cast<int>(b);
}

cudaError_t launch_sample(const Launch& L, uint64_t seed, uint64_t base,
                          const unsigned long long* t_dev, const double* amp, bool dual,
                          cudaStream_t stream) {
  const size_t n = static_cast<size_t>(L.H) * L.N;
  const int write64 = L.precision == RRG_FP64 ? 1 : 0;
  // Full width also for the next closed-loop update's draw on the side
  // stream: it then finishes while the search's short kernels run.  (One
  // block per SM stretched it over the long rollout and slowed the update by
  // 7 %; stream priorities changed nothing, measured on GB300.)
  if (L.sms <= 0) return cudaErrorInvalidConfiguration;
  sample_kernel<<<grid_for(n, 256, L.sms * 16), 256, 0, stream ? stream : L.stream>>>(
      L.d64, L.d32, dual ? L.d64b : nullptr, dual ? L.d32b : nullptr, L.N, L.H, seed, base, t_dev,
      amp[0], amp[1], amp[2], write64, L.scen_gen, L.st, L.pmul, dual ? L.pmulb : nullptr, L.punc_rho,
      L.punc_mask, L.kbase);
  return cudaGetLastError();
}

__global__ void fill_kernel(double* __restrict__ a, size_t n, double v) {
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (size_t q = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < n; q += stride)
    a[q] = v;
}

cudaError_t launch_fill(const Launch& L, double* a, size_t n, double v) {
  if (L.sms <= 0) return cudaErrorInvalidConfiguration;
  fill_kernel<<<grid_for(n, 256, L.sms * 4), 256, 0, L.stream>>>(a, n, v);
  return cudaGetLastError();
}

// Writes pair 0's binary64 values from Philox when the pair was sampled in a
// binary32 mode (its binary64 array is then stale).
__global__ void materialize64_kernel(double* __restrict__ d64, int N, int H,
                                     const SearchState* st) {
  const ScenSrc src = st->src[0];
  if (src.d64_valid) return;
  const size_t HN = static_cast<size_t>(H) * N;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (size_t q = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < HN; q += stride) {
    const uint64_t j = q / static_cast<uint64_t>(N), k = q - j * static_cast<uint64_t>(N);
    const U64x4 w = philox4x64_10(j, src.base + k, src.update, 0ull, src.seed, 0ull);
    d64[q] = uniform_sym(w.w[0], src.amp[0]);
    d64[HN + q] = uniform_sym(w.w[1], src.amp[1]);
    d64[2 * HN + q] = uniform_sym(w.w[2], src.amp[2]);
  }
}

// Marks pair 0's binary64 array valid once every block of the fill is done
// (a separate launch: a block of the fill itself could not know that).
__global__ void mark64_kernel(SearchState* st) { st->src[0].d64_valid = 1; }

cudaError_t launch_materialize64(const Launch& L) {
  const size_t n = static_cast<size_t>(L.H) * L.N;
  if (L.sms <= 0) return cudaErrorInvalidConfiguration;
  materialize64_kernel<<<grid_for(n, 256, L.sms * 16), 256, 0, L.stream>>>(L.d64, L.N, L.H, L.st);
  mark64_kernel<<<1, 1, 0, L.stream>>>(L.st);
  return cudaGetLastError();
}

__global__ void round_scenarios_kernel(const double* __restrict__ d64, float* __restrict__ d32,
                                       size_t n, SearchState* st) {
  if (blockIdx.x == 0 && threadIdx.x == 0) st->src[0].d64_valid = 1;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (size_t q = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < n; q += stride)
    d32[q] = static_cast<float>(d64[q]);
}

cudaError_t launch_round_scenarios(const Launch& L) {
  const size_t n = L.scen_gen ? 0 : 3 * static_cast<size_t>(L.H) * L.N;
  if (L.sms <= 0) return cudaErrorInvalidConfiguration;
  round_scenarios_kernel<<<grid_for(n, 256, L.sms * 16), 256, 0, L.stream>>>(L.d64, L.d32, n, L.st);
  return cudaGetLastError();
}

// One thread per (candidate slot, scenario k); blockIdx.y picks the slot
// through the state's two segments.  classify = 1 is the binary32 pass of
// RRG_FP32_RECHECK: trajectories whose final min slack lies in [-eps, eps)
// are appended to the recheck list and decided later in binary64.  A
// SEG_PROBE lane that survives its probe steps saves its state and reports
// nothing yet; the SEG_CONTINUE lane of the next launch finishes it.  PU:
// parametric uncertainty, each lane folds its scenario's own model constants.
// Where a rollout lane takes its disturbances from.
enum RollSrc : int {
  SRC_REGS = 0,  // the stored array through a register prefetch ring (run_lane)
  SRC_RING = 1,  // the stored array through a shared-memory ring (run_lane_ring, binary32)
  SRC_GEN = 2,   // drawn from Philox inside the trajectory loop (run_lane_gen)
  SRC_TMA = 3    // the stored array through a per-warp TMA ring (run_lane_tma, binary32)
};

// Dynamic shared memory of the TMA-ring rollouts: per warp two stages of
// kTmaStageBytes, then per warp two mbarriers.
extern __shared__ __align__(1024) unsigned char rrg_dyn_smem[];
constexpr size_t kTmaSmemBytes =
    static_cast<size_t>(kRollThreads / 32) * (2 * kTmaStageBytes + 2 * sizeof(uint64_t));

// The lane's outcome for candidate slot i (called by every thread of the
// warp): classified against the recheck band in the binary32 + recheck mode
// (an undecided lane is listed for the binary64 recheck unless its candidate
// has already failed), its P entry, then the warp's AND of the flags, min
// slack and step count folded into the candidate's by one atomic each.
template <typename T>
__device__ __forceinline__ void reduce_lane(const Launch& L, int i, int k, int N, bool final_lane, T smin,
                                            unsigned steps, int jlast, int classify, T eps,
                                            volatile int32_t* dead) {
  bool lane_ok = true, uncertain = false;
  T contrib = inf_v<T>();
  if (final_lane) {
    if (classify) {
      if (smin >= eps) {
        contrib = smin;
      } else if (smin < -eps) {
        lane_ok = false;
        contrib = smin;
      } else {
        uncertain = true;
      }
    } else {
      lane_ok = smin >= T(0);
      contrib = smin;
    }
  }
  if (uncertain && *dead == 0) {
    const uint32_t slot = atomicAdd(L.recheck_count, 1u);
    L.recheck_list[slot] = static_cast<uint32_t>(i) * static_cast<uint32_t>(N) + static_cast<uint32_t>(k);
    L.recheck_jlast[slot] = static_cast<uint32_t>(jlast);
  }
  if (L.P != nullptr && final_lane) L.P[static_cast<size_t>(i) * N + k] = lane_ok ? 1 : 0;

  const bool all_ok = __all_sync(0xffffffffu, lane_ok);
  const T wmin = warp_min<T>(contrib);
  const unsigned wsteps = __reduce_add_sync(0xffffffffu, steps);
  if ((threadIdx.x & 31) == 0) {
    if (!all_ok) L.cand_ok[i] = 0;
    if (wmin < inf_v<T>()) atomicMin(L.cand_min + i, dkey(static_cast<double>(wmin)));
    if (wsteps) {
      atomicAdd(&L.stats->lane_steps, static_cast<unsigned long long>(wsteps));
      if (sizeof(T) == 8) atomicAdd(&L.stats->lane_steps_fp64, static_cast<unsigned long long>(wsteps));
    }
  }
}

template <typename T, bool PU, int SRC>
__device__ __forceinline__ void rollout_body(const Launch& L, const RhsU<T>& K0,
                                             const T* __restrict__ d_pair0,
                                             const T* __restrict__ d_pair1,
                                             const RhsC<T>* __restrict__ cand, int early_exit,
                                             int classify, const void* tm0 = nullptr,
                                             const void* tm1 = nullptr) {
  const T* __restrict__ d = L.st->buf ? d_pair1 : d_pair0;
  const Seg s0 = L.st->seg[0], s1 = L.st->seg[1];
  const int y = blockIdx.y;
  int mode, i;
  if (y < s0.count) {
    mode = s0.mode;
    i = mode == SEG_CONTINUE ? L.st->cont_slot[y] : s0.base + y;
  } else if (y - s0.count < s1.count) {
    mode = s1.mode;
    i = s1.base + (y - s0.count);
  } else {
    return;
  }
  const int N = L.N;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = k < N;
  if (!L.cand_ss[i]) {
    // steady-state check failed: the whole row of P is 0, no rollout
    if (L.P != nullptr && active) L.P[static_cast<size_t>(i) * N + k] = 0;
    return;
  }
  volatile int32_t* dead = L.cand_dead + i;
  const bool cand_stop = early_exit == RRG_EXIT_CANDIDATE;
  if (cand_stop) {
    // another block may already have found a violation; read once per warp so
    // the warp leaves (or stays) as a whole before the warp reductions below
    const int dead0 = __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 ? *dead : 0, 0);
    if (dead0) return;
  }
  RhsC<T> C = cand[i];
  RhsU<T> K = K0;
  const T eps = static_cast<T>(L.eps_abs);
  const T thr = early_exit != RRG_EXIT_NONE ? (classify ? -eps : T(0)) : -inf_v<T>();

  T smin = inf_v<T>();
  unsigned steps = 0;
  int jlast = -1;
  const T band = classify ? eps : -inf_v<T>();
  bool final_lane = active;  // this launch decides the lane
  // segment bounds (the same for every lane of the launch row)
  const int j_end = mode == SEG_PROBE ? L.probe_steps : L.H;
  const int j0 = mode == SEG_CONTINUE ? L.probe_steps : 0;
  LaneState<T>* ls = nullptr;
  T q_ca = T(0), w = T(0), q_sm = T(0), w_abs = T(0);  // the deviation from the candidate's reference point
  T smin0 = inf_v<T>();
  if (active) {
    if (mode != SEG_FULL) ls = static_cast<LaneState<T>*>(L.lane_state) + static_cast<size_t>(i) * N + k;
    double p_atm = L.params[P_P_ATM];
    if constexpr (PU)
      p_atm = scenario_model<T>(L.params,
                                (L.st->buf ? L.pmulb : L.pmul) + static_cast<size_t>(k) * RRG_NPARAM,
                                L.cand_v[i], L.k64.pws, L.y_min, K, C);
    start_state<T>(C, L.st->x, p_atm, q_ca, w, q_sm, w_abs);
    if (mode == SEG_CONTINUE) {
      const LaneState<T> st = *ls;
      if (st.status != 0) {
        final_lane = false;  // finished and reduced in the probe
      } else {
        q_ca = st.q[0];
        w = st.q[1];
        q_sm = st.q[2];
        w_abs = st.w_abs;
        smin0 = st.smin;
        jlast = st.jlast;
      }
    }
  }
  int end = LANE_REACHED_END;
  if constexpr (SRC == SRC_TMA) {
    // every lane of the warp takes part (the chunk copies serve the warp)
    static_assert(sizeof(T) == 4, "the TMA ring is binary32");
    const int wid = threadIdx.x >> 5;
    float* stages = reinterpret_cast<float*>(rrg_dyn_smem) + static_cast<size_t>(wid) * 2 * kTmaStageFloats;
    uint64_t* bars = reinterpret_cast<uint64_t*>(rrg_dyn_smem + (kRollThreads / 32) * 2 * kTmaStageBytes) +
                     2 * wid;
    const bool lane_runs = active && final_lane;
    const void* tm = (L.inject & RRG_INJECT_TMA_NO_COPY) ? nullptr : (L.st->buf ? tm1 : tm0);
    const T s_out = run_lane_tma(K, C, tm, k & ~31, lane_runs, j0, j_end, q_ca, w, q_sm,
                                 w_abs, smin0, static_cast<T>(L.dt), thr, cand_stop ? dead : nullptr,
                                 cand_stop ? dead : nullptr, &steps, &end, band, &jlast, stages, bars,
                                 &L.stats->wait_timeouts);
    if (lane_runs) smin = s_out;
    const unsigned wsteps = __reduce_add_sync(0xffffffffu, steps);
    if ((threadIdx.x & 31) == 0 && wsteps)
      atomicAdd(&L.stats->lane_steps_tma, static_cast<unsigned long long>(wsteps));
  } else if (active && final_lane) {
    if constexpr (SRC == SRC_GEN)
      smin = run_lane_gen<T>(K, C, L.st->src[L.st->buf], k, j0, j_end, q_ca, w, q_sm, w_abs, smin0,
                             static_cast<T>(L.dt), thr,
                             cand_stop ? dead : nullptr, &steps, &end, band, &jlast);
    else if constexpr (SRC == SRC_RING) {
      static_assert(sizeof(T) == 4, "the shared-memory ring is binary32");
      __shared__ float ring[RRG_RING_DEPTH * 3 * kRollThreads];
      smin = run_lane_ring(K, C, d, k, N, L.H, j0, j_end, q_ca, w, q_sm, w_abs, smin0,
                           static_cast<T>(L.dt), thr,
                           cand_stop ? dead : nullptr, &steps, &end, band, &jlast, ring);
    } else
      smin = run_lane<T>(K, C, d, k, N, L.H, j0, j_end, q_ca, w, q_sm, w_abs, smin0,
                         static_cast<T>(L.dt), thr,
                         cand_stop ? dead : nullptr, &steps, &end, band, &jlast);
  }
  if (active && final_lane) {
    if (cand_stop && smin < thr) *dead = 1;
    if (mode == SEG_PROBE) {
      LaneState<T> o;
      o.q[0] = q_ca;
      o.q[1] = w;
      o.q[2] = q_sm;
      o.w_abs = w_abs;
      o.smin = smin;
      o.status = end == LANE_REACHED_END ? 0 : 1;
      o.jlast = jlast;
      *ls = o;
      if (end == LANE_REACHED_END) final_lane = false;
    }
  }
  reduce_lane<T>(L, i, k, N, final_lane, smin, steps, jlast, classify, eps, dead);
}

// SRC: where the lanes take their disturbances from (RollSrc).
template <typename T, int SRC>
__global__ void __launch_bounds__(kRollThreads)
rollout_kernel(const Launch L, const RhsU<T> K, const T* __restrict__ d_pair0,
               const T* __restrict__ d_pair1, const RhsC<T>* __restrict__ cand, int early_exit,
               int classify) {
  rollout_body<T, false, SRC>(L, K, d_pair0, d_pair1, cand, early_exit, classify);
}

// Parametric uncertainty: the per-lane constants need about 30 more
// registers; the binary32 kernel is held to the register budget of
// RRG_PU_MIN_BLOCKS resident blocks per SM.  Measured on GB300 (65,536
// scenarios x 16 candidates x 5,000 steps): 4 blocks at 128 registers ran
// 7 % faster than 5 blocks at 96 registers with spills.
#ifndef RRG_PU_MIN_BLOCKS
#define RRG_PU_MIN_BLOCKS 4
#endif
template <typename T, int SRC>
__global__ void __launch_bounds__(kRollThreads, sizeof(T) == 4 ? RRG_PU_MIN_BLOCKS : 1)
rollout_pu_kernel(const Launch L, const RhsU<T> K, const T* __restrict__ d_pair0,
                  const T* __restrict__ d_pair1, const RhsC<T>* __restrict__ cand, int early_exit,
                  int classify) {
  rollout_body<T, true, SRC>(L, K, d_pair0, d_pair1, cand, early_exit, classify);
}

// Binary32 lanes through the per-warp TMA ring (launches that leave warp
// slots empty, as SRC_RING): the tensor maps of the two scenario pairs are
// kernel parameters, so a captured graph keeps them.
template <bool PU>
__global__ void __launch_bounds__(kRollThreads, PU ? RRG_PU_MIN_BLOCKS : 1)
rollout_tma_kernel(const Launch L, const RhsU<float> K, const float* __restrict__ d_pair0,
                   const float* __restrict__ d_pair1, const RhsC<float>* __restrict__ cand, int early_exit,
                   int classify, const __grid_constant__ CUtensorMap tm0,
                   const __grid_constant__ CUtensorMap tm1) {
  rollout_body<float, PU, SRC_TMA>(L, K, d_pair0, d_pair1, cand, early_exit, classify, &tm0, &tm1);
}

// Two candidates per thread (binary32, register ring): block row y runs the
// launch's rows 2y and 2y + 1 (the slots of the round's full-horizon
// segments; rounds with a pipelined probe are never paired) for the same
// scenarios, through run_lane_pair; a row whose candidate failed the
// steady-state check, or has already been stopped, leaves its partner to run
// alone.  Each candidate's lanes are reduced exactly as in rollout_body.
#ifndef RRG_PAIR_PU_MIN_BLOCKS
#define RRG_PAIR_PU_MIN_BLOCKS 2
#endif
#ifndef RRG_PAIR_MIN_BLOCKS
#define RRG_PAIR_MIN_BLOCKS 1
#endif
// Prefetch depth (and exit block) of a paired thread: each step issues two
// trajectories' instructions, so half the single lane's depth covers the same
// load latency with half the unrolled code.
#ifndef RRG_PAIR_PF
#define RRG_PAIR_PF 8
#endif
template <bool PU>
__global__ void __launch_bounds__(kRollThreads, PU ? RRG_PAIR_PU_MIN_BLOCKS : RRG_PAIR_MIN_BLOCKS)
rollout_pair_kernel(const Launch L, const RhsU<float> K0, const float* __restrict__ d_pair0,
                    const float* __restrict__ d_pair1, const RhsC<float>* __restrict__ cand, int early_exit,
                    int classify) {
  const float* __restrict__ d = L.st->buf ? d_pair1 : d_pair0;
  const Seg s0 = L.st->seg[0], s1 = L.st->seg[1];
  const int rows = s0.count + s1.count;
  const int ya = 2 * static_cast<int>(blockIdx.y), yb = ya + 1;
  if (ya >= rows) return;
  const int ia = ya < s0.count ? s0.base + ya : s1.base + (ya - s0.count);
  const int ib = yb >= rows ? -1 : (yb < s0.count ? s0.base + yb : s1.base + (yb - s0.count));
  const int N = L.N;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = k < N;
  const bool ssa = L.cand_ss[ia] != 0, ssb = ib >= 0 && L.cand_ss[ib] != 0;
  if (!ssa && L.P != nullptr && active) L.P[static_cast<size_t>(ia) * N + k] = 0;
  if (ib >= 0 && !ssb && L.P != nullptr && active) L.P[static_cast<size_t>(ib) * N + k] = 0;
  const bool cand_stop = early_exit == RRG_EXIT_CANDIDATE;
  volatile int32_t* deada = L.cand_dead + ia;
  volatile int32_t* deadb = L.cand_dead + (ib >= 0 ? ib : ia);
  // which candidates this warp runs (uniform: the flags are read by lane 0)
  bool runa = ssa, runb = ssb;
  if (cand_stop) {
    const int da = __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 && runa ? *deada : 0, 0);
    const int db = __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 && runb ? *deadb : 0, 0);
    runa = runa && !da;
    runb = runb && !db;
  }
  if (!runa && !runb) return;
  const float eps = static_cast<float>(L.eps_abs);
  const float thr = early_exit != RRG_EXIT_NONE ? (classify ? -eps : 0.0f) : -inf_v<float>();
  const float band = classify ? eps : -inf_v<float>();
  float sm[2] = {inf_v<float>(), inf_v<float>()};
  unsigned st[2] = {0u, 0u};
  int jl[2] = {-1, -1}, en[2] = {LANE_REACHED_END, LANE_REACHED_END};
  unsigned paired = 0;  // trajectory steps this lane ran two per thread
  if (active) {
    RhsU<float> K = K0;
    RhsC<float> CA = cand[ia], CB = cand[ib >= 0 ? ib : ia];
    double p_atm = L.params[P_P_ATM];
    if constexpr (PU) {
      const double* mk = (L.st->buf ? L.pmulb : L.pmul) + static_cast<size_t>(k) * RRG_NPARAM;
      if (runa) p_atm = scenario_model<float>(L.params, mk, L.cand_v[ia], L.k64.pws, L.y_min, K, CA);
      if (runb) p_atm = scenario_model<float>(L.params, mk, L.cand_v[ib], L.k64.pws, L.y_min, K, CB);
    }
    float za[4], zb[4];
    start_state<float>(CA, L.st->x, p_atm, za[0], za[1], za[2], za[3]);
    start_state<float>(CB, L.st->x, p_atm, zb[0], zb[1], zb[2], zb[3]);
    const float dt = static_cast<float>(L.dt);
    if (runa && runb) {
      paired = 2u * static_cast<unsigned>(run_lane_pair<float, RRG_PAIR_PF>(
                            K, CA, CB, d, k, N, L.H, L.H, za, zb, dt, thr, band, cand_stop ? deada : nullptr,
                            cand_stop ? deadb : nullptr, sm, st, en, jl));
    } else if (runa) {
      sm[0] = run_lane<float, RRG_PAIR_PF>(K, CA, d, k, N, L.H, 0, L.H, za[0], za[1], za[2], za[3],
                                           inf_v<float>(), dt, thr, cand_stop ? deada : nullptr, &st[0],
                                           &en[0], band, &jl[0]);
    } else {
      sm[1] = run_lane<float, RRG_PAIR_PF>(K, CB, d, k, N, L.H, 0, L.H, zb[0], zb[1], zb[2], zb[3],
                                           inf_v<float>(), dt, thr, cand_stop ? deadb : nullptr, &st[1],
                                           &en[1], band, &jl[1]);
    }
    if (cand_stop && runa && sm[0] < thr) *deada = 1;
    if (cand_stop && runb && sm[1] < thr) *deadb = 1;
  }
  if (runa) reduce_lane<float>(L, ia, k, N, active, sm[0], st[0], jl[0], classify, eps, deada);
  if (runb) reduce_lane<float>(L, ib, k, N, active, sm[1], st[1], jl[1], classify, eps, deadb);
  if (runa && runb) {
    const unsigned wp = __reduce_add_sync(0xffffffffu, paired);
    if ((threadIdx.x & 31) == 0 && wp) atomicAdd(&L.stats->lane_steps_paired, static_cast<unsigned long long>(wp));
  }
}

// Two candidates per thread on the TMA ring: block row y runs the launch's
// rows 2y and 2y + 1 (full-horizon segments only, as rollout_pair_kernel)
// for the same scenarios through run_lane_tma_pair; every lane of a warp
// takes part in the ring's copies and waits.  Each candidate's lanes are
// reduced as in rollout_body.
template <bool PU>
__global__ void __launch_bounds__(kRollThreads, PU ? RRG_PAIR_PU_MIN_BLOCKS : RRG_PAIR_MIN_BLOCKS)
rollout_tma_pair_kernel(const Launch L, const RhsU<float> K0, const RhsC<float>* __restrict__ cand,
                        int early_exit, int classify, const __grid_constant__ CUtensorMap tm0,
                        const __grid_constant__ CUtensorMap tm1) {
  const Seg s0 = L.st->seg[0], s1 = L.st->seg[1];
  const int rows = s0.count + s1.count;
  const int ya = 2 * static_cast<int>(blockIdx.y), yb = ya + 1;
  if (ya >= rows) return;
  const int ia = ya < s0.count ? s0.base + ya : s1.base + (ya - s0.count);
  const int ib = yb >= rows ? -1 : (yb < s0.count ? s0.base + yb : s1.base + (yb - s0.count));
  const int N = L.N;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = k < N;
  const bool ssa = L.cand_ss[ia] != 0, ssb = ib >= 0 && L.cand_ss[ib] != 0;
  if (!ssa && L.P != nullptr && active) L.P[static_cast<size_t>(ia) * N + k] = 0;
  if (ib >= 0 && !ssb && L.P != nullptr && active) L.P[static_cast<size_t>(ib) * N + k] = 0;
  const bool cand_stop = early_exit == RRG_EXIT_CANDIDATE;
  volatile int32_t* deada = L.cand_dead + ia;
  volatile int32_t* deadb = L.cand_dead + (ib >= 0 ? ib : ia);
  bool runa = ssa, runb = ssb;
  if (cand_stop) {
    const int da = __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 && runa ? *deada : 0, 0);
    const int db = __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 && runb ? *deadb : 0, 0);
    runa = runa && !da;
    runb = runb && !db;
  }
  if (!runa && !runb) return;
  const float eps = static_cast<float>(L.eps_abs);
  const float thr = early_exit != RRG_EXIT_NONE ? (classify ? -eps : 0.0f) : -inf_v<float>();
  const float band = classify ? eps : -inf_v<float>();
  TmaTraj a{}, b{};
  a.smin = b.smin = inf_v<float>();
  a.jl = b.jl = -1;
  RhsU<float> K = K0;
  RhsC<float> CA = cand[ia], CB = cand[ib >= 0 ? ib : ia];
  if (active) {
    double p_atm = L.params[P_P_ATM];
    if constexpr (PU) {
      const double* mk = (L.st->buf ? L.pmulb : L.pmul) + static_cast<size_t>(k) * RRG_NPARAM;
      if (runa) p_atm = scenario_model<float>(L.params, mk, L.cand_v[ia], L.k64.pws, L.y_min, K, CA);
      if (runb) p_atm = scenario_model<float>(L.params, mk, L.cand_v[ib], L.k64.pws, L.y_min, K, CB);
    }
    start_state<float>(CA, L.st->x, p_atm, a.q_ca, a.w, a.q_sm, a.w_abs);
    start_state<float>(CB, L.st->x, p_atm, b.q_ca, b.w, b.q_sm, b.w_abs);
  }
  const int wid = threadIdx.x >> 5;
  float* stages = reinterpret_cast<float*>(rrg_dyn_smem) + static_cast<size_t>(wid) * 2 * kTmaStageFloats;
  uint64_t* bars = reinterpret_cast<uint64_t*>(rrg_dyn_smem + (kRollThreads / 32) * 2 * kTmaStageBytes) + 2 * wid;
  const void* tm = (L.inject & RRG_INJECT_TMA_NO_COPY) ? nullptr : (L.st->buf ? &tm1 : &tm0);
  unsigned paired = 0;
  run_lane_tma_pair(K, CA, CB, tm, k & ~31, active && runa, active && runb, 0, L.H, a, b,
                    static_cast<float>(L.dt), thr, band, cand_stop ? deada : nullptr,
                    cand_stop ? deadb : nullptr, cand_stop ? deada : nullptr, cand_stop ? deadb : nullptr, stages,
                    bars, &L.stats->wait_timeouts, &paired);
  if (active && cand_stop) {
    if (runa && a.smin < thr) *deada = 1;
    if (runb && b.smin < thr) *deadb = 1;
  }
  const unsigned sa = active && runa ? static_cast<unsigned>(a.j) : 0u;
  const unsigned sb = active && runb ? static_cast<unsigned>(b.j) : 0u;
  if (runa) reduce_lane<float>(L, ia, k, N, active, a.smin, sa, a.jl, classify, eps, deada);
  if (runb) reduce_lane<float>(L, ib, k, N, active, b.smin, sb, b.jl, classify, eps, deadb);
  const unsigned wp = __reduce_add_sync(0xffffffffu, paired);
  const unsigned wt = __reduce_add_sync(0xffffffffu, sa + sb);
  if ((threadIdx.x & 31) == 0) {
    if (wp) atomicAdd(&L.stats->lane_steps_paired, static_cast<unsigned long long>(wp));
    if (wt) atomicAdd(&L.stats->lane_steps_tma, static_cast<unsigned long long>(wt));
  }
}

// RRG_PAIR_FILLED pairs a launch whose paired grid fills the SMs at least
// this many times over: a paired block does twice a single block's work, so
// a short grid ends in a long, half-empty last wave.  Measured on GB300
// (k-section updates, 16 candidates x 5,000 steps): 65,536 scenarios (9
// paired waves) 7.5 % faster with uncertain parameters, 3.6 % nominal;
// 32,768 (4.5 waves) 1 % faster and 3 % slower; 8,192 (1.1 waves) 22 %
// slower.
#ifndef RRG_PAIR_MIN_WAVES
#define RRG_PAIR_MIN_WAVES 6
#endif

// RRG_TMA_AUTO takes the TMA ring for binary32 launches on the stored array
// of at least this many warps per SM, ahead of the other rings and of
// pairing.  The TMA saves the per-step load instructions, which pays where
// many warps compete for issue; a warp running alone pays the chunk's wait,
// warp votes and fence on its dependency chain instead.  Measured on GB300
// (k-section sweep, 16 candidates x 5,000 steps, per update), TMA against the
// per-lane cp.async ring: 16,384 scenarios with uncertain parameters (54
// warps per SM) 6.28 against 6.75 ms, 8,192 (27) 4.46 against 4.53 ms, 4,096
// (13.5) 2.78 against 2.70 ms, 1,024 (3.4) 1.85 against 1.64 ms; the
// 1,024-scenario closed loop (8.8 warps per SM at launch, mostly single
// survivors) 2,743 against 2,927 updates/s.  Against the register ring and
// pairing on launches that fill the SMs: 65,536 parametric 21.8 ms against
// 23.9 (single) and 24.0 (paired), 32,768 10.9 against 11.8; nominal 65,536
// 27.5 against 30.4 and 30.2.
#ifndef RRG_TMA_MIN_WARPS_PER_SM
#define RRG_TMA_MIN_WARPS_PER_SM 24
#endif

cudaError_t launch_rollout(const Launch& L, int m_launch, bool use_fp64, int early_exit,
                           bool recheck_classify, bool allow_pair) {
  dim3 grid((L.N + kRollThreads - 1) / kRollThreads, m_launch);
  const int cls = recheck_classify ? 1 : 0;
  // Binary32 lanes on the stored array: the shared-memory ring when the
  // launch leaves most warp slots empty (each warp then runs its trajectory
  // alone on its scheduler, bound by the step's latency), the register ring
  // when it fills the SMs (bound by issue, where the ring's extra
  // instructions cost more than they save).  Thresholds measured on GB300:
  // nominal model, ring up to 16 warps per SM (the 1,024-scenario closed loop
  // ran 10 % faster, 8,192 x 16 candidates 3 % slower); parametric model
  // (more registers, fewer resident warps), up to 64 (16,384 x 16 candidates
  // 2-6 % faster, 65,536 x 16 6 % slower).
  if (L.sms <= 0) return cudaErrorInvalidConfiguration;
  const int sms = L.sms;
  const long long warps = static_cast<long long>(grid.x) * grid.y * (kRollThreads / 32);
  const bool ring = warps <= (L.pmul ? 64LL : 16LL) * sms;
  const long long pair_blocks = static_cast<long long>(grid.x) * ((m_launch + 1) / 2);
  const bool filled = !ring && L.pair == RRG_PAIR_FILLED &&
                      pair_blocks >= static_cast<long long>(RRG_PAIR_MIN_WAVES) *
                                         pair_blocks_per_sm(L.pmul != nullptr) * sms;
#define RRG_ROLLOUT(KERNEL, T, SRC, KK, D0, D1, CAND, CLS) \
  KERNEL<T, SRC><<<grid, kRollThreads, 0, L.stream>>>(L, KK, D0, D1, CAND, early_exit, CLS)
  if (use_fp64) {
    if (L.pmul) {
      if (L.scen_gen) RRG_ROLLOUT(rollout_pu_kernel, double, SRC_GEN, L.u64, L.d64, L.d64b, L.cand_c64, 0);
      else RRG_ROLLOUT(rollout_pu_kernel, double, SRC_REGS, L.u64, L.d64, L.d64b, L.cand_c64, 0);
    } else {
      if (L.scen_gen) RRG_ROLLOUT(rollout_kernel, double, SRC_GEN, L.u64, L.d64, L.d64b, L.cand_c64, 0);
      else RRG_ROLLOUT(rollout_kernel, double, SRC_REGS, L.u64, L.d64, L.d64b, L.cand_c64, 0);
    }
  } else if (!L.scen_gen && L.tmap != nullptr &&
             (L.tma == RRG_TMA_ALWAYS ||
              (L.tma == RRG_TMA_AUTO && warps >= static_cast<long long>(RRG_TMA_MIN_WARPS_PER_SM) * sms))) {
    // the TMA ring: one tensor copy per warp and chunk of steps (it takes
    // precedence over the register-ring pairing, which it beat where both
    // apply).  Two candidates per thread on it only with RRG_PAIR_ALWAYS:
    // measured on GB300 (65,536 x 16 candidates x 5,000 steps, per update)
    // 22.7 against 21.9 ms with uncertain parameters (the paired kernel holds
    // 3 blocks per SM at 150 registers), 27.9 against 27.6 ms nominal.
    const bool tpair = allow_pair && m_launch > 1 && L.tma_pair_bps > 0 && L.pair == RRG_PAIR_ALWAYS;
    if (tpair) {
      const dim3 g2(grid.x, (m_launch + 1) / 2);
      if (L.pmul)
        rollout_tma_pair_kernel<true><<<g2, kRollThreads, kTmaSmemBytes, L.stream>>>(
            L, L.u32, L.cand_c32, early_exit, cls, L.tmap[0], L.tmap[1]);
      else
        rollout_tma_pair_kernel<false><<<g2, kRollThreads, kTmaSmemBytes, L.stream>>>(
            L, L.u32, L.cand_c32, early_exit, cls, L.tmap[0], L.tmap[1]);
    } else if (L.pmul) {
      rollout_tma_kernel<true><<<grid, kRollThreads, kTmaSmemBytes, L.stream>>>(
          L, L.u32, L.d32, L.d32b, L.cand_c32, early_exit, cls, L.tmap[0], L.tmap[1]);
    } else {
      rollout_tma_kernel<false><<<grid, kRollThreads, kTmaSmemBytes, L.stream>>>(
          L, L.u32, L.d32, L.d32b, L.cand_c32, early_exit, cls, L.tmap[0], L.tmap[1]);
    }
  } else if (allow_pair && !L.scen_gen && m_launch > 1 && (L.pair == RRG_PAIR_ALWAYS || filled)) {
    // two candidates per thread (issue-bound launches: one load of each
    // disturbance and one loop's bookkeeping serve both)
    const dim3 g2(grid.x, (m_launch + 1) / 2);
    if (L.pmul)
      rollout_pair_kernel<true><<<g2, kRollThreads, 0, L.stream>>>(L, L.u32, L.d32, L.d32b, L.cand_c32,
                                                                   early_exit, cls);
    else
      rollout_pair_kernel<false><<<g2, kRollThreads, 0, L.stream>>>(L, L.u32, L.d32, L.d32b, L.cand_c32,
                                                                    early_exit, cls);
  } else {
    if (L.pmul) {
      if (L.scen_gen) RRG_ROLLOUT(rollout_pu_kernel, float, SRC_GEN, L.u32, L.d32, L.d32b, L.cand_c32, cls);
      else if (ring) RRG_ROLLOUT(rollout_pu_kernel, float, SRC_RING, L.u32, L.d32, L.d32b, L.cand_c32, cls);
      else RRG_ROLLOUT(rollout_pu_kernel, float, SRC_REGS, L.u32, L.d32, L.d32b, L.cand_c32, cls);
    } else {
      if (L.scen_gen) RRG_ROLLOUT(rollout_kernel, float, SRC_GEN, L.u32, L.d32, L.d32b, L.cand_c32, cls);
      else if (ring) RRG_ROLLOUT(rollout_kernel, float, SRC_RING, L.u32, L.d32, L.d32b, L.cand_c32, cls);
      else RRG_ROLLOUT(rollout_kernel, float, SRC_REGS, L.u32, L.d32, L.d32b, L.cand_c32, cls);
    }
  }
#undef RRG_ROLLOUT
  return cudaGetLastError();
}

// Binary64 re-run of the trajectories the binary32 pass could not decide,
// over steps 0..jlast of each (the later steps were decided in binary32).
__global__ void __launch_bounds__(64)
recheck_kernel(const Launch L, const RhsU<double> K0, int early_exit) {
  const uint32_t count = *L.recheck_count;
  const int N = L.N;
  const double p_atm = L.params[P_P_ATM];
  const double thr = early_exit != RRG_EXIT_NONE ? 0.0 : -inf_v<double>();
  const int buf = L.st->buf;
  const ScenSrc src = L.st->src[buf];
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    const uint32_t idx = L.recheck_list[e];
    const int j_end = min(static_cast<int>(L.recheck_jlast[e]), L.H);
    const int i = static_cast<int>(idx / static_cast<uint32_t>(N));
    const int k = static_cast<int>(idx - static_cast<uint32_t>(i) * static_cast<uint32_t>(N));
    // a failed candidate needs no more decisions, unless P asks for every entry
    if (L.P == nullptr && !L.cand_ok[i]) continue;
    unsigned steps = 0;
    double smin;
    RhsU<double> K = K0;
    RhsC<double> C = L.cand_c64[i];
    double p_atm_k = p_atm;
    const double* pm = buf ? L.pmulb : L.pmul;
    if (pm != nullptr)
      p_atm_k = scenario_model<double>(L.params, pm + static_cast<size_t>(k) * RRG_NPARAM,
                                       L.cand_v[i], L.k64.pws, L.y_min, K, C);
    double q_ca, w, q_sm, w_abs;
    start_state<double>(C, L.st->x, p_atm_k, q_ca, w, q_sm, w_abs);
    if (src.d64_valid) {
      int end = 0;
      int jl = -1;
      smin = run_lane<double>(K, C, buf ? L.d64b : L.d64, k, N, L.H, 0, j_end, q_ca, w, q_sm,
                              w_abs, inf_v<double>(), L.dt, thr, nullptr, &steps, &end,
                              -inf_v<double>(), &jl);
    } else {
      smin = run_lane_philox(K, C, src, k, j_end, q_ca, w, q_sm, w_abs, L.dt, thr, &steps);
    }
    const bool ok = smin >= 0.0;
    if (!ok) L.cand_ok[i] = 0;
    if (L.P != nullptr) L.P[static_cast<size_t>(i) * N + k] = ok ? 1 : 0;
    atomicMin(L.cand_min + i, dkey(smin));
    atomicAdd(&L.stats->lane_steps, static_cast<unsigned long long>(steps));
    atomicAdd(&L.stats->lane_steps_fp64, static_cast<unsigned long long>(steps));
    atomicAdd(&L.stats->rechecked, 1ull);
  }
}

// ---- host-side set-up of the rollout kernels ------------------------------
// The shared-memory limit is a per-device attribute of the kernels: set once
// for each device a handle is created on.
bool tma_ring_prepare() {
  constexpr int kDevices = 64;
  static std::atomic<int> state[kDevices];  // 0 not yet, 1 set, 2 refused
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) return false;
  const int st = state[dev].load();
  if (st != 0) return st == 1;
  const int sm = static_cast<int>(kTmaSmemBytes);
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const bool ok = cudaFuncSetAttribute(rollout_tma_kernel<false>, a, sm) == cudaSuccess &&
                  cudaFuncSetAttribute(rollout_tma_kernel<true>, a, sm) == cudaSuccess &&
                  cudaFuncSetAttribute(rollout_tma_pair_kernel<false>, a, sm) == cudaSuccess &&
                  cudaFuncSetAttribute(rollout_tma_pair_kernel<true>, a, sm) == cudaSuccess;
  state[dev].store(ok ? 1 : 2);
  return ok;
}

bool encode_scenario_map(CUtensorMap* m, const float* d32, int N, int H) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  if (encode == nullptr || d32 == nullptr || N <= 0 || H <= 0 || N % 4 != 0) return false;
  // dims innermost first: scenario k, step j, component c
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(N), static_cast<cuuint64_t>(H), 3};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(N) * sizeof(float),
                                 static_cast<cuuint64_t>(H) * N * sizeof(float)};
  const cuuint32_t box[3] = {32, static_cast<cuuint32_t>(kTmaChunk), 3};
  const cuuint32_t elem[3] = {1, 1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(d32), dims, strides, box, elem,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int tma_pair_blocks_per_sm(bool pu) {
  int b = 0;
  const cudaError_t e =
      pu ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, rollout_tma_pair_kernel<true>, kRollThreads,
                                                         kTmaSmemBytes)
         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, rollout_tma_pair_kernel<false>, kRollThreads,
                                                         kTmaSmemBytes);
  return e == cudaSuccess && b > 0 ? b : 0;
}

// Resident blocks per SM of the paired kernel (its register count decides).
int pair_blocks_per_sm(bool pu) {
  static const int n[2] = {
      [] { int b = 0; return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, rollout_pair_kernel<false>,
                                                                           kRollThreads, 0) == cudaSuccess && b > 0 ? b : 1; }(),
      [] { int b = 0; return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, rollout_pair_kernel<true>,
                                                                           kRollThreads, 0) == cudaSuccess && b > 0 ? b : 1; }()};
  return n[pu ? 1 : 0];
}

cudaError_t launch_recheck(const Launch& L, int early_exit) {
  recheck_kernel<<<L.recheck_blocks, 64, 0, L.stream>>>(L, L.u64, early_exit);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Search.  Thread 0 of a single block runs the decision logic; the block then
// prepares the round's candidates in parallel (v_i by Eq. 2, constants, the
// steady-state check of Eq. 3 by one equilibrium solve per candidate).

// Bisection tree of Alg. 1 from the state (lo, hi, kappa): heap node 1 is
// the next kappa to test; node 2n is the state after "infeasible" at node n
// (hi <- kappa), node 2n+1 after "feasible" (lo <- kappa); a feasible
// kappa = 1 ends Alg. 1, so the right subtree of a kappa = 1 node is empty.
__device__ int tree_count(bool root_is_one, int d) {
  return root_is_one ? (1 << (d - 1)) : ((1 << d) - 1);
}

__device__ int choose_depth(const SearchState* s, const SearchCfg& c) {
  const int remaining = c.n_bisect - s->iter;
  const bool one = s->kappa == 1.0;
  int d = 1;
  while (d + 1 <= remaining && d + 1 <= 11 && tree_count(one, d + 1) <= c.m_cap) ++d;
  return d;
}

// Tree construction is split: the deciding thread records what to build
// (build_tree returns the node count, known in closed form) and, after a
// barrier, the whole block writes the nodes (build_tree_block), one node per
// thread: each node's kappa is a short chain of binary64 operations and
// GB300's binary64 latency makes a serial loop over up to 2,047 nodes slow.
struct TreeReq {
  int pending, which, base, depth;
  double lo, hi, kappa;
};
__shared__ TreeReq g_tree_req;

__device__ int build_tree(const SearchState* s, int which, int base, int depth) {
  g_tree_req.pending = 1;
  g_tree_req.which = which;
  g_tree_req.base = base;
  g_tree_req.depth = depth;
  g_tree_req.lo = s->lo;
  g_tree_req.hi = s->hi;
  g_tree_req.kappa = s->kappa;
  return tree_count(s->kappa == 1.0, depth);
}

// Heap node n of the requested tree goes to slot base + (its rank among the
// valid nodes in heap order): with a kappa = 1 root the valid nodes are the
// root and its left subtree, so level L >= 1 starts at rank 2^(L-1).
__device__ void build_tree_block(const Launch& L) {
  const TreeReq r = g_tree_req;
  if (!r.pending) return;
  int32_t* map = r.which ? L.st->slot_of_node1 : L.st->slot_of_node;
  const bool one = r.kappa == 1.0;
  const int nodes = 1 << r.depth;
  for (int n = threadIdx.x + 1; n < nodes; n += blockDim.x) {
    const int lev = 31 - __clz(n);
    const int off = n - (1 << lev);
    const bool valid = !one || lev == 0 || off < (1 << (lev - 1));
    if (!valid) {
      map[n] = -1;
      continue;
    }
    double lo = r.lo, hi = r.hi, k = r.kappa;
    for (int b = lev - 1; b >= 0; --b) {
      if ((n >> b) & 1) lo = k; else hi = k;
      k = __dmul_rn(__dadd_rn(lo, hi), 0.5);
    }
    const int rank = !one ? n - 1 : (lev == 0 ? 0 : (1 << (lev - 1)) + off);
    map[n] = r.base + rank;
    L.cand_kappa[r.base + rank] = k;
  }
}

// Follows Alg. 1's path through an evaluated tree of `depth` levels, one
// iteration per level; bit l of *bits is the outcome at level l, *len the
// number of levels walked.
// With `visited`, the slots of the path are recorded; with `expect`, the
// walk stops right after the first level whose outcome differs from bit l of
// *expect (*diverged is then set): beyond it the path leaves the nodes whose
// outcomes are known.
__device__ void walk_tree(SearchState* s, const SearchCfg& c, const int32_t* slot_map, int depth,
                          const int32_t* cand_ok, uint32_t* bits, int* len,
                          int32_t* visited = nullptr, const uint32_t* expect = nullptr,
                          bool* diverged = nullptr) {
  // the walk's state in registers, written back once: each level's decision
  // would otherwise wait on the previous level's stores to global memory
  double kap = s->kappa, lo = s->lo, hi = s->hi, kopt = s->kappa_opt;
  int iter = s->iter, any = s->any, done = s->done;
  int n = 1;
  uint32_t b = 0;
  int l = 0;
  if (diverged) *diverged = false;
  for (int lev = 0; lev < depth; ++lev) {
    const int slot = slot_map[n];
    if (slot < 0) break;  // cannot happen: the path only visits valid nodes
    if (visited) visited[lev] = slot;
    const double k = kap;
    iter += 1;
    ++l;
    const bool ok = cand_ok[slot] != 0;
    if (expect && ok != (((*expect >> lev) & 1u) != 0)) {
      *diverged = true;
      depth = lev + 1;  // apply this level's decision, then stop
    }
    if (ok) {
      b |= 1u << lev;
      kopt = k;
      any = 1;
      if (k == 1.0) { done = 1; break; }
      lo = k;
      n = 2 * n + 1;
    } else {
      hi = k;
      n = 2 * n;
    }
    kap = __dmul_rn(__dadd_rn(lo, hi), 0.5);
    if (iter >= c.n_bisect) { done = 1; break; }
  }
  s->kappa = kap; s->lo = lo; s->hi = hi; s->kappa_opt = kopt;
  s->iter = iter; s->any = any; s->done = done;
  *bits = b;
  *len = l;
}

// The walks' inputs, staged in shared memory by the whole block before the
// deciding thread walks: the slot of each heap node of the round's tree (and
// of the pipelined second tree) and the slots' outcomes, so the walk's levels
// do not chain dependent global loads.
struct WalkStage {
  int32_t map0[kMaxTreeNodes];
  int32_t map1[kMaxTreeNodes];
  int32_t ok[2 * RRG_MAX_CANDIDATES];
};
__device__ void stage_walk(const Launch& L, WalkStage& w, bool second) {
  const SearchState* s = L.st;
  const int n0 = 1 << s->depth;
  for (int n = threadIdx.x; n < n0; n += blockDim.x) w.map0[n] = s->slot_of_node[n];
  if (second) {
    const int n1 = 1 << s->depth1;
    for (int n = threadIdx.x; n < n1; n += blockDim.x) w.map1[n] = s->slot_of_node1[n];
  }
  for (int i = threadIdx.x; i < 2 * L.scfg.m_cap; i += blockDim.x) w.ok[i] = L.cand_ok[i];
}

__device__ void set_segments(SearchState* s, int mode0, int count0, int base0, int mode1,
                             int count1, int base1) {
  s->seg[0].mode = mode0; s->seg[0].count = count0; s->seg[0].base = base0;
  s->seg[1].mode = mode1; s->seg[1].count = count1; s->seg[1].base = base1;
}

__device__ void save_walk_start(SearchState* s) {
  s->w_lo = s->lo; s->w_hi = s->hi; s->w_kappa = s->kappa; s->w_kopt = s->kappa_opt;
  s->w_iter = s->iter; s->w_any = s->any;
}

__device__ void restore_walk_start(SearchState* s) {
  s->lo = s->w_lo; s->hi = s->w_hi; s->kappa = s->w_kappa; s->kappa_opt = s->w_kopt;
  s->iter = s->w_iter; s->any = s->w_any; s->done = 0;
}

// Prepares the first round after the inputs were stored; returns m.
__device__ int first_round(SearchState* s, const SearchCfg& c, double* cand_kappa) {
  s->lo = 0.0; s->hi = 1.0; s->kappa = 1.0; s->kappa_opt = 0.0;
  s->iter = 0; s->any = 0; s->done = 0; s->flags = 0; s->round = 0; s->probe = 0;
  if (c.search == RRG_SEARCH_GRID || c.search == RRG_SEARCH_KSECTION)
    return grid_points(cand_kappa, c.m_cap);
  s->depth = choose_depth(s, c);
  return build_tree(s, 0, 0, s->depth);
}

// Decides from the evaluated round and prepares the next; returns next m.
__device__ int next_round(SearchState* s, const SearchCfg& c, double* cand_kappa,
                          const int32_t* cand_ok, const int32_t* slot_map) {
  const int m = s->m;
  if (c.search == RRG_SEARCH_BISECT || c.search == RRG_SEARCH_SPEC_BISECT) {
    uint32_t bits;
    int len;
    walk_tree(s, c, slot_map, s->depth, cand_ok, &bits, &len);
    s->round += 1;
    if (s->done) return 0;
    s->depth = choose_depth(s, c);
    return build_tree(s, 0, 0, s->depth);
  }
  int best = -1;
  for (int i = 0; i < m; ++i)
    if (cand_ok[i]) best = i;
  if (c.search == RRG_SEARCH_GRID) {
    if (best >= 0) { s->kappa_opt = cand_kappa[best]; s->any = 1; }
    s->round += 1;
    s->done = 1;
    return 0;
  }
  // k-section
  if (s->round == 0) {
    if (best < 0) { s->done = 1; s->round = 1; return 0; }
    s->any = 1;
    s->kappa_opt = cand_kappa[best];
    if (best == m - 1) { s->done = 1; s->round = 1; return 0; }
    s->lo = cand_kappa[best];
    s->hi = cand_kappa[best + 1];
  } else if (best < 0) {
    s->hi = cand_kappa[0];
  } else {
    s->kappa_opt = cand_kappa[best];
    s->lo = cand_kappa[best];
    if (best < m - 1) s->hi = cand_kappa[best + 1];
  }
  s->round += 1;
  if (s->round >= c.n_rounds) { s->done = 1; return 0; }
  return interior_points(cand_kappa, c.m_cap, s->lo, s->hi);
}

// Candidate slot i: v_i by Eq. 2, constants, the steady-state check of
// Eq. 3 and fresh flags.
__device__ void prepare_slot(const Launch& L, int i) {
  const SearchState* s = L.st;
  const double thr_ss =
      __dadd_rn(L.scfg.y_min, __dmul_rn(L.scfg.eps_ss, __dsub_rn(L.scfg.y_c, L.scfg.y_min)));
  const double v = governed(s->v_prev, s->r, L.cand_kappa[i]);
  L.cand_v[i] = v;
  const int ok = candidate_setup(L.k64, L.k32, L.params, v, L.scfg.ss_check, thr_ss, L.y_min,
                                 L.cand_c64 + i, L.cand_c32 + i);
  L.cand_ok[i] = ok;
  L.cand_ss[i] = ok;
  L.cand_dead[i] = ok ? 0 : 1;
  L.cand_min[i] = dkey(inf_v<double>());
}

// One block per candidate slot of the round the search kernel just set up;
// block 0 also empties the recheck list.
__global__ void __launch_bounds__(32) prepare_kernel(const Launch L) {
  const SearchState* s = L.st;
  if (threadIdx.x != 0) return;
  if (blockIdx.x == 0) *L.recheck_count = 0u;
  if (static_cast<int>(blockIdx.x) < s->prep_m) prepare_slot(L, s->prep_base + blockIdx.x);
}

// The same inside a search kernel, one thread per slot of the round it just
// set up (after build_tree_block has written the round's kappas): the
// closed loop's critical path then has no separate prepare launch.
__device__ void prepare_block(const Launch& L) {
  __syncthreads();
  const SearchState* s = L.st;
  if (threadIdx.x == 0) *L.recheck_count = 0u;
  const int base = s->prep_base, m = s->prep_m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) prepare_slot(L, base + i);
}

cudaError_t launch_prepare(const Launch& L, int width) {
  prepare_kernel<<<width > 0 ? width : 1, 32, 0, L.stream>>>(L);
  return cudaGetLastError();
}

__device__ void write_result(SearchState* s, double* v_t, double* kappa, int32_t* flags) {
  s->flags = (s->any ? 0 : 1) | (s->invalid ? 2 : 0);
  const double kap = s->invalid ? 0.0 : s->kappa_opt;
  const double v = s->invalid ? s->v_prev : governed(s->v_prev, s->r, kap);
  s->kappa_opt = kap;
  s->v_t_out = v;
  if (v_t) *v_t = v;
  if (kappa) *kappa = kap;
  if (flags) *flags = s->flags;
}

__global__ void __launch_bounds__(kSearchThreads)
search_begin_kernel(const Launch L, const double* __restrict__ d_x, const double* __restrict__ d_r,
                    const unsigned long long* t_dev, const double* __restrict__ d_v_prev,
                    int pipeline, long long buf_base) {
  SearchState* s = L.st;
  if (threadIdx.x == 0) g_tree_req.pending = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double x0 = d_x[0], x1 = d_x[1], x2 = d_x[2];
    const double r = d_r[t_dev ? *t_dev : 0ull];
    const double vp = *d_v_prev;
    s->x[0] = x0; s->x[1] = x1; s->x[2] = x2;
    s->r = r;
    s->v_prev = vp;
    s->buf = (buf_base >= 0 && t_dev != nullptr && L.d64b != nullptr)
                 ? static_cast<int>((static_cast<unsigned long long>(buf_base) + *t_dev) & 1ull)
                 : 0;
    const bool fin = fabs(x0) <= DBL_MAX && fabs(x1) <= DBL_MAX && fabs(x2) <= DBL_MAX &&
                     fabs(r) <= DBL_MAX && fabs(vp) <= DBL_MAX;
    s->invalid = (!fin || !(vp > 0.0) || !(r > 0.0)) ? 1 : 0;
    int m = first_round(s, L.scfg, L.cand_kappa);
    if (s->invalid) { s->done = 1; m = 0; }
    s->m = m;
    if (pipeline && m > 0) {
      save_walk_start(s);
      s->probe = 1;
      set_segments(s, SEG_PROBE, m, 0, SEG_FULL, 0, 0);
    } else {
      set_segments(s, SEG_FULL, m, 0, SEG_FULL, 0, 0);
    }
    s->prep_base = 0;
    s->prep_m = m;
  }
  __syncthreads();
  build_tree_block(L);
  prepare_block(L);
}

// Between the probe of round 1 and the launch that finishes it: walk round
// 1's tree with the provisional outcomes (a node is provisionally admissible
// while none of its trajectories has violated yet), build round 2's tree
// from where that walk ends (slots m_cap..), and let the next launch both
// continue round 1 and run round 2.
__global__ void __launch_bounds__(kSearchThreads)
search_mid_kernel(const Launch L) {
  SearchState* s = L.st;
  __shared__ WalkStage W;
  if (threadIdx.x == 0) g_tree_req.pending = 0;
  stage_walk(L, W, false);
  __syncthreads();
  if (threadIdx.x == 0) {
    int m1 = 0;
    if (s->probe && !s->done) {
      const int m0 = s->m;
      (void)m0;
      restore_walk_start(s);
      uint32_t bits;
      int len;
      walk_tree(s, L.scfg, W.map0, s->depth, W.ok, &bits, &len, s->cont_slot);
      s->prov_bits = bits;
      s->prov_len = len;
      s->prov_done = s->done;
      s->done = 0;
      if (!s->prov_done) {
        s->depth1 = choose_depth(s, L.scfg);
        m1 = build_tree(s, 1, L.scfg.m_cap, s->depth1);
      }
      // only the nodes on the provisional path are finished: no other node
      // of round 1 can be read by a walk that agrees with the provisional one
      set_segments(s, SEG_CONTINUE, len, 0, SEG_FULL, m1, L.scfg.m_cap);
    }
    s->prep_base = L.scfg.m_cap;
    s->prep_m = m1;
  }
  __syncthreads();
  build_tree_block(L);
  prepare_block(L);
}

__global__ void __launch_bounds__(kSearchThreads)
search_next_kernel(const Launch L, double* v_t, double* kappa, int32_t* flags) {
  SearchState* s = L.st;
  __shared__ WalkStage W;
  if (threadIdx.x == 0) g_tree_req.pending = 0;
  stage_walk(L, W, s->probe != 0);
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    if (!s->done && s->probe) {
      // validate the pipelined pair: walk round 1 again with the final
      // outcomes; only if every decision matches the provisional walk does
      // round 2's tree continue Alg. 1's path
      s->probe = 0;
      restore_walk_start(s);
      uint32_t bits;
      int len;
      bool diverged = false;
      const uint32_t expect = s->prov_bits;
      walk_tree(s, L.scfg, W.map0, s->depth, W.ok, &bits, &len, nullptr, &expect, &diverged);
      s->round += 1;
      if (!diverged && !s->done) {
        walk_tree(s, L.scfg, W.map1, s->depth1, W.ok, &bits, &len);
        s->round += 1;
      } else if (diverged) {
        L.stats->repairs += 1ull;
      }
      if (!s->done) {
        s->depth = choose_depth(s, L.scfg);
        m = build_tree(s, 0, 0, s->depth);
      }
    } else if (!s->done) {
      m = next_round(s, L.scfg, L.cand_kappa, W.ok, W.map0);
    }
    if (s->done) {
      m = 0;
      write_result(s, v_t, kappa, flags);
    }
    s->m = m;
    set_segments(s, SEG_FULL, m, 0, SEG_FULL, 0, 0);
    s->prep_base = 0;
    s->prep_m = m;
    if (L.cond != 0ull) {
      cudaGraphSetConditional(L.cond, s->done ? 0u : 1u);
      if (!s->done) {
        L.stats->cond_launches += L.cond_launches;
        L.stats->cond_rollouts += L.cond_rollouts;
        L.stats->cond_rounds += L.cond_rounds;
      }
    }
  }
  __syncthreads();
  build_tree_block(L);
  prepare_block(L);
}

cudaError_t launch_search_begin(const Launch& L, const double* d_x, const double* d_r,
                                const unsigned long long* t_dev, const double* d_v_prev,
                                long long buf_base) {
  const int pipeline = search_pipelined(L.scfg, L.H) ? 1 : 0;
  search_begin_kernel<<<1, kSearchThreads, 0, L.stream>>>(L, d_x, d_r, t_dev, d_v_prev, pipeline,
                                                          buf_base);
  return cudaGetLastError();
}

cudaError_t launch_search_mid(const Launch& L) {
  search_mid_kernel<<<1, kSearchThreads, 0, L.stream>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_search_next(const Launch& L, double* d_v_t, double* d_kappa, int32_t* d_flags) {
  search_next_kernel<<<1, kSearchThreads, 0, L.stream>>>(L, d_v_t, d_kappa, d_flags);
  return cudaGetLastError();
}

// Explicit candidates (rrg_eval_candidates).
__global__ void __launch_bounds__(kSearchThreads)
eval_prepare_kernel(const Launch L, const double* __restrict__ d_x, double v_prev, double r,
                    const double* __restrict__ d_kappas, int m, const double* __restrict__ d_vp,
                    const double* __restrict__ d_r) {
  SearchState* s = L.st;
  if (threadIdx.x == 0) {
    s->x[0] = d_x[0]; s->x[1] = d_x[1]; s->x[2] = d_x[2];
    s->v_prev = d_vp != nullptr ? *d_vp : v_prev;
    s->r = d_r != nullptr ? *d_r : r;
    s->m = m;
    s->done = 0;
    s->invalid = 0;
    s->probe = 0;
    s->buf = 0;
    set_segments(s, SEG_FULL, m, 0, SEG_FULL, 0, 0);
    s->prep_base = 0;
    s->prep_m = m;
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) L.cand_kappa[i] = d_kappas[i];
}

__global__ void eval_finish_kernel(const Launch L, int m, uint8_t* adm, double* min_slack) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const bool ss_failed = !L.cand_ss[i];
    adm[i] = L.cand_ok[i] ? 1 : 0;
    if (min_slack) min_slack[i] = ss_failed ? __longlong_as_double(0x7ff8000000000000ll)
                                            : dunkey(L.cand_min[i]);
  }
}

cudaError_t launch_eval_prepare(const Launch& L, const double* d_x, double v_prev, double r,
                                const double* d_kappas, int m, const double* d_vp, const double* d_r) {
  eval_prepare_kernel<<<1, kSearchThreads, 0, L.stream>>>(L, d_x, v_prev, r, d_kappas, m, d_vp, d_r);
  return cudaGetLastError();
}

cudaError_t launch_eval_finish(const Launch& L, int m, uint8_t* d_adm, double* d_min_slack) {
  eval_finish_kernel<<<grid_for(m, 128, 64), 128, 0, L.stream>>>(L, m, d_adm, d_min_slack);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Simulated plant of the closed loop (Fig. 1) and the loop bookkeeping.
// The plant's step runs on one warp.  It is binary64 and sits on the closed
// loop's critical path, and GB300's binary64 pipe takes a warp instruction at
// a time however few lanes are active, so a lone thread pays for every
// instruction of the step.  All 32 lanes run the same step; only the x^e - 1
// series is shared out: the 16 leaves of pow_m1_series's Estrin tree go to 16
// lanes, and each level above is one fused multiply-add after two shuffles.
// The tree, its operands and their order are pow_m1_series's, so every lane
// gets its value bit for bit (the plant kernel measured 12.8 against 16.8 us).
// The step around it is rk4_step_fast<double>'s: the same stage points and
// combination, each right-hand side fc3_rhs_fast's with the shared series.
// Called by all 32 lanes of the warp with the same arguments.
__device__ __forceinline__ double pow_m1_warp(const PowSeries* __restrict__ S, double x, double e) {
  if (S != nullptr && S->e == e) {
    const double t = fma(x, S->inv_c, -1.0);
    if (fabs(t) <= 1.0 / 3.0) {
      const int i = static_cast<int>(threadIdx.x & 15);
      const double t2 = t * t, t4 = t2 * t2, t8 = t4 * t4, t16 = t8 * t8, t32 = t16 * t16;
      double p = fma(S->a[2 * i + 1], t, S->a[2 * i]);
      double hi = __shfl_sync(0xffffffffu, p, 2 * i + 1), lo = __shfl_sync(0xffffffffu, p, 2 * i);
      p = fma(hi, t2, lo);
      hi = __shfl_sync(0xffffffffu, p, 2 * i + 1);
      lo = __shfl_sync(0xffffffffu, p, 2 * i);
      p = fma(hi, t4, lo);
      hi = __shfl_sync(0xffffffffu, p, 2 * i + 1);
      lo = __shfl_sync(0xffffffffu, p, 2 * i);
      p = fma(hi, t8, lo);
      const double p1 = __shfl_sync(0xffffffffu, p, 1), p0 = __shfl_sync(0xffffffffu, p, 0);
      return fma(S->a[32], t32, fma(p1, t16, p0));
    }
  }
  return pow(x, e) - 1.0;
}

__device__ __forceinline__ void rhs_plant_warp(const RhsU<double>& U, const RhsC<double>& C, double z_ca,
                                               double z_w, double z_sm, double w, double x_pw, double& d_ca,
                                               double& d_w, double& d_sm) {
  d_ca = U.a1 * z_sm + (C.c_ca - U.a12 * z_ca);
  d_sm = U.g_w * z_w + ((C.c_sm + U.b3 * z_ca) - U.g_sm * z_sm);
  const double W_cp = U.a_w * z_w + (C.W_r - U.a_p * z_sm);
  const double f = torque_factor<double>(U, pow_m1_warp(U.pws, x_pw, U.e), w);
  d_w = (C.e0 - U.e2 * z_w) - W_cp * f;
}

__device__ __forceinline__ void rk4_plant_warp(const RhsU<double>& U, const RhsC<double>& C, double dt0,
                                               double& q_ca, double& w, double& q_sm, double& w_abs,
                                               double e_ca, double e_w, double e_sm) {
  const StepC<double> S = step_consts<double>(U, dt0);
  const double dt = S.dt, h2 = S.h2, h6 = S.h6, g2 = S.g2, g1 = S.g1;
  const double x1 = q_sm * U.inv_p_atm + C.x_r;
  double a1, b1, c1, a2, b2, c2, a3, b3, c3, a4, b4, c4;
  rhs_plant_warp(U, C, q_ca, w, q_sm, w_abs, x1, a1, b1, c1);
  rhs_plant_warp(U, C, q_ca + h2 * a1, w + h2 * b1, q_sm + h2 * c1, w_abs + h2 * b1, x1 + g2 * c1,
                 a2, b2, c2);
  rhs_plant_warp(U, C, q_ca + h2 * a2, w + h2 * b2, q_sm + h2 * c2, w_abs + h2 * b2, x1 + g2 * c2,
                 a3, b3, c3);
  const double p_ca = (q_ca + e_ca) + h6 * (a1 + 2.0 * (a2 + a3));
  const double p_w = (w + e_w) + h6 * (b1 + 2.0 * (b2 + b3));
  const double p_sm = (q_sm + e_sm) + h6 * (c1 + 2.0 * (c2 + c3));
  const double p_wa = p_w + C.r_w;
  rhs_plant_warp(U, C, q_ca + dt * a3, w + dt * b3, q_sm + dt * c3, w_abs + dt * b3, x1 + g1 * c3,
                 a4, b4, c4);
  q_ca = p_ca + h6 * a4;
  w = p_w + h6 * b4;
  q_sm = p_sm + h6 * c4;
  w_abs = p_wa + h6 * b4;
}

// x_{t+1} = RK4(x_t, v) + the plant's own draw (plant_step_fast's step, on the
// warp).
__device__ void plant_step(const Launch& L, const double* x, double v, uint64_t seed, uint64_t upd,
                           const double* amp, double* x_next) {
  const U64x4 r = philox4x64_10(0ull, 0ull, upd, 1ull, seed, 0ull);
  RhsC<double> c64;
  RhsC<float> c32;
  const double q0[3] = {0.0, 0.0, 0.0};
  fold_rhs_cand(L.k64, cand_consts(L.params, v), q0, 0.0, &c64, &c32);
  const double p_atm = L.params[P_P_ATM];
  double q_ca = x[0] - p_atm, w = x[1], q_sm = x[2] - p_atm, w_abs = x[1];
  rk4_plant_warp(L.u64, c64, L.dt, q_ca, w, q_sm, w_abs, uniform_sym(r.w[0], amp[0]),
                 uniform_sym(r.w[1], amp[1]), uniform_sym(r.w[2], amp[2]));
  x_next[0] = q_ca + p_atm;
  x_next[1] = w;
  x_next[2] = q_sm + p_atm;
}

__global__ void plant_kernel(const Launch L, const double* d_x, const double* d_v, uint64_t seed,
                             uint64_t base, const unsigned long long* t_dev, const double* amp,
                             double* x_next) {
  if (blockIdx.x != 0) return;
  double x[3] = {d_x[0], d_x[1], d_x[2]}, xn[3];
  plant_step(L, x, *d_v, seed, base + (t_dev ? *t_dev : 0ull), amp, xn);
  if (threadIdx.x == 0) {
    x_next[0] = xn[0]; x_next[1] = xn[1]; x_next[2] = xn[2];
  }
}

cudaError_t launch_plant(const Launch& L, const double* d_x, const double* d_v, uint64_t seed,
                         uint64_t base, const unsigned long long* t_dev, const double* amp_dev,
                         double* d_x_next) {
  plant_kernel<<<1, 32, 0, L.stream>>>(L, d_x, d_v, seed, base, t_dev, amp_dev, d_x_next);
  return cudaGetLastError();
}

__global__ void loop_init_kernel(LoopState* ls, double x0, double x1, double x2, double v0,
                                 double* x_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ls->x[0] = x0; ls->x[1] = x1; ls->x[2] = x2;
  ls->v_prev = v0;
  ls->t = 0ull;
  if (x_out) { x_out[0] = x0; x_out[1] = x1; x_out[2] = x2; }
}

cudaError_t launch_loop_init(const Launch& L, LoopState* ls, const double* x0, double v0,
                             double* d_x_out) {
  loop_init_kernel<<<1, 32, 0, L.stream>>>(ls, x0[0], x0[1], x0[2], v0, d_x_out);
  return cudaGetLastError();
}

// After the search of update t: record v_t, kappa, flags; move the plant one
// step under v_t; v_prev <- v_t; t <- t + 1.
__global__ void loop_end_kernel(const Launch L, LoopState* ls, uint64_t seed, uint64_t t0,
                                const double* amp, double* v_out, double* kappa_out,
                                int32_t* flags_out, double* x_out) {
  if (blockIdx.x != 0) return;
  const SearchState* s = L.st;
  const unsigned long long t = ls->t;
  const double v = s->v_t_out;
  const double x[3] = {ls->x[0], ls->x[1], ls->x[2]};
  double xn[3];
  plant_step(L, x, v, seed, t0 + t, amp, xn);  // the whole warp (its shuffles order the reads above)
  if (threadIdx.x != 0) return;
  if (v_out) v_out[t] = v;
  if (kappa_out) kappa_out[t] = s->kappa_opt;
  if (flags_out) flags_out[t] = s->flags;
  ls->x[0] = xn[0]; ls->x[1] = xn[1]; ls->x[2] = xn[2];
  ls->v_prev = v;
  ls->t = t + 1;
  if (x_out) {
    x_out[3 * (t + 1) + 0] = xn[0];
    x_out[3 * (t + 1) + 1] = xn[1];
    x_out[3 * (t + 1) + 2] = xn[2];
  }
}

cudaError_t launch_loop_end(const Launch& L, LoopState* ls, uint64_t seed, uint64_t t0,
                            const double* amp_dev, double* d_v_out, double* d_kappa_out,
                            int32_t* d_flags_out, double* d_x_out) {
  loop_end_kernel<<<1, 32, 0, L.stream>>>(L, ls, seed, t0, amp_dev, d_v_out, d_kappa_out,
                                          d_flags_out, d_x_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host-side schedule of rounds (mirrors choose_depth / tree_count above).
static int host_tree_count(bool one, int d) { return one ? (1 << (d - 1)) : ((1 << d) - 1); }

int search_round_count(const SearchCfg& c) {
  if (c.search == RRG_SEARCH_GRID) return 1;
  if (c.search == RRG_SEARCH_KSECTION) return c.n_rounds;
  int iter = 0, rounds = 0;
  bool one = true;
  while (iter < c.n_bisect) {
    int d = 1;
    while (d + 1 <= c.n_bisect - iter && d + 1 <= 11 && host_tree_count(one, d + 1) <= c.m_cap) ++d;
    iter += d;
    one = false;
    ++rounds;
  }
  return rounds;
}

bool search_pipelined(const SearchCfg& c, int horizon) {
  return c.search == RRG_SEARCH_SPEC_BISECT && c.probe_steps > 0 && c.probe_steps < horizon &&
         search_round_count(c) >= 2;
}

static int host_max_depth(const SearchCfg& c) {
  int d = 1;
  while (d + 1 <= 11 && host_tree_count(false, d + 1) <= c.m_cap) ++d;
  return d;
}

int search_extra_rounds(const SearchCfg& c) {
  const int d = host_max_depth(c);
  return (c.n_bisect - 1 + d - 1) / d;
}

int search_extra_width(const SearchCfg& c) {
  return host_tree_count(false, host_max_depth(c));
}

int search_round_width(const SearchCfg& c, int round) {
  if (c.search == RRG_SEARCH_GRID || c.search == RRG_SEARCH_KSECTION) return c.m_cap;
  int iter = 0;
  bool one = true;
  for (int r = 0; iter < c.n_bisect; ++r) {
    int d = 1;
    while (d + 1 <= c.n_bisect - iter && d + 1 <= 11 && host_tree_count(one, d + 1) <= c.m_cap) ++d;
    if (r == round) return host_tree_count(one, d);
    iter += d;
    one = false;
  }
  return 1;
}

}  // namespace rrg
