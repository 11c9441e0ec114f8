// rrg_batch.cu -- many independent robust RG problems in one set of launches.
//
// S instances, each with its own scenario count N_s and horizon H_s, share
// the model and the search settings.  One update of all of them is a fixed
// launch sequence (CUDA-graph capturable):
//
//   batch_sample_kernel      d_j^k of every instance (grid y = instance)
//   batch_begin_kernel       inputs, round-1 candidates (Alg. 3 grid, Eq. 5),
//                            the round's tile list
//   { batch_prepare_kernel   v_i (Eq. 2), candidate constants, steady-state
//                            check (Eq. 3); one thread per (instance, slot)
//     batch_rollout_kernel   persistent: each CTA takes the next tile
//                            (instance, candidate, block of scenarios) from a
//                            queue ordered longest horizon first, and runs
//                            its trajectories as the single-problem rollout
//     batch_recheck_kernel   binary64 re-run of near-zero-slack lanes
//     batch_decide_kernel }  Alg. 3 / k-section decision per instance, the
//                            next round's candidates and tile list
//   batch_plant_kernel       simulated plants (closed loop only)
//
// The tile queue is one atomic counter; a CTA never waits for another.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

#include "rrg_device.cuh"
#include "rrg_internal.h"
#include "rrg_lane.cuh"

namespace rrg {
namespace {

constexpr int kMaxInst = RRG_BATCH_MAX_INSTANCES;
constexpr int kDecideThreads = 1024;
static_assert(kMaxInst <= kDecideThreads, "one decision thread per instance");

struct BInst {
  int32_t N, H;
  long long off;  // element offset of the instance's [3][H][N] binary32 scenarios
};

struct BState {
  double x[3];            // x_t of the current update
  double v_prev, r;
  double lx[3], lv;       // closed-loop state (plant state, last v), kept apart
                          // from single updates' inputs
  double lo, hi, kappa_opt;
  double kappa;           // speculative bisection: the kappa Alg. 1 tests next
  double v_out;
  int32_t m, round, any, done, invalid, flags;
  int32_t iter, pad2;     // speculative bisection: Alg. 1 iterations done
  int32_t cur, pad;                      // scenario pair of the current update
  unsigned long long seed_p[2], update_p[2];  // what each pair holds
};

struct BCfg {
  int S, M, n_rounds, search, ss_check, early_exit;
  int n_bisect, width;  // speculative bisection: N_kappa, tree nodes per round (<= M)
  double dt, y_min, eps_ss, y_c, eps_abs;
  double amp[3];
};

struct BLaunch {
  cudaStream_t stream;
  BCfg c;
  const double* params;
  Fc3K<double> k64;
  Fc3K<float> k32;
  RhsU<double> u64;
  RhsU<float> u32;
  const BInst* inst;
  const int32_t* order;  // instances, longest horizon (then most scenarios) first
  BState* st;
  float* d32;
  float* d32b;         // second scenario pair (closed loops), or nullptr
  double* cand_kappa;
  double* cand_v;
  RhsC<double>* cand_c64;
  RhsC<float>* cand_c32;
  int32_t* cand_ok;
  int32_t* cand_dead;
  int32_t* cand_ss;
  unsigned long long* cand_min;
  int32_t* tile_base;  // [S + 1] over `order`
  uint32_t* queue;     // [0] next tile, [1] tiles of the round
  uint2* recheck_list; // (slot, k)
  uint32_t* recheck_jlast;  // the recheck runs steps 0..jlast
  uint32_t* recheck_count;
  unsigned long long recheck_cap;
  DevStats* stats;
  unsigned long long* t_dev;  // closed-loop update counter
};

// ---------------------------------------------------------------------------
// Sampling: instance s draws with key (seed + s, 0) and the counters of the
// single-problem sampler; only the binary32 copy is stored (the recheck
// regenerates binary64 values from the same counters).
__global__ void batch_sample_kernel(const BLaunch B, uint64_t seed, uint64_t base) {
  const int s = blockIdx.y;
  const BInst I = B.inst[s];
  const uint64_t upd = base + (B.t_dev ? *B.t_dev : 0ull);
  const uint64_t key = seed + static_cast<uint64_t>(s);
  const int pair = (B.d32b != nullptr && (upd & 1ull)) ? 1 : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    B.st[s].seed_p[pair] = key;
    B.st[s].update_p[pair] = upd;
  }
  const size_t HN = static_cast<size_t>(I.H) * I.N;
  float* d = (pair ? B.d32b : B.d32) + I.off;
  const float s0 = static_cast<float>(B.c.amp[0] * 0x1.0p-23),
              s1 = static_cast<float>(B.c.amp[1] * 0x1.0p-23),
              s2 = static_cast<float>(B.c.amp[2] * 0x1.0p-23);
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (size_t q = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < HN; q += stride) {
    const uint64_t j = q / static_cast<uint64_t>(I.N), k = q - j * static_cast<uint64_t>(I.N);
    const U64x4 w = philox4x64_10(j, k, upd, 0ull, key, 0ull);
    d[q] = uniform_sym32(w.w[0], s0);
    d[HN + q] = uniform_sym32(w.w[1], s1);
    d[2 * HN + q] = uniform_sym32(w.w[2], s2);
  }
}

// Tile list of the next round: instance order[o] contributes ceil(m / rows) x
// ceil(N / tile) tiles (rows = 2: two candidate slots per tile); block-wide
// inclusive scan (blockDim = kDecideThreads >= S).
__device__ void build_tiles(const BLaunch& B, int tile, int rows) {
  __shared__ int sc[kDecideThreads];
  const int o = threadIdx.x;
  int cnt = 0;
  if (o < B.c.S) {
    const int s = B.order[o];
    const BState& st = B.st[s];
    cnt = (st.done ? 0 : (st.m + rows - 1) / rows) * ((B.inst[s].N + tile - 1) / tile);
  }
  sc[o] = cnt;
  __syncthreads();
  for (int d = 1; d < kDecideThreads; d <<= 1) {
    const int v = o >= d ? sc[o - d] : 0;
    __syncthreads();
    sc[o] += v;
    __syncthreads();
  }
  if (o < B.c.S) B.tile_base[o + 1] = sc[o];
  if (o == 0) {
    B.tile_base[0] = 0;
    B.queue[0] = 0u;
    B.queue[1] = static_cast<uint32_t>(sc[B.c.S - 1]);
    *B.recheck_count = 0u;
  }
}

// Speculative bisection per instance: the nodes of the next levels of
// Alg. 1's bisection tree from the instance's state that fit in `width`
// (breadth-first; node 2n follows "not admissible" at node n, 2n + 1
// "admissible"; an admissible kappa = 1 ends the search, so it has no
// admissible child), and the walk of Alg. 1's path through their outcomes.
// The same tree and walk as the single-problem speculative bisection and
// rrg_bisect_plan / rrg_bisect_decide, so every instance's kappa is Alg. 1's
// whatever the width.
__device__ int btree_size(bool one, int d) { return one ? (1 << (d - 1)) : ((1 << d) - 1); }

__device__ int btree_depth(const BState& st, int width, int n_bisect) {
  if (st.done || st.iter >= n_bisect || width < 1) return 0;
  const bool one = st.kappa == 1.0;
  int d = 1;
  while (d < 11 && d + 1 <= n_bisect - st.iter && btree_size(one, d + 1) <= width) ++d;
  return d;
}

// kappa of heap node `heap`: Alg. 1's bracket updates along the path the
// node's bits spell out below the root (the instance's state).
__device__ double btree_kappa(const BState& st, uint32_t heap) {
  double lo = st.lo, hi = st.hi, k = st.kappa;
  for (int b = 30 - __clz(heap); b >= 0; --b) {
    if ((heap >> b) & 1u) lo = k; else hi = k;
    k = __dmul_rn(__dadd_rn(lo, hi), 0.5);
  }
  return k;
}

// Writes the round's kappas into kap[0..m), breadth-first, and returns m
// (<= width <= M).  Below a kappa = 1 root only node 2's subtree exists:
// level l >= 1 holds heap nodes 2^l .. 2^l + 2^(l-1) - 1.
__device__ int btree_plan(const BState& st, int width, int n_bisect, double* kap) {
  const int d = btree_depth(st, width, n_bisect);
  if (d == 0) return 0;
  const bool one = st.kappa == 1.0;
  int n = 0;
  kap[n++] = st.kappa;
  for (int l = 1; l < d; ++l) {
    const uint32_t first = 1u << l, count = one ? (1u << (l - 1)) : (1u << l);
    for (uint32_t q = 0; q < count; ++q) kap[n++] = btree_kappa(st, first + q);
  }
  return n;
}

// Alg. 1's walk through the outcomes ok[0..m) of the planned round.
__device__ void btree_walk(BState& st, const int32_t* ok, int m, int n_bisect) {
  // breadth-first position of each heap node of the round (nodes exist
  // level by level; an admissible kappa = 1 root has no node 3)
  const bool one = st.kappa == 1.0;
  uint32_t heap = 1u;
  int pos = 0;
  for (;;) {
    const bool adm = ok[pos] != 0;
    st.iter += 1;
    if (adm) {
      st.kappa_opt = st.kappa;
      st.any = 1;
      if (st.kappa == 1.0) { st.done = 1; return; }
      st.lo = st.kappa;
    } else {
      st.hi = st.kappa;
    }
    st.kappa = __dmul_rn(__dadd_rn(st.lo, st.hi), 0.5);
    if (st.iter >= n_bisect) { st.done = 1; return; }
    heap = 2u * heap + (adm ? 1u : 0u);
    // position of `heap` in the breadth-first order of the round's tree
    const int depth = 31 - __clz(heap);
    int p;
    if (!one) {
      p = static_cast<int>(heap) - 1;
    } else {
      // below a kappa = 1 root only node 2's subtree exists: level l >= 1
      // starts at 2^(l-1) and holds 2^(l-1) nodes (heap 2^l .. 2^l + 2^(l-1) - 1)
      const uint32_t first = 1u << depth;
      if (heap - first >= (1u << (depth - 1))) return;  // node 3's subtree: not in the round
      p = (1 << (depth - 1)) + static_cast<int>(heap - first);
    }
    if (p >= m) return;  // past the round's levels
    pos = p;
  }
}

// Round 1: inputs (device arrays; NULL x / v_prev: the closed loop's state),
// the scenario pair of update base + t, Alg. 3's grid, the tile list.  r is
// read at r[t * S + s] (t = the loop counter, 0 without one).
__global__ void __launch_bounds__(kDecideThreads)
batch_begin_kernel(const BLaunch B, const double* __restrict__ d_x, const double* __restrict__ d_r,
                   const double* __restrict__ d_vp, uint64_t base, int tile, int rows) {
  const int s = threadIdx.x;
  const unsigned long long t = B.t_dev ? *B.t_dev : 0ull;
  if (s < B.c.S) {
    BState& st = B.st[s];
    st.cur = (B.d32b != nullptr && ((base + t) & 1ull)) ? 1 : 0;
    if (d_x) {
      st.x[0] = d_x[3 * s];
      st.x[1] = d_x[3 * s + 1];
      st.x[2] = d_x[3 * s + 2];
    } else {
      st.x[0] = st.lx[0];
      st.x[1] = st.lx[1];
      st.x[2] = st.lx[2];
    }
    st.v_prev = d_vp ? d_vp[s] : st.lv;
    st.r = d_r[t * static_cast<unsigned long long>(B.c.S) + s];
    const bool ok = isfinite(st.x[0]) && isfinite(st.x[1]) && isfinite(st.x[2]) &&
                    isfinite(st.v_prev) && isfinite(st.r) && st.v_prev > 0.0 && st.r > 0.0;
    st.invalid = ok ? 0 : 1;
    st.lo = 0.0;
    st.hi = 1.0;
    st.kappa_opt = 0.0;
    st.any = 0;
    st.round = 0;
    st.flags = 0;
    st.done = ok ? 0 : 1;
    st.kappa = 1.0;
    st.iter = 0;
    double* kap = B.cand_kappa + static_cast<size_t>(s) * B.c.M;
    if (B.c.search == RRG_SEARCH_SPEC_BISECT)
      st.m = ok ? btree_plan(st, B.c.width, B.c.n_bisect, kap) : 0;
    else
      st.m = ok ? grid_points(kap, B.c.M) : 0;
  }
  __syncthreads();
  build_tiles(B, tile, rows);
}

// v_i, candidate constants and the steady-state check of one (instance, slot).
__global__ void batch_prepare_kernel(const BLaunch B) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int M = B.c.M;
  const int s = idx / M, i = idx - s * M;
  if (s >= B.c.S) return;
  const BState& st = B.st[s];
  if (st.done || i >= st.m) return;
  const size_t slot = static_cast<size_t>(s) * M + i;
  const double v = governed(st.v_prev, st.r, B.cand_kappa[slot]);
  B.cand_v[slot] = v;
  const double thr = __dadd_rn(B.c.y_min, __dmul_rn(B.c.eps_ss, __dsub_rn(B.c.y_c, B.c.y_min)));
  const int ok = candidate_setup(B.k64, B.k32, B.params, v, B.c.ss_check, thr, B.c.y_min,
                                 B.cand_c64 + slot, B.cand_c32 + slot);
  B.cand_ok[slot] = ok;
  B.cand_ss[slot] = ok;
  B.cand_dead[slot] = ok ? 0 : 1;
  B.cand_min[slot] = dkey(inf_v<double>());
}

// A lane's outcome for candidate slot `slot` (called by every thread of the
// warp): classified against the recheck band (an undecided lane is listed for
// the binary64 recheck unless the candidate has already failed), then the
// warp's AND of the flags, min slack and step count folded into the slot's.
__device__ __forceinline__ void batch_reduce(const BLaunch& B, size_t slot, int k, bool active, float smin,
                                             unsigned steps, int jlast, float eps,
                                             volatile int32_t* dead) {
  bool lane_ok = true, uncertain = false;
  float contrib = inf_v<float>();
  if (active) {
    if (smin >= eps) {
      contrib = smin;
    } else if (smin < -eps) {
      lane_ok = false;
      contrib = smin;
    } else {
      uncertain = true;
    }
  }
  if (uncertain && *dead == 0) {
    const uint32_t e = atomicAdd(B.recheck_count, 1u);
    if (e < B.recheck_cap) {
      B.recheck_list[e] = make_uint2(static_cast<uint32_t>(slot), static_cast<uint32_t>(k));
      B.recheck_jlast[e] = static_cast<uint32_t>(jlast);
    }
  }
  const bool all_ok = __all_sync(0xffffffffu, lane_ok);
  const float wmin = warp_min<float>(contrib);
  const unsigned wsteps = __reduce_add_sync(0xffffffffu, steps);
  if ((threadIdx.x & 31) == 0) {
    if (!all_ok) B.cand_ok[slot] = 0;
    if (wmin < inf_v<float>()) atomicMin(B.cand_min + slot, dkey(static_cast<double>(wmin)));
    if (wsteps) atomicAdd(&B.stats->lane_steps, static_cast<unsigned long long>(wsteps));
  }
}

// One tile: lanes k of candidate slot (s, i), binary32 rollouts classified
// for the binary64 recheck, reduced into the candidate's flags.  Called by
// every thread of the CTA; returns are warp- or CTA-uniform.
template <int PF>
__device__ __forceinline__ void batch_tile(const BLaunch& B, int s, int i, int k) {
  const BInst I = B.inst[s];
  const size_t slot = static_cast<size_t>(s) * B.c.M + i;
  if (!B.cand_ss[slot]) return;
  volatile int32_t* dead = B.cand_dead + slot;
  const bool cand_stop = B.c.early_exit == RRG_EXIT_CANDIDATE;
  if (cand_stop) {
    const int dead0 = __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 ? *dead : 0, 0);
    if (dead0) return;
  }
  const bool active = k < I.N;
  const float eps = static_cast<float>(B.c.eps_abs);
  const float thr = B.c.early_exit != RRG_EXIT_NONE ? -eps : -inf_v<float>();
  float smin = inf_v<float>();
  unsigned steps = 0;
  int jlast = -1;
  if (active) {
    const BState& st = B.st[s];
    const double p_atm = B.params[P_P_ATM];
    const RhsC<float> C = B.cand_c32[slot];
    float q_ca, w, q_sm, w_abs;  // the deviation from the candidate's reference point
    start_state<float>(C, st.x, p_atm, q_ca, w, q_sm, w_abs);
    int end = LANE_REACHED_END;
    const float* d = (st.cur ? B.d32b : B.d32) + I.off;
    smin = run_lane<float, PF>(B.u32, C, d, k, I.N, I.H, 0, I.H, q_ca,
                               w, q_sm, w_abs, inf_v<float>(), static_cast<float>(B.c.dt),
                               thr, cand_stop ? dead : nullptr,
                               &steps, &end, eps, &jlast);
    if (cand_stop && smin < thr) *dead = 1;
  }
  batch_reduce(B, slot, k, active, smin, steps, jlast, eps, dead);
}

// Persistent rollout: each CTA takes tiles from the queue until none is left.
template <int TILE, int PF>
__global__ void __launch_bounds__(TILE) batch_rollout_kernel(const BLaunch B) {
  __shared__ int sh[3];
  const uint32_t total = B.queue[1];
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t t = atomicAdd(B.queue, 1u);
      int s = -1, i = 0, b = 0;
      if (t < total) {
        // tile_base[lo] <= t < tile_base[hi]; instances without tiles have
        // equal bases and are skipped by taking the last such lo
        int lo = 0, hi = B.c.S;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (static_cast<uint32_t>(B.tile_base[mid]) <= t) lo = mid; else hi = mid;
        }
        s = B.order[lo];
        const int nb = (B.inst[s].N + TILE - 1) / TILE;
        const int local = static_cast<int>(t) - B.tile_base[lo];
        i = local / nb;
        b = local - i * nb;
      }
      sh[0] = s;
      sh[1] = i;
      sh[2] = b;
    }
    __syncthreads();
    const int s = sh[0], i = sh[1], b = sh[2];
    __syncthreads();
    if (s < 0) return;
    batch_tile<PF>(B, s, i, b * TILE + static_cast<int>(threadIdx.x));
  }
}

// Persistent rollout with warp-sized tiles: each warp takes its own 32-lane
// tile from the queue, so a warp whose lanes finish early never waits at a
// CTA barrier for the others.
__device__ __forceinline__ void tile_of(const BLaunch& B, uint32_t t, int tile, int* s, int* i,
                                        int* b) {
  int lo = 0, hi = B.c.S;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (static_cast<uint32_t>(B.tile_base[mid]) <= t) lo = mid; else hi = mid;
  }
  *s = B.order[lo];
  const int nb = (B.inst[*s].N + tile - 1) / tile;
  const int local = static_cast<int>(t) - B.tile_base[lo];
  *i = local / nb;
  *b = local - *i * nb;
}

template <int PF>
__global__ void __launch_bounds__(128) batch_rollout_warp_kernel(const BLaunch B) {
  const uint32_t total = B.queue[1];
  const int lane = static_cast<int>(threadIdx.x & 31);
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(B.queue, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= total) return;
    int s = 0, i = 0, b = 0;
    if (lane == 0) tile_of(B, t, 32, &s, &i, &b);
    s = __shfl_sync(0xffffffffu, s, 0);
    i = __shfl_sync(0xffffffffu, i, 0);
    b = __shfl_sync(0xffffffffu, b, 0);
    batch_tile<PF>(B, s, i, b * 32 + lane);
  }
}

// A warp tile of two candidate slots, 2p and 2p + 1 (the second absent when
// the round has an odd count), of instance s: each lane runs both
// trajectories of its scenario through run_lane_pair (one load of each
// disturbance, two independent step chains), or the one still running
// through run_lane, and reduces each slot as batch_tile does.  The prefetch
// depth is half the single lane's: each step issues two trajectories'
// instructions.  Called by all 32 lanes; returns are warp-uniform.
template <int PF>
__device__ __forceinline__ void batch_tile_pair(const BLaunch& B, int s, int p, int k) {
  const BInst I = B.inst[s];
  const int m = B.st[s].m;
  const size_t slotA = static_cast<size_t>(s) * B.c.M + 2 * p;
  const bool hasB = 2 * p + 1 < m;
  const size_t slotB = hasB ? slotA + 1 : slotA;
  volatile int32_t* deadA = B.cand_dead + slotA;
  volatile int32_t* deadB = B.cand_dead + slotB;
  const bool cand_stop = B.c.early_exit == RRG_EXIT_CANDIDATE;
  bool runA = B.cand_ss[slotA] != 0, runB = hasB && B.cand_ss[slotB] != 0;
  if (cand_stop) {
    const int da = __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 && runA ? *deadA : 0, 0);
    const int db = __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 && runB ? *deadB : 0, 0);
    runA = runA && !da;
    runB = runB && !db;
  }
  if (!runA && !runB) return;
  const bool active = k < I.N;
  const float eps = static_cast<float>(B.c.eps_abs);
  const float thr = B.c.early_exit != RRG_EXIT_NONE ? -eps : -inf_v<float>();
  float sm[2] = {inf_v<float>(), inf_v<float>()};
  unsigned st[2] = {0u, 0u};
  int jl[2] = {-1, -1}, en[2] = {LANE_REACHED_END, LANE_REACHED_END};
  if (active) {
    const BState& bs = B.st[s];
    const double p_atm = B.params[P_P_ATM];
    const RhsC<float> CA = B.cand_c32[slotA], CB = B.cand_c32[slotB];
    float za[4], zb[4];
    start_state<float>(CA, bs.x, p_atm, za[0], za[1], za[2], za[3]);
    start_state<float>(CB, bs.x, p_atm, zb[0], zb[1], zb[2], zb[3]);
    const float* d = (bs.cur ? B.d32b : B.d32) + I.off;
    const float dt = static_cast<float>(B.c.dt);
    if (runA && runB) {
      run_lane_pair<float, PF>(B.u32, CA, CB, d, k, I.N, I.H, I.H, za, zb, dt, thr, eps,
                               cand_stop ? deadA : nullptr, cand_stop ? deadB : nullptr, sm, st, en, jl);
    } else if (runA) {
      sm[0] = run_lane<float, PF>(B.u32, CA, d, k, I.N, I.H, 0, I.H, za[0], za[1], za[2], za[3],
                                  inf_v<float>(), dt, thr, cand_stop ? deadA : nullptr, &st[0], &en[0], eps,
                                  &jl[0]);
    } else {
      sm[1] = run_lane<float, PF>(B.u32, CB, d, k, I.N, I.H, 0, I.H, zb[0], zb[1], zb[2], zb[3],
                                  inf_v<float>(), dt, thr, cand_stop ? deadB : nullptr, &st[1], &en[1], eps,
                                  &jl[1]);
    }
    if (cand_stop && runA && sm[0] < thr) *deadA = 1;
    if (cand_stop && runB && sm[1] < thr) *deadB = 1;
  }
  if (runA) batch_reduce(B, slotA, k, active, sm[0], st[0], jl[0], eps, deadA);
  if (runB) batch_reduce(B, slotB, k, active, sm[1], st[1], jl[1], eps, deadB);
}

// Warp tiles of candidate pairs (the tile list counts ceil(m / 2) pairs per
// instance and scenario block).
template <int PF>
__global__ void __launch_bounds__(128) batch_rollout_warp_pair_kernel(const BLaunch B) {
  const uint32_t total = B.queue[1];
  const int lane = static_cast<int>(threadIdx.x & 31);
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(B.queue, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= total) return;
    int s = 0, p = 0, b = 0;
    if (lane == 0) tile_of(B, t, 32, &s, &p, &b);
    s = __shfl_sync(0xffffffffu, s, 0);
    p = __shfl_sync(0xffffffffu, p, 0);
    b = __shfl_sync(0xffffffffu, b, 0);
    batch_tile_pair<PF>(B, s, p, b * 32 + lane);
  }
}

// ---------------------------------------------------------------------------
// Two lanes per trajectory (warp-cooperative): the lanes 2q and 2q + 1 of a
// warp carry scenario q of a 16-scenario tile.  Both hold the whole state and
// form the same stage points and RK4 combination; of each right-hand side,
// role 0 evaluates the two linear flow derivatives (d_ca, d_sm) and role 1 the
// compressor-speed derivative with its power term and reciprocal (d_w), and
// the pair swaps them with two shuffles.  Each component is the expression of
// fc3_rhs_fast, so the trajectory equals the one-lane rollout bit for bit.
// The warp issues both roles' instructions for half as many trajectories, and
// the swap sits on every stage's dependency chain: the autotuner measures it
// against the one-lane variants.
__device__ __forceinline__ void fc3_rhs_split(const RhsU<float>& U, const RhsC<float>& C, int role,
                                              float z_ca, float z_w, float z_sm, float w, float x_pw,
                                              float& d_ca, float& d_w, float& d_sm) {
  float v0, v1 = 0.0f;
  if (role == 0) {
    v0 = U.a1 * z_sm + (C.c_ca - U.a12 * z_ca);
    v1 = U.g_w * z_w + ((C.c_sm + U.b3 * z_ca) - U.g_sm * z_sm);
  } else {
    const float W_cp = U.a_w * z_w + (C.W_r - U.a_p * z_sm);
    const float f = torque_factor<float>(U, pow_m1<float>(x_pw, U.e, U.pws), w);
    v0 = (C.e0 - U.e2 * z_w) - W_cp * f;
  }
  const float o0 = __shfl_xor_sync(0xffffffffu, v0, 1);
  const float o1 = __shfl_xor_sync(0xffffffffu, v1, 1);
  d_ca = role == 0 ? v0 : o0;
  d_sm = role == 0 ? v1 : o1;
  d_w = role == 0 ? o0 : v0;
}

// rk4_step_fast with the split right-hand side (the same stage points and
// combination, in the same order).  Called by all 32 lanes.
__device__ __forceinline__ void rk4_step_split(const RhsU<float>& U, const RhsC<float>& C,
                                               const StepC<float>& S, int role, float& q_ca, float& w,
                                               float& q_sm, float& w_abs, float e_ca, float e_w,
                                               float e_sm) {
  const float dt = S.dt, h2 = S.h2, h6 = S.h6, g2 = S.g2, g1 = S.g1;
  const float x1 = q_sm * U.inv_p_atm + C.x_r;
  float a1, b1, c1, a2, b2, c2, a3, b3, c3, a4, b4, c4;
  fc3_rhs_split(U, C, role, q_ca, w, q_sm, w_abs, x1, a1, b1, c1);
  fc3_rhs_split(U, C, role, q_ca + h2 * a1, w + h2 * b1, q_sm + h2 * c1, w_abs + h2 * b1, x1 + g2 * c1,
                a2, b2, c2);
  fc3_rhs_split(U, C, role, q_ca + h2 * a2, w + h2 * b2, q_sm + h2 * c2, w_abs + h2 * b2, x1 + g2 * c2,
                a3, b3, c3);
  const float p_ca = (q_ca + e_ca) + h6 * (a1 + 2.0f * (a2 + a3));
  const float p_w = (w + e_w) + h6 * (b1 + 2.0f * (b2 + b3));
  const float p_sm = (q_sm + e_sm) + h6 * (c1 + 2.0f * (c2 + c3));
  const float p_wa = p_w + C.r_w;
  fc3_rhs_split(U, C, role, q_ca + dt * a3, w + dt * b3, q_sm + dt * c3, w_abs + dt * b3, x1 + g1 * c3,
                a4, b4, c4);
  q_ca = p_ca + h6 * a4;
  w = p_w + h6 * b4;
  q_sm = p_sm + h6 * c4;
  w_abs = p_wa + h6 * b4;
}

// run_lane (steps 1..H from step 0) for a lane pair: the same blocks of PF
// steps, block tests, finiteness rule, band tracking and dead-flag use, so the
// decisions and the min slack of a trajectory that does not violate equal
// run_lane's.  The warp steps together while any of its pairs runs (the
// shuffles need every lane); a pair that has stopped, or a lane past the
// instance's scenarios (on = false), keeps stepping without recording.
template <int PF>
__device__ __forceinline__ float run_lane_split(const RhsU<float>& K, const RhsC<float>& C,
                                                const float* __restrict__ d, int k, bool on, int N, int H,
                                                int role, float& q_ca, float& w, float& q_sm, float& w_abs,
                                                float dt, float thr, const volatile int32_t* dead,
                                                unsigned* steps, float band, int* jlast) {
  float smin = inf_v<float>();
  int j = 0, jl = -1, j_stop = 0;
  bool run = on;
  {
    const float s0 = checked_slack<float>(C, q_ca, w, q_sm);
    smin = fmin(smin, s0);
    if (s0 < band) jl = 0;
    if (s0 < thr) run = false;
  }
  const StepC<float> S = step_consts<float>(K, dt);
  const size_t HN = static_cast<size_t>(H) * N;
  const float* pf = d + (on ? k : 0);  // in bounds for every lane
  float r0[PF], r1[PF], r2[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    if (u < H) {
      r0[u] = __ldg(pf);
      r1[u] = __ldg(pf + HN);
      r2[u] = __ldg(pf + 2 * HN);
    } else {
      r0[u] = r1[u] = r2[u] = 0.0f;
    }
    pf += N;
  }
  while (j + PF <= H && __any_sync(0xffffffffu, run)) {
    const int dead_now = (run && dead != nullptr) ? *dead : 0;
    float nf = 0.0f, bmin = inf_v<float>();
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const float e0 = r0[u], e1 = r1[u], e2 = r2[u];
      if (j + PF < H) {
        r0[u] = __ldg(pf);
        r1[u] = __ldg(pf + HN);
        r2[u] = __ldg(pf + 2 * HN);
      }
      pf += N;
      rk4_step_split(K, C, S, role, q_ca, w, q_sm, w_abs, e0, e1, e2);
      ++j;
      const float s = C.y_scale * (q_sm - q_ca) + C.s_off;
      bmin = fmin(bmin, s);
      nf = fma_rn(s, 0.0f, nf);
    }
    if (run) {
      nf = fma_rn(q_ca, 0.0f, fma_rn(w, 0.0f, fma_rn(q_sm, 0.0f, nf)));
      if (nf != nf) bmin = -inf_v<float>();
      smin = fmin(smin, bmin);
      if (bmin < band) jl = j;
      j_stop = j;
      if (smin < thr || (dead_now != 0 && j < H)) run = false;
    }
  }
  const float* dp = d + static_cast<size_t>(j) * N + (on ? k : 0);
  while (j < H && __any_sync(0xffffffffu, run)) {
    const float e0 = __ldg(dp), e1 = __ldg(dp + HN), e2 = __ldg(dp + 2 * HN);
    dp += N;
    rk4_step_split(K, C, S, role, q_ca, w, q_sm, w_abs, e0, e1, e2);
    ++j;
    if (run) {
      const float s = checked_slack<float>(C, q_ca, w, q_sm);
      smin = fmin(smin, s);
      if (s < band) jl = j;
      j_stop = j;
      if (s < thr) run = false;
    }
  }
  *steps = static_cast<unsigned>(j_stop);
  *jlast = jl;
  return smin;
}

// A warp tile of 16 scenarios of candidate slot (s, i), two lanes each:
// batch_tile's classification and reduction with role 0's lanes as the
// trajectories (role 1's take no part in the flags, the min or the step
// count).  Called by all 32 lanes; returns are warp-uniform.
template <int PF>
__device__ __forceinline__ void batch_tile_split(const BLaunch& B, int s, int i, int k, int role) {
  const BInst I = B.inst[s];
  const size_t slot = static_cast<size_t>(s) * B.c.M + i;
  if (!B.cand_ss[slot]) return;
  volatile int32_t* dead = B.cand_dead + slot;
  const bool cand_stop = B.c.early_exit == RRG_EXIT_CANDIDATE;
  if (cand_stop) {
    const int dead0 = __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 ? *dead : 0, 0);
    if (dead0) return;
  }
  const bool on = k < I.N;
  const float eps = static_cast<float>(B.c.eps_abs);
  const float thr = B.c.early_exit != RRG_EXIT_NONE ? -eps : -inf_v<float>();
  const BState& st = B.st[s];
  const double p_atm = B.params[P_P_ATM];
  const RhsC<float> C = B.cand_c32[slot];
  float q_ca, w, q_sm, w_abs;
  start_state<float>(C, st.x, p_atm, q_ca, w, q_sm, w_abs);
  const float* d = (st.cur ? B.d32b : B.d32) + I.off;
  unsigned steps = 0;
  int jlast = -1;
  const float smin = run_lane_split<PF>(B.u32, C, d, k, on, I.N, I.H, role, q_ca, w, q_sm, w_abs,
                                        static_cast<float>(B.c.dt), thr, cand_stop ? dead : nullptr, &steps,
                                        eps, &jlast);
  const bool mine = on && role == 0;
  if (cand_stop && mine && smin < thr) *dead = 1;
  batch_reduce(B, slot, k, mine, smin, mine ? steps : 0u, jlast, eps, dead);
}

// Warp tiles of 16 scenarios at two lanes per trajectory.
template <int PF>
__global__ void __launch_bounds__(128) batch_rollout_split_kernel(const BLaunch B) {
  const uint32_t total = B.queue[1];
  const int lane = static_cast<int>(threadIdx.x & 31);
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(B.queue, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= total) return;
    int s = 0, i = 0, b = 0;
    if (lane == 0) tile_of(B, t, 16, &s, &i, &b);
    s = __shfl_sync(0xffffffffu, s, 0);
    i = __shfl_sync(0xffffffffu, i, 0);
    b = __shfl_sync(0xffffffffu, b, 0);
    batch_tile_split<PF>(B, s, i, b * 16 + (lane >> 1), lane & 1);
  }
}
__global__ void __launch_bounds__(64) batch_recheck_kernel(const BLaunch B) {
  const uint32_t count = min(*B.recheck_count, static_cast<uint32_t>(B.recheck_cap));
  const double p_atm = B.params[P_P_ATM];
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    const uint2 en = B.recheck_list[e];
    const size_t slot = en.x;
    const int k = static_cast<int>(en.y);
    if (!B.cand_ok[slot]) continue;
    const int s = static_cast<int>(slot / B.c.M);
    const BState& st = B.st[s];
    ScenSrc src;
    src.d64_valid = 0;
    src.pad = 0;
    src.seed = st.seed_p[st.cur];
    src.update = st.update_p[st.cur];
    src.base = 0;
    src.amp[0] = B.c.amp[0];
    src.amp[1] = B.c.amp[1];
    src.amp[2] = B.c.amp[2];
    unsigned steps = 0;
    const RhsC<double> C = B.cand_c64[slot];
    double q_ca, w, q_sm, w_abs;
    start_state<double>(C, st.x, p_atm, q_ca, w, q_sm, w_abs);
    const double smin = run_lane_philox(B.u64, C, src, k,
                                        min(static_cast<int>(B.recheck_jlast[e]), B.inst[s].H),
                                        q_ca, w, q_sm, w_abs, B.c.dt,
                                        B.c.early_exit != RRG_EXIT_NONE ? 0.0 : -inf_v<double>(),
                                        &steps);
    if (!(smin >= 0.0)) B.cand_ok[slot] = 0;
    atomicMin(B.cand_min + slot, dkey(smin));
    atomicAdd(&B.stats->lane_steps, static_cast<unsigned long long>(steps));
    atomicAdd(&B.stats->lane_steps_fp64, static_cast<unsigned long long>(steps));
    atomicAdd(&B.stats->rechecked, 1ull);
  }
}

// Alg. 3 / k-section decision from the evaluated round (as the
// single-problem search), the next round's candidates and tiles; `final`
// also writes every instance's result at index t * S + s.
__global__ void __launch_bounds__(kDecideThreads)
batch_decide_kernel(const BLaunch B, int final, int tile, int rows, double* __restrict__ v_out,
                    double* __restrict__ k_out, int32_t* __restrict__ f_out) {
  const int s = threadIdx.x;
  const int M = B.c.M;
  if (s < B.c.S) {
    BState& st = B.st[s];
    double* kap = B.cand_kappa + static_cast<size_t>(s) * M;
    const int32_t* ok = B.cand_ok + static_cast<size_t>(s) * M;
    if (!st.done && st.m > 0) {
      const int m = st.m;
      int best = -1;
      for (int i = 0; i < m; ++i)
        if (ok[i]) best = i;
      int next = 0;
      if (B.c.search == RRG_SEARCH_SPEC_BISECT) {
        btree_walk(st, ok, m, B.c.n_bisect);
        if (!st.done) next = btree_plan(st, B.c.width, B.c.n_bisect, kap);
        if (next == 0) st.done = 1;
      } else if (B.c.search == RRG_SEARCH_GRID) {
        if (best >= 0) { st.kappa_opt = kap[best]; st.any = 1; }
        st.done = 1;
      } else if (st.round == 0 && (best < 0 || best == m - 1)) {
        if (best >= 0) { st.kappa_opt = kap[best]; st.any = 1; }
        st.done = 1;
      } else {
        if (st.round == 0) {
          st.any = 1;
          st.kappa_opt = kap[best];
          st.lo = kap[best];
          st.hi = kap[best + 1];
        } else if (best < 0) {
          st.hi = kap[0];
        } else {
          st.kappa_opt = kap[best];
          st.lo = kap[best];
          if (best < m - 1) st.hi = kap[best + 1];
        }
        if (st.round + 1 >= B.c.n_rounds) st.done = 1;
        else next = interior_points(kap, M, st.lo, st.hi);
      }
      st.round += 1;
      st.m = st.done ? 0 : next;
    }
    if (final) {
      st.done = 1;
      st.m = 0;
      st.flags = (st.any ? 0 : 1) | (st.invalid ? 2 : 0);
      const double kk = st.invalid ? 0.0 : st.kappa_opt;
      st.kappa_opt = kk;
      st.v_out = st.invalid ? st.v_prev : governed(st.v_prev, st.r, kk);
      const unsigned long long o =
          (B.t_dev ? *B.t_dev : 0ull) * static_cast<unsigned long long>(B.c.S) + s;
      if (v_out) v_out[o] = st.v_out;
      if (k_out) k_out[o] = kk;
      if (f_out) f_out[o] = st.flags;
    }
  }
  __syncthreads();
  build_tiles(B, tile, rows);
}

// Simulated plants: x_{t+1} = RK4(x_t, v_t) + d_plant(seed + s, update),
// then the loop counter advances (one block).
__global__ void __launch_bounds__(kDecideThreads)
batch_plant_kernel(const BLaunch B, uint64_t seed, uint64_t base, const double* __restrict__ amp,
                   double* __restrict__ x_out) {
  const int s = threadIdx.x;
  const unsigned long long t = *B.t_dev;
  if (s < B.c.S) {
    BState& st = B.st[s];
    const double v = st.v_out;
    const U64x4 r = philox4x64_10(0ull, 0ull, base + t, 1ull, seed + static_cast<uint64_t>(s), 0ull);
    const double x[3] = {st.x[0], st.x[1], st.x[2]};
    double xn[3];
    plant_step_fast(B.k64, B.u64, B.params, B.c.dt, v, x, uniform_sym(r.w[0], amp[0]),
                    uniform_sym(r.w[1], amp[1]), uniform_sym(r.w[2], amp[2]), xn);
    st.lx[0] = xn[0];
    st.lx[1] = xn[1];
    st.lx[2] = xn[2];
    st.lv = v;
    if (x_out) {
      double* xo = x_out + ((t + 1) * static_cast<unsigned long long>(B.c.S) + s) * 3;
      xo[0] = st.lx[0];
      xo[1] = st.lx[1];
      xo[2] = st.lx[2];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *B.t_dev = t + 1;
}

__global__ void batch_loop_init_kernel(const BLaunch B, const double* __restrict__ x0,
                                       const double* __restrict__ v0, double* __restrict__ x_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) *B.t_dev = 0ull;
  if (s >= B.c.S) return;
  BState& st = B.st[s];
  st.lx[0] = x0[3 * s];
  st.lx[1] = x0[3 * s + 1];
  st.lx[2] = x0[3 * s + 2];
  st.lv = v0[s];
  if (x_out) {
    x_out[3 * s] = st.lx[0];
    x_out[3 * s + 1] = st.lx[1];
    x_out[3 * s + 2] = st.lx[2];
  }
}

// Rollout variants the autotuner chooses from: threads (= scenario lanes)
// per tile, the disturbance prefetch depth, and candidate slots per tile.
struct Variant {
  int tile, pf, rows;
  void (*kernel)(const BLaunch);
};
// tile = 32: warp tiles (CTAs of 4 warps, no CTA barrier); rows = 2: two
// candidates per thread; tile = 16: warp tiles of 16 scenarios, two lanes
// per trajectory
const Variant kVariants[RRG_BATCH_VARIANTS] = {
    {64, 8, 1, batch_rollout_kernel<64, 8>},   {64, 16, 1, batch_rollout_kernel<64, 16>},
    {128, 8, 1, batch_rollout_kernel<128, 8>}, {128, 16, 1, batch_rollout_kernel<128, 16>},
    {256, 8, 1, batch_rollout_kernel<256, 8>}, {256, 16, 1, batch_rollout_kernel<256, 16>},
    {32, 8, 1, batch_rollout_warp_kernel<8>},  {32, 16, 1, batch_rollout_warp_kernel<16>},
    {32, 8, 2, batch_rollout_warp_pair_kernel<8>}, {16, 8, 1, batch_rollout_split_kernel<8>},
};
constexpr int block_threads(int tile) { return tile <= 32 ? 128 : tile; }

}  // namespace
}  // namespace rrg

using namespace rrg;

struct rrg_batch_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  rrg_config cfg{};
  double params[RRG_NPARAM]{};
  BLaunch B{};
  std::vector<BInst> inst;
  int variant = 3;             // 128 lanes per tile, prefetch 16
  int sms = 0;                 // streaming multiprocessors of the device (queried)
  int grid[RRG_BATCH_VARIANTS]{};
  size_t lanes = 0;            // sum of M N_s
  // device memory
  double* params_dev = nullptr;
  PowSeries* pws = nullptr;
  BInst* inst_dev = nullptr;
  int32_t* order_dev = nullptr;
  BState* st = nullptr;
  float* d32 = nullptr;
  float* d32b = nullptr;       // second scenario pair, allocated by the first closed loop
  size_t d32_elems = 0;
  cudaStream_t side = nullptr; // draws update t + 1 while update t searches
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool cl_next_ready = false;
  uint64_t cl_seed = 0, cl_t0 = 0;
  double* cand_kappa = nullptr;
  double* cand_v = nullptr;
  RhsC<double>* cand_c64 = nullptr;
  RhsC<float>* cand_c32 = nullptr;
  int32_t* cand_ok = nullptr;
  int32_t* cand_dead = nullptr;
  int32_t* cand_ss = nullptr;
  unsigned long long* cand_min = nullptr;
  int32_t* tile_base = nullptr;
  uint32_t* queue = nullptr;
  uint2* recheck_list = nullptr;
  uint32_t* recheck_jlast = nullptr;
  uint32_t* recheck_count = nullptr;
  DevStats* stats = nullptr;
  unsigned long long* t_dev = nullptr;
  double* amp_dev = nullptr;
  double* io_h = nullptr;      // pinned staging for the plant amplitudes
  // graph of one closed-loop update
  cudaGraphExec_t cl_exec = nullptr;
  const void* cl_key[5] = {};
  uint64_t cl_key_seed = 0, cl_key_t0 = 0;
  int cl_key_variant = -1, cl_key_width = -1;
  uint64_t cl_per = 0, cl_rl_per = 0;
  // counters and profiling
  uint64_t launches = 0, rollout_launches = 0, rounds = 0;
  bool profiling = false, capturing = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_roll;
  double rollout_ms = 0.0;
  uint64_t timed_rollouts = 0;
  std::string err;
};

namespace {

thread_local std::string g_batch_create_error;

int bset_err(rrg_batch_ctx* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf; else g_batch_create_error = buf;
  return code;
}

#define BCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return bset_err(h, RRG_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

struct BDeviceGuard {
  int prev = -1;
  explicit BDeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~BDeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

void bfree_all(rrg_batch_ctx* h) {
  void* ptrs[] = {h->params_dev, h->pws, h->inst_dev, h->order_dev, h->st, h->d32, h->d32b,
                  h->cand_kappa,
                  h->cand_v, h->cand_c64, h->cand_c32, h->cand_ok, h->cand_dead, h->cand_ss,
                  h->cand_min, h->tile_base, h->queue, h->recheck_list, h->recheck_jlast,
                  h->recheck_count,
                  h->stats, h->t_dev, h->amp_dev};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->io_h) cudaFreeHost(h->io_h);
  for (auto& e : h->ev_free) cudaEventDestroy(e);
  for (auto& pr : h->ev_roll) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  if (h->cl_exec) cudaGraphExecDestroy(h->cl_exec);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

cudaEvent_t btake_event(rrg_batch_ctx* h) {
  if (!h->ev_free.empty()) {
    cudaEvent_t e = h->ev_free.back();
    h->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Folds the timed rollout launches into rollout_ms (after a synchronize).
void bcollect(rrg_batch_ctx* h) {
  for (auto& pr : h->ev_roll) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
      h->rollout_ms += ms;
      h->timed_rollouts++;
    }
    h->ev_free.push_back(pr.first);
    h->ev_free.push_back(pr.second);
  }
  h->ev_roll.clear();
}

// Rounds of one update's search: 1 for Alg. 3, n_rounds for the k-section;
// for the speculative bisection enough trees of the current width to finish
// Alg. 1's n_bisect iterations from kappa = 1 (instances that finish sooner
// skip the rest: their rounds have no tiles).
int batch_rounds(const rrg_batch_ctx* h) {
  const BCfg& c = h->B.c;
  if (c.search == RRG_SEARCH_GRID) return 1;
  if (c.search != RRG_SEARCH_SPEC_BISECT) return c.n_rounds;
  int d0 = 1, d1 = 1;
  while (d0 + 1 <= c.n_bisect && (1 << d0) <= c.width) ++d0;            // 2^(d-1) nodes from the root
  while (d1 + 1 <= c.n_bisect && (1 << (d1 + 1)) - 1 <= c.width) ++d1;  // 2^d - 1 nodes below it
  const int rest = c.n_bisect - d0;
  return 1 + (rest > 0 ? (rest + d1 - 1) / d1 : 0);
}

int enqueue_rollout(rrg_batch_ctx* h) {
  const Variant& v = kVariants[h->variant];
  const bool timed = h->profiling && !h->capturing;
  cudaEvent_t a = nullptr, b = nullptr;
  if (timed) {
    a = btake_event(h);
    b = btake_event(h);
    if (a && b) BCK(cudaEventRecord(a, h->stream));
  }
  v.kernel<<<h->grid[h->variant], block_threads(v.tile), 0, h->stream>>>(h->B);
  BCK(cudaGetLastError());
  if (timed && a && b) {
    BCK(cudaEventRecord(b, h->stream));
    h->ev_roll.emplace_back(a, b);
  }
  h->launches++;
  h->rollout_launches++;
  return RRG_OK;
}

// One update of every instance: sample, then the rounds of the search.
int enqueue_sample(rrg_batch_ctx* h, uint64_t seed, uint64_t base, cudaStream_t stream) {
  int blocks = 1;
  for (const BInst& I : h->inst) {
    const size_t hn = static_cast<size_t>(I.H) * I.N;
    blocks = std::max(blocks, static_cast<int>(std::min<size_t>((hn + 255) / 256, 64)));
  }
  batch_sample_kernel<<<dim3(blocks, h->B.c.S), 256, 0, stream>>>(h->B, seed, base);
  BCK(cudaGetLastError());
  h->launches++;
  return RRG_OK;
}

// The search of one update of every instance on scenarios already drawn for
// update base + t.
int enqueue_search_all(rrg_batch_ctx* h, const double* d_x, const double* d_r, const double* d_vp,
                       uint64_t base, double* v_out, double* k_out, int32_t* f_out) {
  const BLaunch& B = h->B;
  const int S = B.c.S;
  const int tile = kVariants[h->variant].tile, rows = kVariants[h->variant].rows;
  batch_begin_kernel<<<1, kDecideThreads, 0, h->stream>>>(B, d_x, d_r, d_vp, base, tile, rows);
  BCK(cudaGetLastError());
  h->launches++;
  const int rounds = batch_rounds(h);
  const int prep_blocks = (S * B.c.M + 127) / 128;
  for (int r = 0; r < rounds; ++r) {
    batch_prepare_kernel<<<prep_blocks, 128, 0, h->stream>>>(B);
    BCK(cudaGetLastError());
    int rc = enqueue_rollout(h);
    if (rc != RRG_OK) return rc;
    batch_recheck_kernel<<<2 * h->sms, 64, 0, h->stream>>>(B);
    BCK(cudaGetLastError());
    const int final = r == rounds - 1;
    batch_decide_kernel<<<1, kDecideThreads, 0, h->stream>>>(B, final, tile, rows, v_out, k_out, f_out);
    BCK(cudaGetLastError());
    h->launches += 3;
    h->rounds++;
  }
  return RRG_OK;
}

// Sample, then search (one update of every instance, single stream).
int enqueue_update(rrg_batch_ctx* h, const double* d_x, const double* d_r, const double* d_vp,
                   uint64_t seed, uint64_t base, double* v_out, double* k_out, int32_t* f_out) {
  int rc = enqueue_sample(h, seed, base, h->stream);
  if (rc != RRG_OK) return rc;
  return enqueue_search_all(h, d_x, d_r, d_vp, base, v_out, k_out, f_out);
}

}  // namespace

extern "C" {

int rrg_batch_create(const double* model_params, int n_params, const rrg_config* cfg,
                     int n_instances, const int32_t* n_scenarios, const int32_t* horizons,
                     void* cuda_stream, rrg_batch_handle* out) {
  g_batch_create_error.clear();
  rrg_batch_ctx* h = nullptr;
  if (!out) return bset_err(h, RRG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!model_params || n_params != RRG_NPARAM)
    return bset_err(h, RRG_EINVAL, "model_params must hold %d values", RRG_NPARAM);
  for (int i = 0; i < RRG_NPARAM; ++i)
    if (!std::isfinite(model_params[i])) return bset_err(h, RRG_EINVAL, "model_params[%d] not finite", i);
  int rc = check_config(cfg);
  if (rc != RRG_OK) return bset_err(h, rc, "%s", rrg_last_error(nullptr));
  if (cfg->search != RRG_SEARCH_GRID && cfg->search != RRG_SEARCH_KSECTION &&
      cfg->search != RRG_SEARCH_SPEC_BISECT)
    return bset_err(h, RRG_ENOTIMPL, "batched instances run RRG_SEARCH_GRID, RRG_SEARCH_KSECTION or "
                    "RRG_SEARCH_SPEC_BISECT");
  if (cfg->search == RRG_SEARCH_SPEC_BISECT && cfg->n_bisect > 62)
    return bset_err(h, RRG_EINVAL, "n_bisect must be <= 62");
  if (cfg->precision != RRG_FP32_RECHECK)
    return bset_err(h, RRG_ENOTIMPL, "batched instances run RRG_FP32_RECHECK");
  if (cfg->param_unc_rel != 0.0 || cfg->scenarios_in_register != 0 || cfg->scenario_base != 0)
    return bset_err(h, RRG_ENOTIMPL, "batched instances have no parametric uncertainty and store "
                    "their scenarios (param_unc_rel, scenarios_in_register and scenario_base must be 0)");
  if (n_instances < 1 || n_instances > kMaxInst)
    return bset_err(h, RRG_EINVAL, "n_instances must be in [1, %d]", kMaxInst);
  if (!n_scenarios || !horizons) return bset_err(h, RRG_EINVAL, "n_scenarios and horizons must be non-NULL");
  const int M = cfg->max_candidates;
  std::vector<BInst> inst(n_instances);
  unsigned long long lanes = 0, elems = 0;
  for (int s = 0; s < n_instances; ++s) {
    if (n_scenarios[s] < 1 || horizons[s] < 1)
      return bset_err(h, RRG_EINVAL, "instance %d: n_scenarios and horizon must be >= 1", s);
    inst[s].N = n_scenarios[s];
    inst[s].H = horizons[s];
    inst[s].off = static_cast<long long>(elems);
    const unsigned long long e = 3ull * static_cast<unsigned long long>(horizons[s]) *
                                 static_cast<unsigned long long>(n_scenarios[s]);
    elems += (e + 31ull) & ~31ull;  // 128-byte aligned blocks
    lanes += static_cast<unsigned long long>(M) * static_cast<unsigned long long>(n_scenarios[s]);
  }
  if (lanes >= (1ull << 31)) return bset_err(h, RRG_EINVAL, "sum of max_candidates * n_scenarios >= 2^31");

  h = new (std::nothrow) rrg_batch_ctx();
  if (!h) return bset_err(nullptr, RRG_ENOMEM, "host allocation failed");
  h->cfg = *cfg;
  h->inst = inst;
  h->lanes = lanes;
  std::memcpy(h->params, model_params, sizeof h->params);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      h->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
      h->own_stream = e == cudaSuccess;
    }
  }
  const size_t S = n_instances, SM = S * M;
  auto alloc = [&](auto** p, size_t n) {
    if (e == cudaSuccess) {
      e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(**p) + 16);
      if (e != cudaSuccess) cudaGetLastError();
    }
  };
  alloc(&h->params_dev, RRG_NPARAM);
  alloc(&h->pws, 1);
  alloc(&h->inst_dev, S);
  alloc(&h->order_dev, S);
  alloc(&h->st, S);
  alloc(&h->d32, static_cast<size_t>(elems));
  h->d32_elems = static_cast<size_t>(elems);
  alloc(&h->cand_kappa, SM);
  alloc(&h->cand_v, SM);
  alloc(&h->cand_c64, SM);
  alloc(&h->cand_c32, SM);
  alloc(&h->cand_ok, SM);
  alloc(&h->cand_dead, SM);
  alloc(&h->cand_ss, SM);
  alloc(&h->cand_min, SM);
  alloc(&h->tile_base, S + 1);
  alloc(&h->queue, 2);
  alloc(&h->recheck_list, static_cast<size_t>(lanes));
  alloc(&h->recheck_jlast, static_cast<size_t>(lanes));
  alloc(&h->recheck_count, 1);
  alloc(&h->stats, 1);
  alloc(&h->t_dev, 1);
  alloc(&h->amp_dev, 3);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->io_h), 4 * sizeof(double));
  // longest horizon first, then most scenarios (a longest-processing-time
  // order for the tile queue)
  std::vector<int32_t> order(S);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (inst[a].H != inst[b].H) return inst[a].H > inst[b].H;
    return inst[a].N > inst[b].N;
  });
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->params_dev, h->params, sizeof h->params, cudaMemcpyHostToDevice, h->stream);
  PowSeries ps;
  make_pow_series((h->params[P_GAMMA] - 1.0) / h->params[P_GAMMA], &ps);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->pws, &ps, sizeof ps, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->inst_dev, inst.data(), S * sizeof(BInst), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->order_dev, order.data(), S * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->st, 0, S * sizeof(BState), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->stats, 0, sizeof(DevStats), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->t_dev, 0, sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d32, 0, static_cast<size_t>(elems) * sizeof(float), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  int nsm = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  h->sms = nsm;
  for (int v = 0; v < RRG_BATCH_VARIANTS && e == cudaSuccess; ++v) {
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kVariants[v].kernel,
                                                      block_threads(kVariants[v].tile), 0);
    h->grid[v] = std::max(1, per) * nsm;
  }
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? RRG_ENOMEM : RRG_ECUDA;
    bset_err(nullptr, code, "rrg_batch_create: %s", cudaGetErrorString(e));
    bfree_all(h);
    delete h;
    return code;
  }
  BLaunch& B = h->B;
  B.stream = h->stream;
  B.c.S = n_instances;
  B.c.M = M;
  B.c.n_rounds = cfg->n_rounds;
  B.c.search = cfg->search;
  B.c.n_bisect = cfg->n_bisect;
  B.c.width = M;
  B.c.ss_check = cfg->ss_check;
  B.c.early_exit = cfg->early_exit;
  B.c.dt = cfg->dt;
  B.c.y_min = cfg->y_min;
  B.c.eps_ss = cfg->eps_ss;
  B.c.y_c = cfg->y_c;
  B.c.eps_abs = cfg->recheck_eps_rel * std::fabs(cfg->y_min);
  for (int i = 0; i < 3; ++i) B.c.amp[i] = cfg->dist_amp[i];
  B.params = h->params_dev;
  fold_constants(h->params, &B.k64, &B.k32);
  B.k64.pws = h->pws;
  fold_rhs(B.k64, &B.u64, &B.u32);
  B.inst = h->inst_dev;
  B.order = h->order_dev;
  B.st = h->st;
  B.d32 = h->d32;
  B.d32b = nullptr;
  B.cand_kappa = h->cand_kappa;
  B.cand_v = h->cand_v;
  B.cand_c64 = h->cand_c64;
  B.cand_c32 = h->cand_c32;
  B.cand_ok = h->cand_ok;
  B.cand_dead = h->cand_dead;
  B.cand_ss = h->cand_ss;
  B.cand_min = h->cand_min;
  B.tile_base = h->tile_base;
  B.queue = h->queue;
  B.recheck_list = h->recheck_list;
  B.recheck_jlast = h->recheck_jlast;
  B.recheck_count = h->recheck_count;
  B.recheck_cap = lanes;
  B.stats = h->stats;
  B.t_dev = nullptr;
  *out = h;
  return RRG_OK;
}

int rrg_batch_destroy(rrg_batch_handle h) {
  if (!h) return RRG_OK;
  int rc = RRG_OK;
  {
    BDeviceGuard g(h->device);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = RRG_ECUDA;
    bfree_all(h);
  }
  delete h;
  return rc;
}

const char* rrg_batch_last_error(rrg_batch_handle h) {
  return h ? h->err.c_str() : g_batch_create_error.c_str();
}

int rrg_batch_step_dev(rrg_batch_handle h, const double* d_x, const double* d_r,
                       const double* d_v_prev, uint64_t seed, uint64_t update_index,
                       double* d_v_t, double* d_kappa, int32_t* d_flags) {
  if (!h) return RRG_EINVAL;
  if (!d_x || !d_r || !d_v_prev) return bset_err(h, RRG_EINVAL, "d_x, d_r and d_v_prev must be non-NULL");
  BDeviceGuard g(h->device);
  h->B.t_dev = nullptr;
  h->cl_next_ready = false;  // this draw may overwrite a closed loop's next update
  return enqueue_update(h, d_x, d_r, d_v_prev, seed, update_index, d_v_t, d_kappa, d_flags);
}

int rrg_batch_closed_loop_dev(rrg_batch_handle h, const double* d_x0, const double* d_v0,
                              const double* d_r_seq, int T, uint64_t seed, uint64_t t0,
                              const double* plant_amp, int use_graph, double* d_v_out,
                              double* d_kappa_out, int32_t* d_flags_out, double* d_x_out) {
  if (!h) return RRG_EINVAL;
  if (T < 0 || !d_r_seq || !plant_amp || (d_x0 && !d_v0))
    return bset_err(h, RRG_EINVAL, "T >= 0, d_r_seq and plant_amp non-NULL, d_v0 with d_x0");
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(plant_amp[i]) || plant_amp[i] < 0.0)
      return bset_err(h, RRG_EINVAL, "plant_amp must be finite and >= 0");
  BDeviceGuard g(h->device);
  // the second scenario pair and the side stream, on first use
  if (!h->B.d32b) {
    if (!h->d32b) BCK(cudaMalloc(reinterpret_cast<void**>(&h->d32b), h->d32_elems * sizeof(float) + 16));
    if (!h->side) BCK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    if (!h->ev_fork) BCK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    if (!h->ev_join) BCK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    h->B.d32b = h->d32b;
    h->cl_next_ready = false;
    if (h->cl_exec) {
      cudaGraphExecDestroy(h->cl_exec);
      h->cl_exec = nullptr;
    }
  }
  h->B.t_dev = h->t_dev;
  std::memcpy(h->io_h, plant_amp, 3 * sizeof(double));
  BCK(cudaMemcpyAsync(h->amp_dev, h->io_h, 3 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  if (d_x0) {
    batch_loop_init_kernel<<<(h->B.c.S + 127) / 128, 128, 0, h->stream>>>(h->B, d_x0, d_v0, d_x_out);
    BCK(cudaGetLastError());
    h->launches++;
    h->cl_next_ready = false;
  }
  if (T == 0) return RRG_OK;
  // the first update's scenarios, unless the previous call of this run drew them
  if (!(h->cl_next_ready && h->cl_seed == seed && h->cl_t0 == t0)) {
    int rc = enqueue_sample(h, seed, t0, h->stream);
    if (rc != RRG_OK) return rc;
  }
  h->cl_seed = seed;
  h->cl_t0 = t0;
  h->cl_next_ready = true;
  // one update: draw update t + 1 on the side stream (into the other pair)
  // while update t searches; join before the plant advances the counter the
  // sampler reads
  auto one = [&]() -> int {
    BCK(cudaEventRecord(h->ev_fork, h->stream));
    BCK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    int rc = enqueue_sample(h, seed, t0 + 1, h->side);
    if (rc != RRG_OK) return rc;
    BCK(cudaEventRecord(h->ev_join, h->side));
    rc = enqueue_search_all(h, nullptr, d_r_seq, nullptr, t0, d_v_out, d_kappa_out, d_flags_out);
    if (rc != RRG_OK) return rc;
    BCK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    batch_plant_kernel<<<1, kDecideThreads, 0, h->stream>>>(h->B, seed, t0, h->amp_dev, d_x_out);
    BCK(cudaGetLastError());
    h->launches++;
    return RRG_OK;
  };
  if (!use_graph) {
    for (int t = 0; t < T; ++t) {
      int rc = one();
      if (rc != RRG_OK) return rc;
    }
    return RRG_OK;
  }
  const void* key[5] = {d_r_seq, d_v_out, d_kappa_out, d_flags_out, d_x_out};
  const bool hit = h->cl_exec && std::memcmp(key, h->cl_key, sizeof key) == 0 &&
                   h->cl_key_seed == seed && h->cl_key_t0 == t0 && h->cl_key_variant == h->variant &&
                   h->cl_key_width == h->B.c.width;
  if (!hit) {
    if (h->cl_exec) {
      cudaGraphExecDestroy(h->cl_exec);
      h->cl_exec = nullptr;
    }
    const uint64_t l0 = h->launches, r0 = h->rollout_launches, rd0 = h->rounds;
    cudaGraph_t graph = nullptr;
    BCK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    int rc = one();
    h->capturing = false;
    cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
    if (rc != RRG_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (ce != cudaSuccess) return bset_err(h, RRG_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&h->cl_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      h->cl_exec = nullptr;
      return bset_err(h, RRG_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    }
    h->cl_per = h->launches - l0;
    h->cl_rl_per = h->rollout_launches - r0;
    h->launches = l0;
    h->rollout_launches = r0;
    h->rounds = rd0;
    std::memcpy(h->cl_key, key, sizeof key);
    h->cl_key_seed = seed;
    h->cl_key_t0 = t0;
    h->cl_key_variant = h->variant;
    h->cl_key_width = h->B.c.width;
  }
  for (int t = 0; t < T; ++t) {
    const cudaError_t ce = cudaGraphLaunch(h->cl_exec, h->stream);
    if (ce != cudaSuccess) return bset_err(h, RRG_ECUDA, "graph launch: %s", cudaGetErrorString(ce));
    h->launches += h->cl_per;
    h->rollout_launches += h->cl_rl_per;
    h->rounds += batch_rounds(h);
  }
  return RRG_OK;
}

int rrg_batch_set_variant(rrg_batch_handle h, int variant) {
  if (!h) return RRG_EINVAL;
  if (variant < 0 || variant >= RRG_BATCH_VARIANTS)
    return bset_err(h, RRG_EINVAL, "variant must be in [0, %d)", RRG_BATCH_VARIANTS);
  h->variant = variant;
  return RRG_OK;
}

int rrg_batch_get_variant(rrg_batch_handle h, int* variant, int* tile_lanes, int* prefetch) {
  if (!h) return RRG_EINVAL;
  if (variant) *variant = h->variant;
  if (tile_lanes) *tile_lanes = kVariants[h->variant].tile;
  if (prefetch) *prefetch = kVariants[h->variant].pf;
  return RRG_OK;
}

int rrg_batch_set_width(rrg_batch_handle h, int width) {
  if (!h) return RRG_EINVAL;
  if (h->cfg.search != RRG_SEARCH_SPEC_BISECT)
    return bset_err(h, RRG_EINVAL, "the width is a parameter of RRG_SEARCH_SPEC_BISECT only (for the grid "
                    "searches it is the grid size, fixed at creation)");
  if (width < 1 || width > h->B.c.M) return bset_err(h, RRG_EINVAL, "width must be in [1, max_candidates]");
  BDeviceGuard g(h->device);
  BCK(cudaStreamSynchronize(h->stream));
  h->B.c.width = width;
  return RRG_OK;
}

int rrg_batch_get_width(rrg_batch_handle h, int* width) {
  if (!h || !width) return RRG_EINVAL;
  *width = h->B.c.width;
  return RRG_OK;
}

int rrg_batch_autotune_width(rrg_batch_handle h, const double* d_x, const double* d_r,
                             const double* d_v_prev, uint64_t seed, uint64_t update_index, int repeats,
                             int* width_out, int32_t* widths, double* ms_out, int* n_out) {
  if (!h) return RRG_EINVAL;
  if (h->cfg.search != RRG_SEARCH_SPEC_BISECT)
    return bset_err(h, RRG_EINVAL, "the width is tuned for RRG_SEARCH_SPEC_BISECT only");
  if (!d_x || !d_r || !d_v_prev || repeats < 1)
    return bset_err(h, RRG_EINVAL, "d_x, d_r, d_v_prev non-NULL and repeats >= 1");
  BDeviceGuard g(h->device);
  h->B.t_dev = nullptr;
  h->cl_next_ready = false;
  BCK(cudaStreamSynchronize(h->stream));
  bcollect(h);
  // the tree sizes: 2^d - 1 and 2^(d-1) (from a kappa = 1 root) nodes
  std::vector<int> cand;
  for (int w = 1; w <= h->B.c.M; w *= 2) {
    cand.push_back(w);
    if (2 * w - 1 > w && 2 * w - 1 <= h->B.c.M) cand.push_back(2 * w - 1);
  }
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  if (cand.size() > static_cast<size_t>(RRG_BATCH_MAX_WIDTHS)) cand.resize(RRG_BATCH_MAX_WIDTHS);
  cudaEvent_t a = nullptr, b = nullptr;
  BCK(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return bset_err(h, RRG_ECUDA, "event"); }
  const int keep = h->B.c.width;
  double best = 0.0;
  int best_w = keep, rc = RRG_OK;
  for (size_t q = 0; q < cand.size() && rc == RRG_OK; ++q) {
    h->B.c.width = cand[q];
    double total = 0.0;
    for (int rep = 0; rep <= repeats && rc == RRG_OK; ++rep) {
      if (cudaEventRecord(a, h->stream) != cudaSuccess) { rc = bset_err(h, RRG_ECUDA, "event record"); break; }
      rc = enqueue_update(h, d_x, d_r, d_v_prev, seed, update_index, nullptr, nullptr, nullptr);
      if (rc != RRG_OK) break;
      if (cudaEventRecord(b, h->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
        rc = bset_err(h, RRG_ECUDA, "event wait");
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0) total += ms;  // the first run warms up
    }
    const double mean = total / repeats;
    if (widths) widths[q] = cand[q];
    if (ms_out) ms_out[q] = mean;
    if (q == 0 || mean < best) {
      best = mean;
      best_w = cand[q];
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  bcollect(h);
  h->B.c.width = rc == RRG_OK ? best_w : keep;
  if (rc != RRG_OK) return rc;
  if (width_out) *width_out = best_w;
  if (n_out) *n_out = static_cast<int>(cand.size());
  return RRG_OK;
}

int rrg_batch_autotune(rrg_batch_handle h, const double* d_x, const double* d_r,
                       const double* d_v_prev, uint64_t seed, uint64_t update_index, int repeats,
                       int* variant_out, double* ms_out) {
  if (!h) return RRG_EINVAL;
  if (!d_x || !d_r || !d_v_prev || repeats < 1)
    return bset_err(h, RRG_EINVAL, "d_x, d_r, d_v_prev non-NULL and repeats >= 1");
  BDeviceGuard g(h->device);
  h->B.t_dev = nullptr;
  h->cl_next_ready = false;
  const bool prof = h->profiling;
  const double ms0 = h->rollout_ms;
  const uint64_t n0 = h->timed_rollouts;
  BCK(cudaStreamSynchronize(h->stream));
  bcollect(h);
  double best = 0.0;
  int best_v = h->variant;
  for (int v = 0; v < RRG_BATCH_VARIANTS; ++v) {
    h->variant = v;
    h->profiling = true;
    double total = 0.0;
    for (int rep = 0; rep <= repeats; ++rep) {
      const double before = h->rollout_ms;
      int rc = enqueue_update(h, d_x, d_r, d_v_prev, seed, update_index, nullptr, nullptr, nullptr);
      if (rc != RRG_OK) { h->profiling = prof; return rc; }
      BCK(cudaStreamSynchronize(h->stream));
      bcollect(h);
      if (rep > 0) total += h->rollout_ms - before;  // the first run warms up
    }
    const double ms = total / repeats;
    if (ms_out) ms_out[v] = ms;
    if (v == 0 || ms < best) {
      best = ms;
      best_v = v;
    }
  }
  h->variant = best_v;
  h->profiling = prof;
  h->rollout_ms = ms0;
  h->timed_rollouts = n0;
  if (variant_out) *variant_out = best_v;
  return RRG_OK;
}

int rrg_batch_set_profiling(rrg_batch_handle h, int on) {
  if (!h) return RRG_EINVAL;
  h->profiling = on != 0;
  return RRG_OK;
}

int rrg_batch_get_stats(rrg_batch_handle h, rrg_stats* out) {
  if (!h || !out) return RRG_EINVAL;
  BDeviceGuard g(h->device);
  BCK(cudaStreamSynchronize(h->stream));
  bcollect(h);
  DevStats d{};
  BCK(cudaMemcpy(&d, h->stats, sizeof d, cudaMemcpyDeviceToHost));
  std::memset(out, 0, sizeof *out);
  out->launches = h->launches;
  out->rollout_launches = h->rollout_launches;
  out->lane_steps = d.lane_steps;
  out->lane_steps_fp64 = d.lane_steps_fp64;
  out->rechecked = d.rechecked;
  out->rounds = h->rounds;
  out->rollout_ms = h->rollout_ms;
  out->recheck_ms = 0.0;
  out->timed_rollouts = h->timed_rollouts;
  out->repairs = 0;
  out->graph_conditional = 0;
  return RRG_OK;
}

int rrg_batch_reset_stats(rrg_batch_handle h) {
  if (!h) return RRG_EINVAL;
  BDeviceGuard g(h->device);
  BCK(cudaStreamSynchronize(h->stream));
  bcollect(h);
  BCK(cudaMemsetAsync(h->stats, 0, sizeof(DevStats), h->stream));
  BCK(cudaStreamSynchronize(h->stream));
  h->launches = h->rollout_launches = h->rounds = 0;
  h->rollout_ms = 0.0;
  h->timed_rollouts = 0;
  return RRG_OK;
}

}  // extern "C"
