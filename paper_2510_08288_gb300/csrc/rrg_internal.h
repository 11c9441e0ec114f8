// rrg_internal.h -- types shared by the kernels (rrg_kernels.cu) and the
// host side of the C ABI (rrg_capi.cu).  Not part of the public interface.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/rrg.h"

#include "rrg_device.cuh"

namespace rrg {

// FC3 parameter indices (the layout documented in rrg.h).
enum ParamIdx {
  P_P_ATM = 0, P_T_ATM, P_T_ST, P_R_A, P_V_SM, P_V_CA, P_K_SM, P_K_CA,
  P_N_CELL, P_FARADAY, P_M_O2, P_X_O2, P_GAMMA, P_C_P, P_ETA_CP, P_J_CP,
  P_ETA_CM, P_K_T, P_K_V, P_R_CM, P_A_W, P_A_P, P_LAM_REF, P_K_P,
  P_C0, P_C1, P_C2, P_COUNT
};
static_assert(P_COUNT == RRG_NPARAM, "parameter layout");

constexpr int kMaxTreeNodes = 2 * RRG_MAX_CANDIDATES;

// What the blocks of one rollout launch do with their candidate slot.
enum SegMode : int32_t {
  SEG_FULL = 0,      // steps 0..H
  SEG_PROBE = 1,     // steps 0..probe_steps; survivors save their state
  SEG_CONTINUE = 2,  // resume a probed trajectory at probe_steps, run to H;
                     // row y continues slot cont_slot[y]
};

// A launch covers up to two slot ranges: blockIdx.y < seg[0].count maps to
// slot seg[0].base + y, the next seg[1].count rows to seg[1].base + ...
struct Seg {
  int32_t mode, count, base;
};

// Saved state of a probed trajectory (status 0: still running, continue it;
// 1: finished in the probe and already reduced).
template <typename T>
struct LaneState {
  T q[3];         // deviation from the candidate's reference point
  T w_abs;        // the absolute speed carried with it
  T smin;
  int32_t status;
  int32_t jlast;  // last step with slack below the recheck band so far (-1: none)
};

// Origin of a scenario pair.  In the binary32 modes the sampler writes only
// the binary32 copy; the binary64 values (needed by the few rechecked
// trajectories) are regenerated from the same Philox counters on demand.
struct ScenSrc {
  int32_t d64_valid;     // 1: the binary64 array holds the values
  int32_t pad;
  unsigned long long seed, update;
  unsigned long long base;  // global index of scenario 0 (the Philox counter's k)
  double amp[3];
};

// Device-resident state of one RG update's search (one per handle).
struct SearchState {
  double x[3];        // x_t (absolute coordinates)
  double v_prev, r;   // v_{t-1}, r_t
  double lo, hi;      // bisection bracket / k-section bracket
  double kappa;       // next kappa Alg. 1 would test
  double kappa_opt;   // best admissible kappa so far
  int32_t iter;       // Alg. 1 iterations consumed
  int32_t any;        // some evaluated candidate was admissible
  int32_t done;       // search finished; outputs written
  int32_t flags;      // RRG flags of the result
  int32_t m;          // candidates of the current round
  int32_t depth;      // tree levels of the current round (bisection)
  int32_t round;      // rounds finished
  int32_t invalid;    // inputs rejected on the device
  double v_t_out;     // governed reference of the finished search
  int32_t buf;        // scenario pair of the current update (0: d64/d32, 1: d64b/d32b)
  ScenSrc src[2];     // where each pair's binary64 values are
  Seg seg[2];         // what the next rollout launch runs
  int32_t prep_base;  // slots the next prepare launch fills: prep_base ..
  int32_t prep_m;     //   prep_base + prep_m - 1
  // pipelined first round of the speculative bisection: the round is probed,
  // the next tree is built from the provisional outcomes, and both run
  // together; the real outcomes are compared with the provisional ones
  int32_t probe;      // 1 while a probed round awaits validation
  int32_t depth1;     // levels of the tree built from provisional outcomes
  int32_t prov_len, prov_done;
  uint32_t prov_bits;
  int32_t cont_slot[16];  // the probed round's slots on the provisional path
  double w_lo, w_hi, w_kappa, w_kopt;  // search state before the probed round
  int32_t w_iter, w_any;
  int32_t slot_of_node[kMaxTreeNodes];   // bisection tree: heap node -> slot
  int32_t slot_of_node1[kMaxTreeNodes];  // tree of the pipelined second round
};

// Device counters of a handle.
struct DevStats {
  unsigned long long lane_steps;
  unsigned long long lane_steps_fp64;
  unsigned long long rechecked;
  unsigned long long repairs;   // probed rounds whose provisional outcome was wrong
  // kernels, rollout launches and search rounds run by the conditional body
  // of a captured closed-loop update (counted by the kernel that opens it)
  unsigned long long cond_launches, cond_rollouts, cond_rounds;
  unsigned long long lane_steps_paired;  // of lane_steps, run two trajectories per thread
  unsigned long long wait_timeouts;      // bounded waits that gave up (TMA ring copies)
  unsigned long long lane_steps_tma;     // of lane_steps, fed by the TMA ring
};

// Closed-loop device state.
struct LoopState {
  double x[3];
  double v_prev;
  unsigned long long t;   // updates done since the loop started
};

// Search configuration passed by value to the search kernels.
struct SearchCfg {
  int search;        // RRG_SEARCH_*
  int m_cap;         // candidates per round
  int n_bisect;      // N_kappa
  int n_rounds;      // k-section rounds
  int ss_check;
  int probe_steps;   // > 0: pipeline the first two bisection rounds
  double y_min, eps_ss, y_c;
};

// Everything a launch needs; filled by the host side from the handle.
struct Launch {
  cudaStream_t stream;
  int N, H, precision, early_exit, m_cap;
  int scen_gen;                 // disturbances drawn inside the trajectory loop
  unsigned long long kbase;     // global index of the handle's scenario 0 (scenario sharding)
  int pair;                     // RRG_PAIR_*: two candidates per thread in binary32 rollouts
                                //   of full-horizon rows (never, launches that fill the SMs, always)
  // conditional-node handle of a captured closed-loop update (0: none); the
  // search kernel that validates the pipelined rounds sets it to "the search
  // is not finished", which runs the remaining rounds
  unsigned long long cond;
  uint32_t cond_launches, cond_rollouts, cond_rounds;  // what one run of that body launches
  double dt, y_min, eps_abs;
  SearchCfg scfg;
  const double* params;         // [RRG_NPARAM] (device)
  Fc3K<double> k64;             // folded model constants, passed by value
  Fc3K<float> k32;
  RhsU<double> u64;             // the rollout's multiplied-out constants
  RhsU<float> u32;
  double* d64;                  // scenarios [3][H][N]
  float* d32;
  double* d64b;                 // second pair for closed loops (sampling of update t+1
  float* d32b;                  //   overlaps update t), or nullptr
  SearchState* st;
  double* cand_kappa;
  double* cand_v;
  RhsC<double>* cand_c64;       // per-slot rollout constants of the candidate
  RhsC<float>* cand_c32;
  int32_t* cand_ok;    // AND of the round's trajectory decisions
  int32_t* cand_dead;  // set once the candidate is known to fail
  int32_t* cand_ss;    // steady-state check passed
  unsigned long long* cand_min;
  uint32_t* recheck_list;
  uint32_t* recheck_jlast;      // per entry: the recheck runs steps 0..jlast
  uint32_t* recheck_count;
  DevStats* stats;
  uint8_t* P;                   // optional
  int recheck_blocks;
  int sms;                      // streaming multiprocessors of the device (> 0; launches
                                //   refuse a descriptor without it)
  int probe_steps;              // steps of a SEG_PROBE segment
  void* lane_state;             // LaneState<T>[m_cap * N] for probed rounds
  // parametric uncertainty: per-scenario parameter multipliers m[k * NPARAM
  // + p] of each scenario pair (nullptr when off)
  double* pmul;
  double* pmulb;
  double punc_rho;
  uint32_t punc_mask;
  // host: the tensor maps of the two binary32 scenario arrays (the second
  // repeats the first until a second pair exists), or nullptr: the binary32
  // rings then use per-lane asynchronous copies
  const CUtensorMap* tmap;
  int tma;                      // RRG_TMA_*: which ring launches take the TMA
  int inject;                   // RRG_INJECT_* test switches (0 in normal use)
  int tma_pair_bps;             // resident blocks per SM of the paired TMA kernel (0: never paired)
};

// Folds the FC3 parameter vector into the constants the kernels use
// (binary64, then rounded once to binary32).  Only products and quotients
// occur, so no multiply-add can be fused and host and device agree bit for
// bit.  Called once per handle on the host and, under parametric
// uncertainty, once per trajectory on the device.
__host__ __device__ inline void fold_constants(const double* P, Fc3K<double>* k64,
                                               Fc3K<float>* k32) {
  Fc3K<double> K{};
  K.inv_p_atm = 1.0 / P[P_P_ATM];
  K.a_w = P[P_A_W];
  K.a_p = P[P_A_P];
  K.k_sm = P[P_K_SM];
  K.k_ca = P[P_K_CA];
  K.e = (P[P_GAMMA] - 1.0) / P[P_GAMMA];
  K.C_cp = P[P_C_P] * P[P_T_ATM] / P[P_ETA_CP];
  K.C_m = P[P_ETA_CM] * P[P_K_T] / P[P_R_CM];
  K.k_v = P[P_K_V];
  K.K_p = P[P_K_P];
  K.RT_Vca = P[P_R_A] * P[P_T_ST] / P[P_V_CA];
  K.RT_Vsm = P[P_R_A] * P[P_T_ST] / P[P_V_SM];
  K.inv_J = 1.0 / P[P_J_CP];
  K.pws = nullptr;
  *k64 = K;
  Fc3K<float> F{};
  F.inv_p_atm = static_cast<float>(K.inv_p_atm);
  F.a_w = static_cast<float>(K.a_w);
  F.a_p = static_cast<float>(K.a_p);
  F.k_sm = static_cast<float>(K.k_sm);
  F.k_ca = static_cast<float>(K.k_ca);
  F.e = static_cast<float>(K.e);
  F.C_cp = static_cast<float>(K.C_cp);
  F.C_m = static_cast<float>(K.C_m);
  F.k_v = static_cast<float>(K.k_v);
  F.K_p = static_cast<float>(K.K_p);
  F.RT_Vca = static_cast<float>(K.RT_Vca);
  F.RT_Vsm = static_cast<float>(K.RT_Vsm);
  F.inv_J = static_cast<float>(K.inv_J);
  F.pws = nullptr;
  *k32 = F;
}

// Constants of the closed loop at setpoint I (binary64; every operation
// rounded separately, so each call site computes the same bits).
__device__ __forceinline__ CandK<double> cand_consts(const double* __restrict__ P, double I) {
  CandK<double> C;
  C.W_o2 = __ddiv_rn(__dmul_rn(__dmul_rn(P[P_M_O2], P[P_N_CELL]), I), __dmul_rn(4.0, P[P_FARADAY]));
  const double W_ref = __ddiv_rn(__dmul_rn(P[P_LAM_REF], C.W_o2), P[P_X_O2]);
  const double v_ff = __dadd_rn(__dadd_rn(P[P_C0], __dmul_rn(P[P_C1], I)),
                                __dmul_rn(__dmul_rn(P[P_C2], I), I));
  C.V0 = __dadd_rn(v_ff, __dmul_rn(P[P_K_P], W_ref));
  C.y_scale = __ddiv_rn(__dmul_rn(P[P_X_O2], P[P_K_SM]), C.W_o2);
  return C;
}

__device__ __forceinline__ CandK<float> cand_round(const CandK<double>& C) {
  CandK<float> F;
  F.W_o2 = static_cast<float>(C.W_o2);
  F.V0 = static_cast<float>(C.V0);
  F.y_scale = static_cast<float>(C.y_scale);
  return F;
}

// Binary64 product and sum rounded on their own on host and device alike
// (the device compiler would otherwise fuse a product into a following add).
__host__ __device__ inline double mul_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ inline double add_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(a, b);
#else
  return a + b;
#endif
}

// The multiplied-out constants of the rollout right-hand side (products and
// sums of the folded binary64 constants, each rounded on its own, then
// rounded once to binary32), the same bits on the host and the device.
__host__ __device__ inline void fold_rhs(const Fc3K<double>& K, RhsU<double>* u64, RhsU<float>* u32) {
  RhsU<double> U;
  U.a1 = mul_rn(K.RT_Vca, K.k_sm);
  U.a12 = add_rn(U.a1, mul_rn(K.RT_Vca, K.k_ca));
  U.a_w = K.a_w;
  U.a_p = K.a_p;
  U.b3 = mul_rn(K.RT_Vsm, K.k_sm);
  U.g_w = mul_rn(K.RT_Vsm, K.a_w);
  U.g_sm = add_rn(mul_rn(K.RT_Vsm, K.a_p), U.b3);
  U.inv_p_atm = K.inv_p_atm;
  U.e = K.e;
  U.e1 = mul_rn(mul_rn(K.C_m, K.K_p), K.inv_J);
  U.e2 = mul_rn(mul_rn(K.C_m, K.k_v), K.inv_J);
  U.e3 = mul_rn(K.C_cp, K.inv_J);
  U.pws = K.pws;
  *u64 = U;
  RhsU<float> F;
  F.a1 = static_cast<float>(U.a1);
  F.a12 = static_cast<float>(U.a12);
  F.a_w = static_cast<float>(U.a_w);
  F.a_p = static_cast<float>(U.a_p);
  F.b3 = static_cast<float>(U.b3);
  F.g_w = static_cast<float>(U.g_w);
  F.g_sm = static_cast<float>(U.g_sm);
  F.inv_p_atm = static_cast<float>(U.inv_p_atm);
  F.e = static_cast<float>(U.e);
  F.e1 = static_cast<float>(U.e1);
  F.e2 = static_cast<float>(U.e2);
  F.e3 = static_cast<float>(U.e3);
  F.pws = nullptr;
  *u32 = F;
}

// Candidate constants of the rollouts about the reference point q_r (gauge
// coordinates; binary32 values, or 0 for the gauge form), with the output
// bound y_min folded into the slack offset.  Every operation is rounded on
// its own in binary64 (no fused multiply-add), so each call site computes the
// same bits; the products a1, a2, b3, e2 are those of fold_rhs.
__device__ __forceinline__ void fold_rhs_cand(const Fc3K<double>& K, const CandK<double>& C,
                                              const double q_r[3], double y_min,
                                              RhsC<double>* c64, RhsC<float>* c32) {
  const double a1 = __dmul_rn(K.RT_Vca, K.k_sm), a2 = __dmul_rn(K.RT_Vca, K.k_ca);
  const double b3 = __dmul_rn(K.RT_Vsm, K.k_sm);
  const double e2 = __dmul_rn(__dmul_rn(K.C_m, K.k_v), K.inv_J);
  const double s_r = __dsub_rn(q_r[2], q_r[0]);
  RhsC<double> R;
  R.W_r = __dsub_rn(__dmul_rn(K.a_w, q_r[1]), __dmul_rn(K.a_p, q_r[2]));
  R.c_ca = __dsub_rn(__dsub_rn(__dmul_rn(a1, s_r), __dmul_rn(a2, q_r[0])), __dmul_rn(K.RT_Vca, C.W_o2));
  R.c_sm = __dsub_rn(__dmul_rn(K.RT_Vsm, R.W_r), __dmul_rn(b3, s_r));
  R.e0 = __dsub_rn(__dmul_rn(__dmul_rn(K.C_m, C.V0), K.inv_J), __dmul_rn(e2, q_r[1]));
  R.x_r = __dadd_rn(1.0, __dmul_rn(q_r[2], K.inv_p_atm));
  R.y_scale = C.y_scale;
  R.s_off = __dsub_rn(__dmul_rn(C.y_scale, s_r), y_min);
  R.r_ca = q_r[0];
  R.r_w = q_r[1];
  R.r_sm = q_r[2];
  *c64 = R;
  c32->c_ca = static_cast<float>(R.c_ca);
  c32->c_sm = static_cast<float>(R.c_sm);
  c32->W_r = static_cast<float>(R.W_r);
  c32->e0 = static_cast<float>(R.e0);
  c32->x_r = static_cast<float>(R.x_r);
  c32->y_scale = static_cast<float>(R.y_scale);
  c32->s_off = static_cast<float>(R.s_off);
  c32->r_ca = static_cast<float>(R.r_ca);
  c32->r_w = static_cast<float>(R.r_w);
  c32->r_sm = static_cast<float>(R.r_sm);
}

// Coefficients of the binary64 x^e - 1 series (host).
inline void make_pow_series(double e, PowSeries* S) {
  const double c = 1.5, lc = std::log(c);
  const double ce = std::exp(e * lc);
  S->e = e;
  S->inv_c = 1.0 / c;
  S->a[0] = std::expm1(e * lc);
  double b = 1.0;  // binom(e, n)
  for (int n = 1; n <= 32; ++n) {
    b = b * (e - static_cast<double>(n - 1)) / static_cast<double>(n);
    S->a[n] = ce * b;
  }
}

// ---- kernel launchers (rrg_kernels.cu) --------------------------------
// dual: write the pair (base + *t_dev) & 1 (closed loops with two pairs).
// In the binary32 modes only the binary32 copy is written.
cudaError_t launch_sample(const Launch& L, uint64_t seed, uint64_t base,
                          const unsigned long long* t_dev, const double* amp, bool dual = false,
                          cudaStream_t stream = nullptr);
// Fills pair 0's binary64 array from its Philox counters if it was sampled
// lazily (no-op otherwise).
cudaError_t launch_materialize64(const Launch& L);
cudaError_t launch_round_scenarios(const Launch& L);
cudaError_t launch_fill(const Launch& L, double* a, size_t n, double v);
// buf_base >= 0: the update index is buf_base + *t_dev and selects the
// scenario pair by its parity; otherwise pair 0
cudaError_t launch_search_begin(const Launch& L, const double* d_x, const double* d_r,
                                const unsigned long long* t_dev, const double* d_v_prev,
                                long long buf_base = -1);
cudaError_t launch_search_next(const Launch& L, double* d_v_t, double* d_kappa,
                               int32_t* d_flags);
cudaError_t launch_search_mid(const Launch& L);
// Candidate set-up for the slots the last search kernel chose: one block per
// candidate (the binary64 equilibrium solves spread over the SMs).
cudaError_t launch_prepare(const Launch& L, int width);
// d_vp / d_r (optional): read v_prev and r on the device instead (a captured
// graph replayed with new inputs).
cudaError_t launch_eval_prepare(const Launch& L, const double* d_x, double v_prev, double r,
                                const double* d_kappas, int m, const double* d_vp = nullptr,
                                const double* d_r = nullptr);
cudaError_t launch_eval_finish(const Launch& L, int m, uint8_t* d_adm, double* d_min_slack);
// Tensor map of a binary32 scenario array [3][H][N] for the TMA ring (boxes
// of 32 scenarios x one chunk of steps x 3 components); false when N is not a
// multiple of 4 (row strides must be multiples of 16 bytes) or the driver
// refuses.  tma_ring_prepare() sets the TMA kernels' shared-memory limit on
// the current device (once per device); false if the runtime refuses.
bool encode_scenario_map(CUtensorMap* m, const float* d32, int N, int H);
bool tma_ring_prepare();
// Resident blocks per SM of the two-candidates-per-thread TMA kernel (after
// tma_ring_prepare on the current device; 0 if the runtime does not answer).
int tma_pair_blocks_per_sm(bool pu);
// Resident blocks per SM of the two-candidates-per-thread rollout kernel
// (queried from the runtime on the first call, then cached).
int pair_blocks_per_sm(bool pu);
// allow_pair: the round's rows are all full-horizon segments (no pipelined
// probe), so two candidates may share a thread (Launch::pair).
cudaError_t launch_rollout(const Launch& L, int m_launch, bool use_fp64, int early_exit,
                           bool recheck_classify, bool allow_pair = false);
cudaError_t launch_recheck(const Launch& L, int early_exit);
cudaError_t launch_equilibrium(const Launch& L, double v, double* d_out4, int32_t* d_status);
cudaError_t launch_step_latency(const Launch& L, double v, int steps, double* d_out2, int32_t* d_status);
cudaError_t launch_plant(const Launch& L, const double* d_x, const double* d_v, uint64_t seed,
                         uint64_t base, const unsigned long long* t_dev, const double* amp_dev,
                         double* d_x_next);
cudaError_t launch_loop_end(const Launch& L, LoopState* ls, uint64_t seed, uint64_t t0,
                            const double* amp_dev, double* d_v_out, double* d_kappa_out,
                            int32_t* d_flags_out, double* d_x_out);
cudaError_t launch_loop_init(const Launch& L, LoopState* ls, const double* x0, double v0,
                             double* d_x_out);

// Discrete adjoint of the min-slack objective (rrg_adjoint.cu), for the m
// candidate slots the last candidate set-up prepared; layouts in the file.
constexpr int kAdjOutStride = 3 + 4 + RRG_NPARAM;
// argmin = false: the argmin pass is left to the reverse sweep (lane_min /
// lane_arg given to launch_adjoint_reverse), one launch fewer.
cudaError_t launch_adjoint_forward(const Launch& L, bool fp64, int m, int checkpoint, double* ckpt,
                                   double* lane_min, int* lane_arg, double* d_out,
                                   cudaEvent_t fwd_begin, cudaEvent_t fwd_end, bool argmin = true);
// The reverse sweeps read v_prev and r from the search state the candidate
// set-up wrote.
cudaError_t launch_adjoint_reverse(const Launch& L, bool fp64, int slot0, int count, int checkpoint,
                                   const double* ckpt, void* seg, double* d_out,
                                   const double* lane_min = nullptr, const int* lane_arg = nullptr);

// Binary32-vs-binary64 slack error of every trajectory of the m candidates
// the last eval_prepare + prepare set up (rrg_error.cu): per lane o = i N + k
// the largest |s32_j - s64_j| over j = 0..H and its step, both min slacks and
// the number of steps the band rule [-band, band) would decide wrongly and
// the largest ratio of a step's error to max(band, |s64_j|).  j_err, smin32,
// smin64, unsafe, ratio may be null.
cudaError_t launch_slack_error(const Launch& L, int m, float band, double* err, int32_t* j_err,
                               double* smin32, double* smin64, int32_t* unsafe, double* ratio);

// Configuration check shared with the handle-less entry point (rrg_capi.cu);
// on failure the message is readable with rrg_last_error(NULL).
int check_config(const rrg_config* c);
void set_thread_error(const char* msg);

// Number of search rounds each strategy enqueues (host-side schedule).
int search_round_count(const SearchCfg& c);
// Candidate count of round `round` of the schedule.
int search_round_width(const SearchCfg& c, int round);
// True when the first two rounds are pipelined (probe + continue).
bool search_pipelined(const SearchCfg& c, int horizon);
// Standard rounds enqueued after a pipelined pair (enough to finish the
// search from any level a wrong provisional outcome can send it back to),
// and the candidate width they need.
int search_extra_rounds(const SearchCfg& c);
int search_extra_width(const SearchCfg& c);

}  // namespace rrg
