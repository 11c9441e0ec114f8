// rrg_capi.cu -- host side of the C ABI declared in include/rrg.h: handle
// life cycle, argument validation, device memory, and the fixed launch
// sequence of one RG update (see rrg_kernels.cu).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "rrg_device.cuh"
#include "rrg_internal.h"

using namespace rrg;

namespace {
thread_local std::string g_create_error;
}

struct rrg_ctx {
  int device = 0;
  int sms = 0;                  // streaming multiprocessors of the device (queried)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  rrg_config cfg{};
  double params[RRG_NPARAM]{};
  SearchCfg scfg{};
  int pair = RRG_PAIR_FILLED;   // trajectories per thread of the binary32 rollouts (rrg_set_pairing)
  // tensor maps of the binary32 scenario arrays (pair 0, pair 1) for the TMA
  // ring; tma_ok once both describe the arrays in use
  CUtensorMap tmap[2];
  bool tma_ok = false;
  int tma_mode = RRG_TMA_AUTO;  // rrg_set_tma
  int inject = 0;               // rrg_set_injection
  int tma_pair_bps = 0;         // occupancy of the paired TMA kernel (queried at creation)
  Launch L{};
  // device memory
  double* params_dev = nullptr;
  double* d64 = nullptr;
  float* d32 = nullptr;
  double* d64b = nullptr;       // second scenario pair, allocated by the first closed loop
  float* d32b = nullptr;
  PowSeries* pws = nullptr;     // binary64 x^e - 1 series of the model's exponent
  double* pmul = nullptr;       // parameter multipliers of each pair (parametric uncertainty)
  double* pmulb = nullptr;
  cudaStream_t side = nullptr;  // samples update t+1 while update t runs
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool cl_next_ready = false;   // the closed loop's next update is already sampled
  uint64_t cl_seed = 0, cl_t0 = 0;
  // adjoint buffers (allocated on first use)
  double* adj_ckpt = nullptr;
  size_t adj_ckpt_cap = 0;
  double* adj_lane_min = nullptr;
  int* adj_lane_arg = nullptr;
  size_t adj_lane_cap = 0;      // lanes (m N) the lane arrays and adj_out hold
  double* adj_seg = nullptr;
  size_t adj_seg_cap = 0;
  double* adj_out = nullptr;   // [0] g, [1..2] k*, j* (as long long), [3..] gradient
  double* adj_out_h = nullptr;  // pinned host copies of adj_out and the steady-state flags
  int32_t* adj_ss_h = nullptr;
  // binary32-vs-binary64 slack error per lane (allocated on first use)
  void* err_buf = nullptr;
  size_t err_cap = 0;
  // the captured one-update graph of the last closed loop, reused while the
  // run's pointers and indices stay the same
  cudaGraphExec_t cl_exec = nullptr;
  const void* cl_key[6] = {};
  uint64_t cl_key_seed = 0, cl_key_t0 = 0;
  uint64_t cl_per = 0, cl_rl_per = 0, cl_rd_per = 0;
  bool cl_conditional = false;  // the cached graph uses a conditional node
  // the captured search of rrg_step (fixed io_dev / flag_dev pointers),
  // discarded whenever the launch descriptor changes (fill_launch)
  cudaGraphExec_t st_exec = nullptr;
  uint64_t st_per = 0, st_rl_per = 0, st_rd_per = 0;
  bool st_refused = false;      // the graph API refused: rrg_step launches directly
  // the captured gradient call (rrg_slack_gradients), keyed by its shape and
  // the adjoint buffers
  cudaGraphExec_t ad_exec = nullptr;
  int ad_m = 0, ad_ck = 0, ad_prec = -1;
  const void* ad_key[5] = {};
  uint64_t ad_per = 0, ad_rl_per = 0;
  bool ad_refused = false;
  SearchState* st = nullptr;
  double* cand_kappa = nullptr;
  double* cand_v = nullptr;
  RhsC<double>* cand_c64 = nullptr;
  RhsC<float>* cand_c32 = nullptr;
  int32_t* cand_ok = nullptr;
  int32_t* cand_dead = nullptr;
  int32_t* cand_ss = nullptr;
  unsigned long long* cand_min = nullptr;
  uint32_t* recheck_list = nullptr;
  uint32_t* recheck_jlast = nullptr;
  uint32_t* recheck_count = nullptr;
  DevStats* stats = nullptr;
  void* lane_state = nullptr;
  uint8_t* P_dev = nullptr;
  double* io_dev = nullptr;     // [0..2] x, [3] r, [4] v, [5..8] out, [8] amp.. see offsets
  int32_t* flag_dev = nullptr;  // [0] flags, [1] status
  double* kap_dev = nullptr;    // [m_cap] kappas in, [m_cap] min slack out
  uint8_t* adm_dev = nullptr;
  LoopState* loop = nullptr;
  // closed-loop I/O staging (grown on demand)
  double* cl_dev = nullptr;
  size_t cl_cap = 0;
  // pinned host staging
  double* io_h = nullptr;
  int32_t* flag_h = nullptr;
  // counters and profiling
  uint64_t launches = 0, rollout_launches = 0, rounds = 0;
  bool profiling = false;
  bool capturing = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_roll, ev_rec;
  double rollout_ms = 0.0, recheck_ms = 0.0;
  uint64_t timed_rollouts = 0;
  std::string err;
};

namespace {

// io_dev / io_h offsets (doubles)
constexpr int IO_X = 0, IO_R = 3, IO_V = 4, IO_OUT = 5, IO_AMP = 9, IO_LEN = 12;

int set_err(rrg_ctx* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf; else g_create_error = buf;
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return set_err(h, RRG_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

bool is_fin(double x) { return std::isfinite(x); }

int validate_cfg(const rrg_config* c) {
  if (!c) return set_err(nullptr, RRG_EINVAL, "cfg is NULL");
  if (!(c->dt > 0.0) || !is_fin(c->dt)) return set_err(nullptr, RRG_EINVAL, "dt must be > 0");
  if (c->horizon < 1) return set_err(nullptr, RRG_EINVAL, "horizon must be >= 1");
  if (c->n_scenarios < 1) return set_err(nullptr, RRG_EINVAL, "n_scenarios must be >= 1");
  if (c->max_candidates < 1 || c->max_candidates > RRG_MAX_CANDIDATES)
    return set_err(nullptr, RRG_EINVAL, "max_candidates must be in [1, %d]", RRG_MAX_CANDIDATES);
  if (c->n_bisect < 1 || c->n_bisect > 60)
    return set_err(nullptr, RRG_EINVAL, "n_bisect must be in [1, 60]");
  if (c->n_rounds < 1 || c->n_rounds > 64)
    return set_err(nullptr, RRG_EINVAL, "n_rounds must be in [1, 64]");
  if (c->search < RRG_SEARCH_BISECT || c->search > RRG_SEARCH_SPEC_BISECT)
    return set_err(nullptr, RRG_EINVAL, "unknown search %d", c->search);
  if ((c->search == RRG_SEARCH_GRID || c->search == RRG_SEARCH_KSECTION) && c->max_candidates < 2)
    return set_err(nullptr, RRG_EINVAL, "grid searches need max_candidates >= 2");
  if (c->precision < RRG_FP64 || c->precision > RRG_FP32_RECHECK)
    return set_err(nullptr, RRG_EINVAL, "unknown precision %d", c->precision);
  if (c->early_exit < RRG_EXIT_NONE || c->early_exit > RRG_EXIT_CANDIDATE)
    return set_err(nullptr, RRG_EINVAL, "unknown early_exit %d", c->early_exit);
  if (!is_fin(c->y_min) || !is_fin(c->y_c) || !is_fin(c->eps_ss) || c->eps_ss < 0.0 ||
      c->eps_ss >= 1.0)
    return set_err(nullptr, RRG_EINVAL, "y_min, y_c must be finite and eps_ss in [0, 1)");
  if (!is_fin(c->recheck_eps_rel) || c->recheck_eps_rel < 0.0)
    return set_err(nullptr, RRG_EINVAL, "recheck_eps_rel must be >= 0");
  for (int i = 0; i < 3; ++i)
    if (!is_fin(c->dist_amp[i]) || c->dist_amp[i] < 0.0)
      return set_err(nullptr, RRG_EINVAL, "dist_amp must be finite and >= 0");
  if (c->probe_steps < 0) return set_err(nullptr, RRG_EINVAL, "probe_steps must be >= 0");
  if (!is_fin(c->param_unc_rel) || c->param_unc_rel < 0.0 || c->param_unc_rel >= 1.0)
    return set_err(nullptr, RRG_EINVAL, "param_unc_rel must be in [0, 1)");
  if (c->scenarios_in_register != 0 && c->scenarios_in_register != 1)
    return set_err(nullptr, RRG_EINVAL, "scenarios_in_register must be 0 or 1");
  if (c->scenario_base < 0 || c->scenario_base > (int64_t(1) << 62))
    return set_err(nullptr, RRG_EINVAL, "scenario_base must be in [0, 2^62]");
  if (c->param_unc_mask >> RRG_NPARAM)
    return set_err(nullptr, RRG_EINVAL, "param_unc_mask has bits at or above RRG_NPARAM");
  const unsigned long long lanes =
      2ull * static_cast<unsigned long long>(c->max_candidates) * static_cast<unsigned long long>(c->n_scenarios);
  if (lanes >= (1ull << 32)) return set_err(nullptr, RRG_EINVAL, "2 * max_candidates * n_scenarios >= 2^32");
  return RRG_OK;
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T) + 16);
}

void free_all(rrg_ctx* h) {
  void* ptrs[] = {h->params_dev, h->d64, h->d32, h->d64b, h->d32b, h->st, h->cand_kappa,
                  h->cand_v, h->cand_c64, h->cand_c32, h->cand_ok, h->cand_dead, h->cand_ss,
                  h->cand_min, h->recheck_list, h->recheck_jlast, h->recheck_count, h->stats, h->P_dev, h->io_dev,
                  h->flag_dev, h->kap_dev, h->adm_dev, h->loop, h->cl_dev, h->lane_state,
                  h->adj_ckpt, h->adj_lane_min, h->adj_lane_arg, h->adj_seg, h->adj_out,
                  h->pmul, h->pmulb, h->pws, h->err_buf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->io_h) cudaFreeHost(h->io_h);
  if (h->flag_h) cudaFreeHost(h->flag_h);
  for (auto& e : h->ev_free) cudaEventDestroy(e);
  for (auto& pr : h->ev_roll) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  for (auto& pr : h->ev_rec) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  if (h->cl_exec) cudaGraphExecDestroy(h->cl_exec);
  if (h->st_exec) cudaGraphExecDestroy(h->st_exec);
  if (h->ad_exec) cudaGraphExecDestroy(h->ad_exec);
  if (h->adj_out_h) cudaFreeHost(h->adj_out_h);
  if (h->adj_ss_h) cudaFreeHost(h->adj_ss_h);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

void fill_launch(rrg_ctx* h) {
  if (h->st_exec) {  // the captured step graph holds the old descriptor
    cudaGraphExecDestroy(h->st_exec);
    h->st_exec = nullptr;
  }
  h->st_refused = false;  // a new descriptor may capture where the old one did not
  if (h->ad_exec) {
    cudaGraphExecDestroy(h->ad_exec);
    h->ad_exec = nullptr;
  }
  h->ad_refused = false;
  Launch& L = h->L;
  const rrg_config& c = h->cfg;
  L.stream = h->stream;
  L.pair = h->pair;
  L.tmap = h->tma_ok && h->tma_mode != RRG_TMA_NEVER ? h->tmap : nullptr;
  L.tma = h->tma_mode;
  L.inject = h->inject;
  L.tma_pair_bps = h->tma_pair_bps;
  L.N = c.n_scenarios;
  L.H = c.horizon;
  L.precision = c.precision;
  L.early_exit = c.early_exit;
  L.m_cap = c.max_candidates;
  L.dt = c.dt;
  L.y_min = c.y_min;
  L.eps_abs = c.precision == RRG_FP32_RECHECK ? c.recheck_eps_rel * std::fabs(c.y_min) : 0.0;
  L.scen_gen = c.scenarios_in_register;
  L.kbase = static_cast<unsigned long long>(c.scenario_base);
  L.scfg = h->scfg;
  L.params = h->params_dev;
  fold_constants(h->params, &L.k64, &L.k32);
  L.k64.pws = h->pws;
  fold_rhs(L.k64, &L.u64, &L.u32);
  L.d64 = h->d64;
  L.d32 = h->d32;
  L.st = h->st;
  L.cand_kappa = h->cand_kappa;
  L.cand_v = h->cand_v;
  L.cand_c64 = h->cand_c64;
  L.cand_c32 = h->cand_c32;
  L.cand_ok = h->cand_ok;
  L.cand_dead = h->cand_dead;
  L.cand_ss = h->cand_ss;
  L.cand_min = h->cand_min;
  L.recheck_list = h->recheck_list;
  L.recheck_jlast = h->recheck_jlast;
  L.recheck_count = h->recheck_count;
  L.stats = h->stats;
  L.P = nullptr;
  L.sms = h->sms;
  L.recheck_blocks = 2 * h->sms;
  L.probe_steps = h->scfg.probe_steps;
  L.lane_state = h->lane_state;
  L.pmul = h->pmul;
  L.pmulb = h->pmulb;
  L.punc_rho = c.param_unc_rel;
  L.punc_mask = c.param_unc_mask;
}

cudaEvent_t take_event(rrg_ctx* h) {
  if (!h->ev_free.empty()) {
    cudaEvent_t e = h->ev_free.back();
    h->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Rollout of the current round (+ recheck in FP32_RECHECK mode unless the
// launch is a probe, whose lanes are not decided yet).
// allow_pair = false for the two launches of a pipelined pair (probe and
// continuation segments), whose rows cannot share a thread.
int enqueue_round_work(rrg_ctx* h, const Launch& L, int width, int early_exit, bool recheck = true,
                       bool allow_pair = true) {
  const bool timed = h->profiling && !h->capturing;
  cudaEvent_t a = nullptr, b = nullptr;
  if (timed) { a = take_event(h); b = take_event(h); }
  if (a && b) CK(cudaEventRecord(a, h->stream));
  const bool fp64 = h->cfg.precision == RRG_FP64;
  CK(launch_rollout(L, width, fp64, early_exit, h->cfg.precision == RRG_FP32_RECHECK, allow_pair));
  if (a && b) {
    CK(cudaEventRecord(b, h->stream));
    h->ev_roll.emplace_back(a, b);
  }
  h->launches++;
  h->rollout_launches++;
  if (recheck && h->cfg.precision == RRG_FP32_RECHECK) {
    cudaEvent_t c = nullptr, d = nullptr;
    if (timed) { c = take_event(h); d = take_event(h); }
    if (c && d) CK(cudaEventRecord(c, h->stream));
    CK(launch_recheck(L, early_exit));
    if (c && d) {
      CK(cudaEventRecord(d, h->stream));
      h->ev_rec.emplace_back(c, d);
    }
    h->launches++;
  }
  return RRG_OK;
}

// The search of one RG update on already-sampled scenarios.  Each search
// kernel decides on the device, sets up the next round's candidates (kappas,
// constants, steady-state check) and the slots the following rollout runs;
// the host only enqueues the fixed sequence.
// The standard rounds that follow a pipelined pair (they finish the search,
// after a wrong provisional outcome or when more levels remain; no-ops
// otherwise).
int enqueue_extra_rounds(rrg_ctx* h, double* d_vt, double* d_kappa, int32_t* d_flags) {
  const Launch& L = h->L;
  const SearchCfg& c = h->scfg;
  const int extra = search_extra_rounds(c), wx = search_extra_width(c);
  for (int r = 0; r < extra; ++r) {
    int rc = enqueue_round_work(h, L, wx, h->cfg.early_exit);
    if (rc != RRG_OK) return rc;
    CK(launch_search_next(L, d_vt, d_kappa, d_flags));
    h->launches++;
    h->rounds++;
  }
  return RRG_OK;
}

// with_extra = false: a pipelined search stops after the validating search
// kernel (the caller enqueues enqueue_extra_rounds, e.g. in a conditional
// graph node).
int enqueue_search(rrg_ctx* h, const double* d_x, const double* d_r,
                   const unsigned long long* t_dev, const double* d_vp, double* d_vt,
                   double* d_kappa, int32_t* d_flags, long long buf_base = -1,
                   bool with_extra = true) {
  const Launch& L = h->L;
  const SearchCfg& c = h->scfg;
  const int R = search_round_count(c);
  // every search kernel also prepares the candidates of the round it sets up
  CK(launch_search_begin(L, d_x, d_r, t_dev, d_vp, buf_base));
  h->launches++;
  int r0 = 0;
  const bool pipe = search_pipelined(c, h->cfg.horizon);
  if (pipe) {
    // probe of round 1, then round 1's remainder together with round 2; the
    // rounds after it only do work when the validation found a wrong guess
    const int w0 = search_round_width(c, 0), w1 = search_round_width(c, 1);
    int rc = enqueue_round_work(h, L, w0, h->cfg.early_exit, false, false);
    if (rc != RRG_OK) return rc;
    CK(launch_search_mid(L));
    h->launches++;
    // rows: the <= 11 path nodes of round 1 that continue, then round 2
    rc = enqueue_round_work(h, L, (w0 < 11 ? w0 : 11) + w1, h->cfg.early_exit, true, false);
    if (rc != RRG_OK) return rc;
    CK(launch_search_next(L, d_vt, d_kappa, d_flags));
    h->launches++;
    h->rounds++;
    // after a wrong provisional outcome the search resumes from the level
    // where it went wrong; these rounds do nothing when it went right
    return with_extra ? enqueue_extra_rounds(h, d_vt, d_kappa, d_flags) : RRG_OK;
  }
  for (int r = r0; r < R; ++r) {
    const int width = search_round_width(c, r);
    int rc = enqueue_round_work(h, L, width, h->cfg.early_exit);
    if (rc != RRG_OK) return rc;
    CK(launch_search_next(L, d_vt, d_kappa, d_flags));
    h->launches++;
    h->rounds++;
  }
  return RRG_OK;
}

bool x_ok(const double* x) { return x && is_fin(x[0]) && is_fin(x[1]) && is_fin(x[2]); }

// Launches, rollout launches and rounds of the rounds after a pipelined
// pair: per round rollout (+ recheck), next.
void extra_round_counts(const rrg_ctx* h, uint32_t* launches, uint32_t* rollouts, uint32_t* rounds) {
  const uint32_t extra = static_cast<uint32_t>(search_extra_rounds(h->scfg));
  const uint32_t rec = h->cfg.precision == RRG_FP32_RECHECK ? 1u : 0u;
  *launches = extra * (2u + rec);
  *rollouts = extra;
  *rounds = extra;
}

// One closed-loop update as a graph with a conditional node around the rounds
// that follow the pipelined pair; nullptr if any graph call fails (the stream
// is left outside any capture).
cudaGraph_t capture_conditional_update(rrg_ctx* h, uint64_t seed, uint64_t t0, const double* amp,
                                       const double* d_r_seq, double* d_v_out, double* d_kappa_out,
                                       int32_t* d_flags_out, double* d_x_out) {
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaGraph_t G = nullptr;
  if (cudaGraphCreate(&G, 0) != cudaSuccess) return nullptr;
  bool ok = true;
  auto end_capture = [&]() {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(h->stream, &g);
    }
    cudaGetLastError();
  };
  cudaGraphConditionalHandle hc = 0;
  ok = cudaGraphConditionalHandleCreate(&hc, G, 1u, cudaGraphCondAssignDefault) == cudaSuccess;
  std::vector<cudaGraphNode_t> sinks;
  // part 1: draw of update t + 1 (side stream), the search up to the kernel
  // that validates the pipelined pair, the join
  if (ok) ok = cudaStreamBeginCaptureToGraph(h->stream, G, nullptr, nullptr, 0, mode) == cudaSuccess;
  if (ok) {
    const Launch& L = h->L;
    h->capturing = true;
    h->L.cond = hc;
    extra_round_counts(h, &h->L.cond_launches, &h->L.cond_rollouts, &h->L.cond_rounds);
    ok = cudaEventRecord(h->ev_fork, h->stream) == cudaSuccess &&
         cudaStreamWaitEvent(h->side, h->ev_fork, 0) == cudaSuccess &&
         launch_sample(L, seed, t0 + 1, &h->loop->t, h->cfg.dist_amp, true, h->side) == cudaSuccess &&
         cudaEventRecord(h->ev_join, h->side) == cudaSuccess;
    if (ok)
      ok = enqueue_search(h, h->loop->x, d_r_seq, &h->loop->t, &h->loop->v_prev, nullptr, nullptr,
                          nullptr, static_cast<long long>(t0), false) == RRG_OK;
    h->L.cond = 0ull;
    if (ok) ok = cudaStreamWaitEvent(h->stream, h->ev_join, 0) == cudaSuccess;
    if (ok) {
      cudaStreamCaptureStatus st;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      ok = cudaStreamGetCaptureInfo(h->stream, &st, nullptr, nullptr, &deps, nullptr, &nd) == cudaSuccess &&
           nd > 0;
      if (ok) sinks.assign(deps, deps + nd);
    }
    cudaGraph_t g1 = nullptr;
    ok = (cudaStreamEndCapture(h->stream, &g1) == cudaSuccess) && ok;
  }
  // part 2: the conditional node and its body (the remaining rounds)
  cudaGraphNode_t cn = nullptr;
  if (ok) {
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    ok = cudaGraphAddNode(&cn, G, sinks.data(), nullptr, sinks.size(), &cp) == cudaSuccess;
    cudaGraph_t body = ok ? cp.conditional.phGraph_out[0] : nullptr;
    if (ok) ok = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, mode) == cudaSuccess;
    if (ok) {
      ok = enqueue_extra_rounds(h, nullptr, nullptr, nullptr) == RRG_OK;
      ok = (cudaStreamEndCapture(h->stream, &body) == cudaSuccess) && ok;
    }
  }
  // part 3: plant step and loop bookkeeping, after the conditional node
  if (ok) ok = cudaStreamBeginCaptureToGraph(h->stream, G, &cn, nullptr, 1, mode) == cudaSuccess;
  if (ok) {
    ok = launch_loop_end(h->L, h->loop, seed, t0, amp, d_v_out, d_kappa_out, d_flags_out, d_x_out) ==
         cudaSuccess;
    cudaGraph_t g3 = nullptr;
    ok = (cudaStreamEndCapture(h->stream, &g3) == cudaSuccess) && ok;
  }
  h->capturing = false;
  if (!ok) {
    end_capture();
    cudaGraphDestroy(G);
    return nullptr;
  }
  return G;
}

// Host counters of the unconditional part of one captured update (sample;
// begin; probe rollout; mid; rollout (+ recheck); next; loop end), without
// enqueueing anything.  Runs of the conditional body are counted on the
// device by the kernel that opens it.
void enqueue_count_only(rrg_ctx* h) {
  const uint64_t rec = h->cfg.precision == RRG_FP32_RECHECK ? 1 : 0;
  h->launches += 1 + 1 + 1 + 1 + (1 + rec) + 1 + 1;
  h->rollout_launches += 2;
  h->rounds += 1;
}

}  // namespace

namespace {

// Grows a device buffer to n elements (contents not kept).
template <typename T>
cudaError_t grow(T** p, size_t* cap, size_t n) {
  if (n <= *cap) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
  if (e == cudaSuccess) *cap = n;
  return e;
}

}  // namespace

namespace {

// Scratch of the adjoint for m kappas (grown on demand; a buffer queued work
// may still use is freed only after the stream drained).
int adj_buffers(rrg_ctx* h, size_t M, int checkpoint) {
  const size_t N = h->cfg.n_scenarios, H = h->cfg.horizon;
  const size_t ckpt_need = M * N * (H / checkpoint + 1) * 3;
  const size_t seg_need = M * (H + 1) * 12;  // every step's state and stage points, per kappa
  if (ckpt_need > h->adj_ckpt_cap || seg_need > h->adj_seg_cap || M * N > h->adj_lane_cap)
    CK(cudaStreamSynchronize(h->stream));
  CK(grow(&h->adj_ckpt, &h->adj_ckpt_cap, ckpt_need));
  CK(grow(&h->adj_seg, &h->adj_seg_cap, seg_need));
  if (M * N > h->adj_lane_cap) {
    size_t c1 = 0, c2 = 0, c3 = 0;
    if (h->adj_lane_min) { cudaFree(h->adj_lane_min); h->adj_lane_min = nullptr; }
    if (h->adj_lane_arg) { cudaFree(h->adj_lane_arg); h->adj_lane_arg = nullptr; }
    if (h->adj_out) { cudaFree(h->adj_out); h->adj_out = nullptr; }
    h->adj_lane_cap = 0;
    CK(grow(&h->adj_lane_min, &c1, M * N));
    CK(grow(&h->adj_lane_arg, &c2, M * N));
    CK(grow(&h->adj_out, &c3, static_cast<size_t>(h->cfg.max_candidates) * kAdjOutStride));
    h->adj_lane_cap = M * N;
  }
  // pinned staging of the results: a pageable destination would make each
  // read a staged copy
  if (!h->adj_out_h)
    CK(cudaMallocHost(reinterpret_cast<void**>(&h->adj_out_h),
                      static_cast<size_t>(h->cfg.max_candidates) * kAdjOutStride * sizeof(double)));
  if (!h->adj_ss_h)
    CK(cudaMallocHost(reinterpret_cast<void**>(&h->adj_ss_h),
                      static_cast<size_t>(h->cfg.max_candidates) * sizeof(int32_t)));
  return RRG_OK;
}

// The inputs of an adjoint call into io_dev (x_t, r_t, v_prev) and kap_dev
// (the m kappas), from the pinned staging.
int adj_upload(rrg_ctx* h, const double* x_t, double v_prev, double r_t, const double* kappas, int m) {
  double* kap_h = h->io_h + IO_LEN;
  std::memcpy(h->io_h + IO_X, x_t, 3 * sizeof(double));
  h->io_h[IO_R] = r_t;
  h->io_h[IO_V] = v_prev;
  std::memcpy(kap_h, kappas, static_cast<size_t>(m) * sizeof(double));
  CK(cudaMemcpyAsync(h->io_dev, h->io_h, IO_LEN * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->kap_dev, kap_h, m * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  return RRG_OK;
}

// Enqueues the candidate set-up of the m uploaded kappas (v_prev and r read
// on the device), the binary64 scenario fill if the gradient reads it, the
// forward pass and the argmin (no sync; buffers sized by adj_buffers).
int adj_enqueue_forward_kernels(rrg_ctx* h, int m, int checkpoint, int precision, bool argmin) {
  const Launch& L = h->L;
  // candidate set-up (kappas, setpoints, rollout constants, steady-state check)
  CK(launch_eval_prepare(L, h->io_dev + IO_X, 0.0, 0.0, h->kap_dev, m, h->io_dev + IO_V, h->io_dev + IO_R));
  CK(launch_prepare(L, m));
  h->launches += 2;
  const bool use32 = precision == RRG_FP32 && h->cfg.precision != RRG_FP64 && !h->cfg.scenarios_in_register;
  if (!use32) {
    CK(launch_materialize64(L));
    h->launches += 2;
  }
  // the forward pass rolls out every scenario: timed as a rollout launch
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (h->profiling && !h->capturing) { ea = take_event(h); eb = take_event(h); }
  if (!(ea && eb)) {
    if (ea) h->ev_free.push_back(ea);
    if (eb) h->ev_free.push_back(eb);
    ea = eb = nullptr;
  }
  CK(launch_adjoint_forward(L, precision == RRG_FP64, m, checkpoint, h->adj_ckpt, h->adj_lane_min,
                            h->adj_lane_arg, h->adj_out, ea, eb, argmin));
  if (ea) h->ev_roll.emplace_back(ea, eb);
  h->launches += argmin ? 2 : 1;
  h->rollout_launches += 1;
  return RRG_OK;
}

int adj_enqueue_forward(rrg_ctx* h, const double* x_t, double v_prev, double r_t, const double* kappas,
                        int m, int checkpoint, int precision, bool argmin = true) {
  int rc = adj_buffers(h, static_cast<size_t>(m), checkpoint);
  if (rc == RRG_OK) rc = adj_upload(h, x_t, v_prev, r_t, kappas, m);
  if (rc == RRG_OK) rc = adj_enqueue_forward_kernels(h, m, checkpoint, precision, argmin);
  return rc;
}

// with_argmin: the reverse sweep finds each slot's argmin itself (after a
// forward pass enqueued without its argmin pass).
int adj_enqueue_reverse(rrg_ctx* h, int slot0, int count, int checkpoint, int precision,
                        bool with_argmin = false) {
  CK(launch_adjoint_reverse(h->L, precision == RRG_FP64, slot0, count, checkpoint, h->adj_ckpt, h->adj_seg,
                            h->adj_out, with_argmin ? h->adj_lane_min : nullptr,
                            with_argmin ? h->adj_lane_arg : nullptr));
  h->launches += 1;
  return RRG_OK;
}

// The kernels of one gradient call (set-up, forward pass, reverse sweeps with
// their argmin) captured as a graph on the handle's fixed buffers; sets the
// host counters one replay adds.  nullptr if the capture fails.
cudaGraphExec_t capture_gradient(rrg_ctx* h, int m, int checkpoint, int precision) {
  const uint64_t l0 = h->launches, r0 = h->rollout_launches;
  if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  h->capturing = true;
  int rc = adj_enqueue_forward_kernels(h, m, checkpoint, precision, false);
  if (rc == RRG_OK) rc = adj_enqueue_reverse(h, 0, m, checkpoint, precision, true);
  h->capturing = false;
  h->ad_per = h->launches - l0;
  h->ad_rl_per = h->rollout_launches - r0;
  h->launches = l0;
  h->rollout_launches = r0;
  cudaGraph_t G = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(h->stream, &G);
  if (rc != RRG_OK || ce != cudaSuccess) {
    if (G) cudaGraphDestroy(G);
    cudaGetLastError();
    return nullptr;
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ci = cudaGraphInstantiate(&ex, G, 0);
  cudaGraphDestroy(G);
  if (ci != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return ex;
}

// Reads slots 0..m-1 of the adjoint's output (and the steady-state flags)
// after the stream drained.
int adj_read(rrg_ctx* h, int m, std::vector<double>* out, std::vector<int32_t>* ss) {
  const size_t n = static_cast<size_t>(m) * kAdjOutStride;
  CK(cudaMemcpyAsync(h->adj_out_h, h->adj_out, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (ss) CK(cudaMemcpyAsync(h->adj_ss_h, h->cand_ss, m * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  out->assign(h->adj_out_h, h->adj_out_h + n);
  if (ss) ss->assign(h->adj_ss_h, h->adj_ss_h + m);
  return RRG_OK;
}

}  // namespace

extern "C" {

void rrg_config_default(rrg_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof *c);
  c->dt = 0.01;
  c->horizon = 500;
  c->n_scenarios = 32;
  c->max_candidates = 32;
  c->n_bisect = 12;
  c->n_rounds = 3;
  c->search = RRG_SEARCH_SPEC_BISECT;
  c->precision = RRG_FP32_RECHECK;
  c->early_exit = RRG_EXIT_CANDIDATE;
  c->ss_check = 1;
  c->y_min = 1.9;
  c->eps_ss = 0.05;
  c->y_c = 2.2;
  c->recheck_eps_rel = 1e-6;
  c->dist_amp[0] = 50.0;
  c->dist_amp[1] = 10.0;
  c->dist_amp[2] = 50.0;
  c->probe_steps = 128;
  c->param_unc_rel = 0.0;
  c->param_unc_mask = RRG_PARAM_UNC_MASK_FC3;
  c->scenarios_in_register = 0;
  c->scenario_base = 0;
}

const char* rrg_last_error(rrg_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int rrg_create(const double* model_params, int n_params, const rrg_config* cfg, void* cuda_stream,
               rrg_handle* out) {
  g_create_error.clear();
  if (!out) return set_err(nullptr, RRG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!model_params || n_params != RRG_NPARAM)
    return set_err(nullptr, RRG_EINVAL, "model_params must hold %d values", RRG_NPARAM);
  for (int i = 0; i < RRG_NPARAM; ++i)
    if (!is_fin(model_params[i])) return set_err(nullptr, RRG_EINVAL, "model_params[%d] not finite", i);
  int rc = validate_cfg(cfg);
  if (rc != RRG_OK) return rc;

  rrg_ctx* h = new (std::nothrow) rrg_ctx();
  if (!h) return set_err(nullptr, RRG_ENOMEM, "host allocation failed");
  h->cfg = *cfg;
  std::memcpy(h->params, model_params, sizeof h->params);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      h->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
      h->own_stream = e == cudaSuccess;
    }
  }
  const rrg_config& c = h->cfg;
  const size_t N = c.n_scenarios, H = c.horizon, M = c.max_candidates;
  const size_t HN3 = 3 * H * N;
#define ALLOC(ptr, n)                                                   \
  if (e == cudaSuccess) {                                               \
    e = dalloc(&h->ptr, (n));                                           \
    if (e != cudaSuccess) { cudaGetLastError(); }                       \
  }
  ALLOC(params_dev, RRG_NPARAM);
  ALLOC(pws, 1);
  ALLOC(d64, HN3);
  // in-register scenarios need no binary32 array (the binary64 one stays for
  // rrg_get_scenarios and the adjoint)
  const size_t n32 = c.scenarios_in_register ? 1 : HN3;
  ALLOC(d32, n32);
  ALLOC(st, 1);
  // two slot ranges: a pipelined round and the round after it run together
  ALLOC(cand_kappa, 2 * M);
  ALLOC(cand_v, 2 * M);
  ALLOC(cand_c64, 2 * M);
  ALLOC(cand_c32, 2 * M);
  ALLOC(cand_ok, 2 * M);
  ALLOC(cand_dead, 2 * M);
  ALLOC(cand_ss, 2 * M);
  ALLOC(cand_min, 2 * M);
  ALLOC(recheck_list, 2 * M * N);
  ALLOC(recheck_jlast, 2 * M * N);
  if (e == cudaSuccess && c.search == RRG_SEARCH_SPEC_BISECT && c.probe_steps > 0) {
    e = cudaMalloc(&h->lane_state, M * N * sizeof(LaneState<double>));
    if (e != cudaSuccess) cudaGetLastError();
  }
  ALLOC(recheck_count, 1);
  ALLOC(stats, 1);
  ALLOC(io_dev, IO_LEN);
  ALLOC(flag_dev, 4);
  ALLOC(kap_dev, 2 * M);
  ALLOC(adm_dev, M);
  ALLOC(loop, 1);
  if (c.param_unc_rel > 0.0) ALLOC(pmul, N * RRG_NPARAM);
#undef ALLOC
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->io_h), IO_LEN * sizeof(double) + 2 * M * sizeof(double) + M);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->flag_h), 4 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->stats, 0, sizeof(DevStats), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->st, 0, sizeof(SearchState), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d64, 0, HN3 * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d32, 0, n32 * sizeof(float), h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->params_dev, h->params, sizeof h->params, cudaMemcpyHostToDevice, h->stream);
  PowSeries ps;
  make_pow_series((h->params[P_GAMMA] - 1.0) / h->params[P_GAMMA], &ps);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->pws, &ps, sizeof ps, cudaMemcpyHostToDevice, h->stream);
  fill_launch(h);
  // the zero scenarios are explicit values (marks pair 0's binary64 array valid)
  if (e == cudaSuccess) e = launch_round_scenarios(h->L);
  if (e == cudaSuccess && h->pmul) e = launch_fill(h->L, h->pmul, N * RRG_NPARAM, 1.0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? RRG_ENOMEM : RRG_ECUDA;
    set_err(nullptr, code, "rrg_create: %s", cudaGetErrorString(e));
    free_all(h);
    delete h;
    return code;
  }
  SearchCfg& s = h->scfg;
  s.search = c.search;
  s.m_cap = c.search == RRG_SEARCH_BISECT ? 1 : c.max_candidates;
  s.n_bisect = c.n_bisect;
  s.n_rounds = c.n_rounds;
  s.ss_check = c.ss_check;
  s.probe_steps = c.search == RRG_SEARCH_SPEC_BISECT ? c.probe_steps : 0;
  s.y_min = c.y_min;
  s.eps_ss = c.eps_ss;
  s.y_c = c.y_c;
  // occupancy of the paired kernel and the TMA kernels' shared-memory limit,
  // set once here (never inside a capture)
  (void)pair_blocks_per_sm(false);
  (void)pair_blocks_per_sm(true);
  if (!c.scenarios_in_register && tma_ring_prepare() &&
      encode_scenario_map(&h->tmap[0], h->d32, c.n_scenarios, c.horizon)) {
    h->tmap[1] = h->tmap[0];
    h->tma_ok = true;
    h->tma_pair_bps = tma_pair_blocks_per_sm(c.param_unc_rel > 0.0);
  }
  fill_launch(h);
  *out = h;
  return RRG_OK;
}

int rrg_destroy(rrg_handle h) {
  if (!h) return RRG_OK;
  int rc = RRG_OK;
  {
    DeviceGuard g(h->device);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = RRG_ECUDA;
    free_all(h);
  }
  delete h;
  return rc;
}

int rrg_sample_scenarios(rrg_handle h, uint64_t seed, uint64_t update_index) {
  if (!h) return RRG_EINVAL;
  DeviceGuard g(h->device);
  h->cl_next_ready = false;  // pair 0 may hold a closed loop's next update
  CK(launch_sample(h->L, seed, update_index, nullptr, h->cfg.dist_amp));
  h->launches++;
  return RRG_OK;
}

int rrg_set_scenarios(rrg_handle h, const double* d) {
  if (!h) return RRG_EINVAL;
  if (!d) return set_err(h, RRG_EINVAL, "d is NULL");
  if (h->cfg.scenarios_in_register)
    return set_err(h, RRG_EINVAL, "the handle draws its scenarios in-register (scenarios_in_register = 1)");
  DeviceGuard g(h->device);
  h->cl_next_ready = false;
  const size_t n = 3 * static_cast<size_t>(h->cfg.horizon) * h->cfg.n_scenarios;
  CK(cudaMemcpyAsync(h->d64, d, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(launch_round_scenarios(h->L));
  h->launches++;
  CK(cudaStreamSynchronize(h->stream));
  return RRG_OK;
}

int rrg_get_param_multipliers(rrg_handle h, double* m) {
  if (!h) return RRG_EINVAL;
  if (!m) return set_err(h, RRG_EINVAL, "m is NULL");
  DeviceGuard g(h->device);
  const size_t n = static_cast<size_t>(h->cfg.n_scenarios) * RRG_NPARAM;
  if (!h->pmul) {
    CK(cudaStreamSynchronize(h->stream));
    for (size_t q = 0; q < n; ++q) m[q] = 1.0;
    return RRG_OK;
  }
  CK(cudaMemcpyAsync(m, h->pmul, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return RRG_OK;
}

int rrg_set_param_multipliers(rrg_handle h, const double* m) {
  if (!h) return RRG_EINVAL;
  if (!m) return set_err(h, RRG_EINVAL, "m is NULL");
  if (!h->pmul) return set_err(h, RRG_EINVAL, "the handle has no parametric uncertainty (param_unc_rel = 0)");
  const size_t n = static_cast<size_t>(h->cfg.n_scenarios) * RRG_NPARAM;
  for (size_t q = 0; q < n; ++q)
    if (!is_fin(m[q]) || !(m[q] > 0.0))
      return set_err(h, RRG_EINVAL, "m[%zu] must be finite and > 0", q);
  DeviceGuard g(h->device);
  h->cl_next_ready = false;
  CK(cudaMemcpyAsync(h->pmul, m, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return RRG_OK;
}

int rrg_get_scenarios(rrg_handle h, double* d) {
  if (!h) return RRG_EINVAL;
  if (!d) return set_err(h, RRG_EINVAL, "d is NULL");
  DeviceGuard g(h->device);
  const size_t n = 3 * static_cast<size_t>(h->cfg.horizon) * h->cfg.n_scenarios;
  CK(launch_materialize64(h->L));
  h->launches += 2;
  CK(cudaMemcpyAsync(d, h->d64, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return RRG_OK;
}

int rrg_eval_candidates(rrg_handle h, const double* x_t, double v_prev, double r_t,
                        const double* kappas, int m, uint8_t* admissible, double* min_slack,
                        uint8_t* P) {
  if (!h) return RRG_EINVAL;
  if (!x_ok(x_t) || !is_fin(v_prev) || !is_fin(r_t) || !(v_prev > 0.0) || !(r_t > 0.0))
    return set_err(h, RRG_EINVAL, "x_t, v_prev, r_t must be finite and v_prev, r_t > 0");
  if (!kappas || !admissible || m < 1 || m > h->cfg.max_candidates)
    return set_err(h, RRG_EINVAL, "need 1 <= m <= max_candidates and non-NULL kappas/admissible");
  for (int i = 0; i < m; ++i)
    if (!(kappas[i] >= 0.0 && kappas[i] <= 1.0))
      return set_err(h, RRG_EINVAL, "kappas[%d] outside [0, 1]", i);
  DeviceGuard g(h->device);
  const int M = h->cfg.max_candidates;
  double* kap_h = h->io_h + IO_LEN;
  uint8_t* adm_h = reinterpret_cast<uint8_t*>(h->io_h + IO_LEN + 2 * M);
  std::memcpy(h->io_h + IO_X, x_t, 3 * sizeof(double));
  std::memcpy(kap_h, kappas, m * sizeof(double));
  CK(cudaMemcpyAsync(h->io_dev, h->io_h, IO_LEN * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->kap_dev, kap_h, m * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  Launch L = h->L;
  int early = h->cfg.early_exit;
  if (P) {
    if (!h->P_dev) CK(cudaMalloc(reinterpret_cast<void**>(&h->P_dev),
                                 static_cast<size_t>(M) * h->cfg.n_scenarios));
    L.P = h->P_dev;
    if (early > RRG_EXIT_LANE) early = RRG_EXIT_LANE;
  }
  CK(launch_eval_prepare(L, h->io_dev + IO_X, v_prev, r_t, h->kap_dev, m));
  CK(launch_prepare(L, m));
  h->launches += 2;
  int rc = enqueue_round_work(h, L, m, early);
  if (rc != RRG_OK) return rc;
  CK(launch_eval_finish(L, m, h->adm_dev, h->kap_dev + M));
  h->launches++;
  CK(cudaMemcpyAsync(adm_h, h->adm_dev, m, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(kap_h + M, h->kap_dev + M, m * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (P)
    CK(cudaMemcpyAsync(P, h->P_dev, static_cast<size_t>(m) * h->cfg.n_scenarios,
                       cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::memcpy(admissible, adm_h, m);
  if (min_slack) std::memcpy(min_slack, kap_h + M, m * sizeof(double));
  return RRG_OK;
}

int rrg_slack_error(rrg_handle h, const double* x_t, double v_prev, double r_t,
                    const double* kappas, int m, double band, double* err, int32_t* j_err,
                    double* smin32, double* smin64, int32_t* unsafe, double* ratio) {
  if (!h) return RRG_EINVAL;
  if (h->cfg.precision == RRG_FP64)
    return set_err(h, RRG_EINVAL, "the handle draws no binary32 scenarios (precision RRG_FP64)");
  if (!x_ok(x_t) || !is_fin(v_prev) || !is_fin(r_t) || !(v_prev > 0.0) || !(r_t > 0.0))
    return set_err(h, RRG_EINVAL, "x_t, v_prev, r_t must be finite and v_prev, r_t > 0");
  if (!kappas || !err || m < 1 || m > h->cfg.max_candidates)
    return set_err(h, RRG_EINVAL, "need 1 <= m <= max_candidates and non-NULL kappas/err");
  if (!(band >= 0.0) || !(band <= 1e30))
    return set_err(h, RRG_EINVAL, "band must be finite and >= 0");
  for (int i = 0; i < m; ++i)
    if (!(kappas[i] >= 0.0 && kappas[i] <= 1.0))
      return set_err(h, RRG_EINVAL, "kappas[%d] outside [0, 1]", i);
  DeviceGuard g(h->device);
  const size_t lanes = static_cast<size_t>(m) * h->cfg.n_scenarios;
  const size_t need = lanes * (4 * sizeof(double) + 2 * sizeof(int32_t));
  if (need > h->err_cap) {
    CK(cudaStreamSynchronize(h->stream));
    if (h->err_buf) cudaFree(h->err_buf);
    h->err_buf = nullptr;
    h->err_cap = 0;
    CK(cudaMalloc(&h->err_buf, need));
    h->err_cap = need;
  }
  double* d_err = static_cast<double*>(h->err_buf);
  double* d_s32 = d_err + lanes;
  double* d_s64 = d_s32 + lanes;
  double* d_ratio = d_s64 + lanes;
  int32_t* d_j = reinterpret_cast<int32_t*>(d_ratio + lanes);
  int32_t* d_bad = d_j + lanes;
  double* kap_h = h->io_h + IO_LEN;
  std::memcpy(h->io_h + IO_X, x_t, 3 * sizeof(double));
  std::memcpy(kap_h, kappas, m * sizeof(double));
  CK(cudaMemcpyAsync(h->io_dev, h->io_h, IO_LEN * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->kap_dev, kap_h, m * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  const Launch& L = h->L;
  CK(launch_eval_prepare(L, h->io_dev + IO_X, v_prev, r_t, h->kap_dev, m));
  CK(launch_prepare(L, m));
  CK(launch_slack_error(L, m, static_cast<float>(band), d_err, d_j, d_s32, d_s64, d_bad, d_ratio));
  h->launches += 3;
  CK(cudaMemcpyAsync(err, d_err, lanes * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (smin32) CK(cudaMemcpyAsync(smin32, d_s32, lanes * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (smin64) CK(cudaMemcpyAsync(smin64, d_s64, lanes * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (j_err) CK(cudaMemcpyAsync(j_err, d_j, lanes * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  if (unsafe) CK(cudaMemcpyAsync(unsafe, d_bad, lanes * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  if (ratio) CK(cudaMemcpyAsync(ratio, d_ratio, lanes * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return RRG_OK;
}

// The search of rrg_step, captured once on the handle's fixed io pointers:
// with a pipelined search the rounds after the pipelined pair sit in a
// conditional node (as in the closed-loop graph), else, or if the graph API
// refuses a step, the plain sequence.  Sets the host counters one replay adds
// (the conditional body's are added on the device when it runs); nullptr if
// nothing could be captured.
cudaGraphExec_t capture_step(rrg_ctx* h) {
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  double* io = h->io_dev;
  const uint64_t l0 = h->launches, r0 = h->rollout_launches, d0 = h->rounds;
  auto end_capture = [&]() {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(h->stream, &g);
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
  };
  cudaGraph_t G = nullptr;
  if (search_pipelined(h->scfg, h->cfg.horizon)) {
    bool ok = cudaGraphCreate(&G, 0) == cudaSuccess;
    cudaGraphConditionalHandle hc = 0;
    if (ok) ok = cudaGraphConditionalHandleCreate(&hc, G, 1u, cudaGraphCondAssignDefault) == cudaSuccess;
    std::vector<cudaGraphNode_t> sinks;
    if (ok) ok = cudaStreamBeginCaptureToGraph(h->stream, G, nullptr, nullptr, 0, mode) == cudaSuccess;
    if (ok) {
      h->capturing = true;
      h->L.cond = hc;
      extra_round_counts(h, &h->L.cond_launches, &h->L.cond_rollouts, &h->L.cond_rounds);
      ok = enqueue_search(h, io + IO_X, io + IO_R, nullptr, io + IO_V, io + IO_OUT, io + IO_OUT + 1,
                          h->flag_dev, -1, false) == RRG_OK;
      h->L.cond = 0ull;
      h->capturing = false;
      h->st_per = h->launches - l0;
      h->st_rl_per = h->rollout_launches - r0;
      h->st_rd_per = h->rounds - d0;
      if (ok) {
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        ok = cudaStreamGetCaptureInfo(h->stream, &st, nullptr, nullptr, &deps, nullptr, &nd) == cudaSuccess &&
             nd > 0;
        if (ok) sinks.assign(deps, deps + nd);
      }
      cudaGraph_t g1 = nullptr;
      ok = (cudaStreamEndCapture(h->stream, &g1) == cudaSuccess) && ok;
    }
    if (ok) {
      cudaGraphNodeParams cp{};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = hc;
      cp.conditional.type = cudaGraphCondTypeIf;
      cp.conditional.size = 1;
      cudaGraphNode_t cn = nullptr;
      ok = cudaGraphAddNode(&cn, G, sinks.data(), nullptr, sinks.size(), &cp) == cudaSuccess;
      cudaGraph_t body = ok ? cp.conditional.phGraph_out[0] : nullptr;
      if (ok) ok = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, mode) == cudaSuccess;
      if (ok) {
        h->capturing = true;
        ok = enqueue_extra_rounds(h, io + IO_OUT, io + IO_OUT + 1, h->flag_dev) == RRG_OK;
        h->capturing = false;
        ok = (cudaStreamEndCapture(h->stream, &body) == cudaSuccess) && ok;
      }
    }
    if (!ok) {
      end_capture();
      if (G) cudaGraphDestroy(G);
      G = nullptr;
    }
    h->launches = l0;
    h->rollout_launches = r0;
    h->rounds = d0;
  }
  if (!G) {
    if (cudaStreamBeginCapture(h->stream, mode) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    h->capturing = true;
    const int rc = enqueue_search(h, io + IO_X, io + IO_R, nullptr, io + IO_V, io + IO_OUT, io + IO_OUT + 1,
                                  h->flag_dev);
    h->capturing = false;
    h->st_per = h->launches - l0;
    h->st_rl_per = h->rollout_launches - r0;
    h->st_rd_per = h->rounds - d0;
    h->launches = l0;
    h->rollout_launches = r0;
    h->rounds = d0;
    const cudaError_t ce = cudaStreamEndCapture(h->stream, &G);
    if (rc != RRG_OK || ce != cudaSuccess) {
      if (G) cudaGraphDestroy(G);
      end_capture();
      return nullptr;
    }
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ce = cudaGraphInstantiate(&ex, G, 0);
  cudaGraphDestroy(G);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return ex;
}

int rrg_step(rrg_handle h, const double* x_t, double r_t, double v_prev, double* v_t,
             double* kappa, int32_t* flags) {
  if (!h) return RRG_EINVAL;
  if (!x_ok(x_t) || !is_fin(v_prev) || !is_fin(r_t) || !(v_prev > 0.0) || !(r_t > 0.0))
    return set_err(h, RRG_EINVAL, "x_t, v_prev, r_t must be finite and v_prev, r_t > 0");
  DeviceGuard g(h->device);
  std::memcpy(h->io_h + IO_X, x_t, 3 * sizeof(double));
  h->io_h[IO_R] = r_t;
  h->io_h[IO_V] = v_prev;
  CK(cudaMemcpyAsync(h->io_dev, h->io_h, 5 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  // the search as one graph replay (its launch gaps cost about 50 us per
  // update when enqueued kernel by kernel), except while the library times
  // rollout launches (profiling), which needs the direct launches' events
  if (!h->profiling && !h->st_exec && !h->st_refused) {
    h->st_exec = capture_step(h);
    h->st_refused = h->st_exec == nullptr;
  }
  if (!h->profiling && h->st_exec) {
    CK(cudaGraphLaunch(h->st_exec, h->stream));
    h->launches += h->st_per;
    h->rollout_launches += h->st_rl_per;
    h->rounds += h->st_rd_per;
  } else {
    int rc = enqueue_search(h, h->io_dev + IO_X, h->io_dev + IO_R, nullptr, h->io_dev + IO_V,
                            h->io_dev + IO_OUT, h->io_dev + IO_OUT + 1, h->flag_dev);
    if (rc != RRG_OK) return rc;
  }
  CK(cudaMemcpyAsync(h->io_h + IO_OUT, h->io_dev + IO_OUT, 2 * sizeof(double),
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->flag_h, h->flag_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (v_t) *v_t = h->io_h[IO_OUT];
  if (kappa) *kappa = h->io_h[IO_OUT + 1];
  if (flags) *flags = h->flag_h[0];
  return RRG_OK;
}

int rrg_step_dev(rrg_handle h, const double* d_x_t, const double* d_r_t, const double* d_v_prev,
                 double* d_v_t, double* d_kappa, int32_t* d_flags) {
  if (!h) return RRG_EINVAL;
  if (!d_x_t || !d_r_t || !d_v_prev) return set_err(h, RRG_EINVAL, "input pointers must be non-NULL");
  DeviceGuard g(h->device);
  return enqueue_search(h, d_x_t, d_r_t, nullptr, d_v_prev, d_v_t, d_kappa, d_flags);
}

int rrg_equilibrium(rrg_handle h, double v, double* x_eq, double* y_ss) {
  if (!h) return RRG_EINVAL;
  if (!is_fin(v) || !(v > 0.0)) return set_err(h, RRG_EINVAL, "v must be finite and > 0");
  DeviceGuard g(h->device);
  CK(launch_equilibrium(h->L, v, h->io_dev + IO_OUT, h->flag_dev + 1));
  h->launches++;
  CK(cudaMemcpyAsync(h->io_h + IO_OUT, h->io_dev + IO_OUT, 4 * sizeof(double),
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->flag_h + 1, h->flag_dev + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->flag_h[1] != 0) return set_err(h, RRG_EINVAL, "no equilibrium found for v = %g", v);
  if (x_eq) std::memcpy(x_eq, h->io_h + IO_OUT, 3 * sizeof(double));
  if (y_ss) *y_ss = h->io_h[IO_OUT + 3];
  return RRG_OK;
}

int rrg_step_latency(rrg_handle h, double v, int steps, double* cycles_per_step) {
  if (!h) return RRG_EINVAL;
  if (!is_fin(v) || !(v > 0.0) || steps < 1 || !cycles_per_step)
    return set_err(h, RRG_EINVAL, "v must be finite and > 0, steps >= 1, cycles_per_step non-NULL");
  DeviceGuard g(h->device);
  double best = 0.0;
  for (int rep = 0; rep < 3; ++rep) {  // the first run also warms the instruction caches
    CK(launch_step_latency(h->L, v, steps, h->io_dev + IO_OUT, h->flag_dev + 1));
    h->launches++;
    CK(cudaMemcpyAsync(h->io_h + IO_OUT, h->io_dev + IO_OUT, 2 * sizeof(double),
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h->flag_h + 1, h->flag_dev + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->flag_h[1] != 0) return set_err(h, RRG_EINVAL, "no equilibrium found for v = %g", v);
    if (rep == 0 || h->io_h[IO_OUT] < best) best = h->io_h[IO_OUT];
  }
  *cycles_per_step = best;
  return RRG_OK;
}

int rrg_plant_step(rrg_handle h, const double* x_t, double v_t, uint64_t seed, uint64_t t,
                   const double* plant_amp, double* x_next) {
  if (!h) return RRG_EINVAL;
  if (!x_ok(x_t) || !is_fin(v_t) || !x_ok(plant_amp) || !x_next)
    return set_err(h, RRG_EINVAL, "x_t, v_t, plant_amp must be finite and x_next non-NULL");
  DeviceGuard g(h->device);
  std::memcpy(h->io_h + IO_X, x_t, 3 * sizeof(double));
  h->io_h[IO_V] = v_t;
  std::memcpy(h->io_h + IO_AMP, plant_amp, 3 * sizeof(double));
  CK(cudaMemcpyAsync(h->io_dev, h->io_h, IO_LEN * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(launch_plant(h->L, h->io_dev + IO_X, h->io_dev + IO_V, seed, t, nullptr, h->io_dev + IO_AMP,
                  h->io_dev + IO_OUT));
  h->launches++;
  CK(cudaMemcpyAsync(h->io_h + IO_OUT, h->io_dev + IO_OUT, 3 * sizeof(double),
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::memcpy(x_next, h->io_h + IO_OUT, 3 * sizeof(double));
  return RRG_OK;
}

int rrg_closed_loop_dev(rrg_handle h, const double* x0, double v0, const double* d_r_seq, int T,
                        uint64_t seed, uint64_t t0, const double* plant_amp, int use_graph,
                        double* d_v_out, double* d_kappa_out, int32_t* d_flags_out,
                        double* d_x_out) {
  if (!h) return RRG_EINVAL;
  if ((x0 && (!x_ok(x0) || !is_fin(v0) || !(v0 > 0.0))) || !x_ok(plant_amp) || !d_r_seq || T < 0)
    return set_err(h, RRG_EINVAL, "x0, v0, plant_amp must be finite, v0 > 0, T >= 0, r_seq non-NULL");
  DeviceGuard g(h->device);
  // the second scenario pair and the side stream, on first use (each piece
  // is retried until all exist; the launch descriptor sees none before)
  if (!h->L.d64b) {
    const size_t n = 3 * static_cast<size_t>(h->cfg.horizon) * h->cfg.n_scenarios;
    if (!h->d64b) CK(cudaMalloc(reinterpret_cast<void**>(&h->d64b), n * sizeof(double)));
    const size_t n32 = h->cfg.scenarios_in_register ? 1 : n;
    if (!h->d32b) CK(cudaMalloc(reinterpret_cast<void**>(&h->d32b), n32 * sizeof(float)));
    if (h->pmul && !h->pmulb) {
      const size_t np = static_cast<size_t>(h->cfg.n_scenarios) * RRG_NPARAM;
      CK(cudaMalloc(reinterpret_cast<void**>(&h->pmulb), np * sizeof(double)));
      CK(launch_fill(h->L, h->pmulb, np, 1.0));
    }
    if (!h->side) CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    if (!h->ev_fork) CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    if (!h->ev_join) CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    if (h->st_exec) {
      cudaGraphExecDestroy(h->st_exec);
      h->st_exec = nullptr;
    }
    if (h->tma_ok && !encode_scenario_map(&h->tmap[1], h->d32b, h->cfg.n_scenarios, h->cfg.horizon)) {
      h->tma_ok = false;  // the rings fall back to per-lane asynchronous copies
      h->L.tmap = nullptr;
    }
    h->L.d64b = h->d64b;
    h->L.d32b = h->d32b;
    h->L.pmulb = h->pmulb;
  }
  std::memcpy(h->io_h + IO_AMP, plant_amp, 3 * sizeof(double));
  CK(cudaMemcpyAsync(h->io_dev + IO_AMP, h->io_h + IO_AMP, 3 * sizeof(double),
                     cudaMemcpyHostToDevice, h->stream));
  if (x0) {
    CK(launch_loop_init(h->L, h->loop, x0, v0, d_x_out));
    h->launches++;
    h->cl_next_ready = false;
  }
  if (T == 0) return RRG_OK;
  const double* amp = h->io_dev + IO_AMP;
  const Launch& L = h->L;
  // scenarios of the first update of this call, unless the previous call of
  // the same run already drew them
  if (!(h->cl_next_ready && h->cl_seed == seed && h->cl_t0 == t0)) {
    CK(launch_sample(L, seed, t0, &h->loop->t, h->cfg.dist_amp, true));
    h->launches++;
  }
  // one update: draw update t+1 on the side stream (into the other pair)
  // while update t searches and moves the plant on the main stream
  auto enqueue_update = [&]() -> int {
    CK(cudaEventRecord(h->ev_fork, h->stream));
    CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    CK(launch_sample(L, seed, t0 + 1, &h->loop->t, h->cfg.dist_amp, true, h->side));
    CK(cudaEventRecord(h->ev_join, h->side));
    h->launches++;
    int rc = enqueue_search(h, h->loop->x, d_r_seq, &h->loop->t, &h->loop->v_prev, nullptr,
                            nullptr, nullptr, static_cast<long long>(t0));
    if (rc != RRG_OK) return rc;
    // the side-stream sampler reads the update counter, which loop_end
    // advances: join before it
    CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    CK(launch_loop_end(L, h->loop, seed, t0, amp, d_v_out, d_kappa_out, d_flags_out, d_x_out));
    h->launches++;
    return RRG_OK;
  };
  h->cl_seed = seed;
  h->cl_t0 = t0;
  h->cl_next_ready = true;
  if (!use_graph) {
    for (int t = 0; t < T; ++t) {
      int rc = enqueue_update();
      if (rc != RRG_OK) return rc;
    }
    return RRG_OK;
  }
  // Capture one update and replay it T times; the update index lives on the
  // device (loop->t), so every replay works on the next time step.  The
  // instantiated graph is kept for later calls of the same run.
  const void* key[6] = {d_r_seq, d_v_out, d_kappa_out, d_flags_out, d_x_out, h->loop};
  const bool hit = h->cl_exec != nullptr && std::memcmp(key, h->cl_key, sizeof key) == 0 &&
                   h->cl_key_seed == seed && h->cl_key_t0 == t0;
  if (!hit) {
    if (h->cl_exec) {
      cudaGraphExecDestroy(h->cl_exec);
      h->cl_exec = nullptr;
    }
    const uint64_t launches0 = h->launches, rl0 = h->rollout_launches, rounds0 = h->rounds;
    cudaGraph_t graph = nullptr;
    // A pipelined search rarely needs the rounds after its pipelined pair:
    // they go into a conditional node that runs only when the validating
    // search kernel reports the search unfinished.  Falls back to the plain
    // capture (rounds always enqueued, no-ops when done) if the graph API
    // refuses any step.
    if (search_pipelined(h->scfg, h->cfg.horizon)) {
      graph = capture_conditional_update(h, seed, t0, amp, d_r_seq, d_v_out, d_kappa_out,
                                         d_flags_out, d_x_out);
      h->launches = launches0;
      h->rollout_launches = rl0;
      h->rounds = rounds0;
    }
    int rc = RRG_OK;
    cudaError_t ce = cudaSuccess;
    h->cl_conditional = graph != nullptr;
    if (!graph) {
      CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      h->capturing = true;
      rc = enqueue_update();
      h->capturing = false;
      ce = cudaStreamEndCapture(h->stream, &graph);
      if (rc != RRG_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
      if (ce != cudaSuccess) return set_err(h, RRG_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
    } else {
      enqueue_count_only(h);
    }
    ce = cudaGraphInstantiate(&h->cl_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      h->cl_exec = nullptr;
      return set_err(h, RRG_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    }
    h->cl_per = h->launches - launches0;
    h->cl_rl_per = h->rollout_launches - rl0;
    h->cl_rd_per = h->rounds - rounds0;
    h->launches = launches0;
    h->rollout_launches = rl0;
    h->rounds = rounds0;
    std::memcpy(h->cl_key, key, sizeof key);
    h->cl_key_seed = seed;
    h->cl_key_t0 = t0;
  }
  for (int t = 0; t < T; ++t) {
    const cudaError_t ce = cudaGraphLaunch(h->cl_exec, h->stream);
    if (ce != cudaSuccess) return set_err(h, RRG_ECUDA, "graph launch: %s", cudaGetErrorString(ce));
    h->launches += h->cl_per;
    h->rollout_launches += h->cl_rl_per;
    h->rounds += h->cl_rd_per;
  }
  return RRG_OK;
}

int rrg_closed_loop(rrg_handle h, const double* x0, double v0, const double* r_seq, int T,
                    uint64_t seed, uint64_t t0, const double* plant_amp, int use_graph,
                    double* v_out, double* kappa_out, int32_t* flags_out, double* x_out) {
  if (!h) return RRG_EINVAL;
  if (T < 0 || (T > 0 && !r_seq)) return set_err(h, RRG_EINVAL, "T >= 0 and r_seq non-NULL");
  DeviceGuard g(h->device);
  // staging: r[T], v[T], kappa[T], x[3(T+1)], flags[T] (as int32 in doubles)
  const size_t need = static_cast<size_t>(T) * 3 + 3 * (static_cast<size_t>(T) + 1) + T + 4;
  if (need > h->cl_cap) {
    if (h->cl_dev) cudaFree(h->cl_dev);
    h->cl_dev = nullptr;
    h->cl_cap = 0;
    CK(cudaMalloc(reinterpret_cast<void**>(&h->cl_dev), need * sizeof(double)));
    h->cl_cap = need;
  }
  double* d_r = h->cl_dev;
  double* d_v = d_r + T;
  double* d_k = d_v + T;
  double* d_x = d_k + T;
  int32_t* d_f = reinterpret_cast<int32_t*>(d_x + 3 * (static_cast<size_t>(T) + 1));
  if (T > 0)
    CK(cudaMemcpyAsync(d_r, r_seq, T * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  int rc = rrg_closed_loop_dev(h, x0, v0, d_r, T, seed, t0, plant_amp, use_graph, d_v, d_k, d_f, d_x);
  if (rc != RRG_OK) return rc;
  if (v_out && T) CK(cudaMemcpyAsync(v_out, d_v, T * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (kappa_out && T)
    CK(cudaMemcpyAsync(kappa_out, d_k, T * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (flags_out && T)
    CK(cudaMemcpyAsync(flags_out, d_f, T * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  if (x_out)
    CK(cudaMemcpyAsync(x_out, d_x, 3 * (static_cast<size_t>(T) + 1) * sizeof(double),
                       cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return RRG_OK;
}

int rrg_slack_gradients(rrg_handle h, const double* x_t, double v_prev, double r_t, const double* kappas,
                        int m, int checkpoint, int precision, double* g, double* grad, int64_t* k_star,
                        int64_t* j_star, uint8_t* ss_ok) {
  if (!h) return RRG_EINVAL;
  if (!x_ok(x_t) || !is_fin(v_prev) || !is_fin(r_t) || !(v_prev > 0.0) || !(r_t > 0.0))
    return set_err(h, RRG_EINVAL, "x_t, v_prev, r_t must be finite and v_prev, r_t > 0");
  if (!kappas || m < 1 || m > h->cfg.max_candidates)
    return set_err(h, RRG_EINVAL, "need 1 <= m <= max_candidates and non-NULL kappas");
  for (int i = 0; i < m; ++i)
    if (!(kappas[i] >= 0.0 && kappas[i] <= 1.0))
      return set_err(h, RRG_EINVAL, "kappas[%d] outside [0, 1]", i);
  if (checkpoint < 1 || checkpoint > 1 << 16)
    return set_err(h, RRG_EINVAL, "checkpoint must be in [1, 65536]");
  if (precision != RRG_FP64 && precision != RRG_FP32)
    return set_err(h, RRG_EINVAL, "precision must be RRG_FP64 or RRG_FP32");
  DeviceGuard gd(h->device);
  int rc = adj_buffers(h, static_cast<size_t>(m), checkpoint);
  if (rc == RRG_OK) rc = adj_upload(h, x_t, v_prev, r_t, kappas, m);
  if (rc != RRG_OK) return rc;
  // the kernels as one graph replay (as rrg_step), except while the library
  // times rollout launches; the graph is keyed by the call's shape and the
  // adjoint buffers (which adj_buffers may have reallocated)
  const void* key[5] = {h->adj_ckpt, h->adj_seg, h->adj_lane_min, h->adj_lane_arg, h->adj_out};
  if (h->ad_exec && (h->ad_m != m || h->ad_ck != checkpoint || h->ad_prec != precision ||
                     std::memcmp(key, h->ad_key, sizeof key) != 0)) {
    cudaGraphExecDestroy(h->ad_exec);
    h->ad_exec = nullptr;
    h->ad_refused = false;
  }
  if (!h->profiling && !h->ad_exec && !h->ad_refused) {
    h->ad_exec = capture_gradient(h, m, checkpoint, precision);
    h->ad_refused = h->ad_exec == nullptr;
    h->ad_m = m;
    h->ad_ck = checkpoint;
    h->ad_prec = precision;
    std::memcpy(h->ad_key, key, sizeof key);
  }
  if (!h->profiling && h->ad_exec) {
    CK(cudaGraphLaunch(h->ad_exec, h->stream));
    h->launches += h->ad_per;
    h->rollout_launches += h->ad_rl_per;
  } else {
    rc = adj_enqueue_forward_kernels(h, m, checkpoint, precision, false);
    if (rc == RRG_OK) rc = adj_enqueue_reverse(h, 0, m, checkpoint, precision, true);
    if (rc != RRG_OK) return rc;
  }
  std::vector<double> out;
  std::vector<int32_t> ss;
  rc = adj_read(h, m, &out, ss_ok ? &ss : nullptr);
  if (rc != RRG_OK) return rc;
  for (int i = 0; i < m; ++i) {
    const double* o = out.data() + static_cast<size_t>(i) * kAdjOutStride;
    long long kj[2];
    std::memcpy(kj, o + 1, sizeof kj);
    if (g) g[i] = o[0];
    if (k_star) k_star[i] = kj[0];
    if (j_star) j_star[i] = kj[1];
    if (grad) std::memcpy(grad + static_cast<size_t>(i) * (4 + RRG_NPARAM), o + 3, (4 + RRG_NPARAM) * sizeof(double));
    if (ss_ok) ss_ok[i] = ss[i] ? 1 : 0;
  }
  return RRG_OK;
}

int rrg_slack_gradient(rrg_handle h, const double* x_t, double v_prev, double r_t, double kappa,
                       int checkpoint, int precision, double* g, double* grad, int64_t* k_star,
                       int64_t* j_star) {
  if (!h) return RRG_EINVAL;
  if (!(kappa >= 0.0 && kappa <= 1.0)) return set_err(h, RRG_EINVAL, "kappa outside [0, 1]");
  return rrg_slack_gradients(h, x_t, v_prev, r_t, &kappa, 1, checkpoint, precision, g, grad, k_star,
                             j_star, nullptr);
}


// Adjoint-driven search (see rrg.h).  Each round is one synchronous call:
//   A. the forward pass and argmin (no reverse sweep) at kappa = j / G, j =
//      0..G (G = 8, or the largest power of two with G + 1 <= max_candidates):
//      g and the steady-state outcome at each point.  kappa = 1 is judged
//      by the handle's own evaluation unless the binary32 g(1) is below
//      -1e-4, far outside the binary32 error (below 1e-5 on these
//      workloads), or its steady-state check failed.  Alg. 1's path below
//      kappa = 1 through the grid's outcomes gives a bracket of width 1 / G;
//   B. the reverse sweep of the bracket's upper end on the states the
//      forward pass saved, and a Newton step from there (the secant through
//      both ends' values when it leaves the bracket);
//   C. Newton steps on g(kappa) = 0, one gradient each, inside the bracket
//      (narrowed by each outcome), until the step, or the next iterate's
//      error predicted from the curvature of the last two slopes, is below
//      tol / 4;
//   D. the handle evaluates [k - tol/2, k + tol/2] around the last iterate;
//      if it does not judge the lower end admissible and the upper one not,
//      exact rounds of max_candidates points equispaced inside the judged
//      bracket (Alg. 3's rule) shrink it to at most tol.
// Only the handle's evaluations decide; the gradients steer.
int rrg_newton_search(rrg_handle h, const double* x_t, double r_t, double v_prev, double tol,
                      int max_iter, int checkpoint, int precision, double* kappa, int32_t* flags,
                      int32_t* iterations) {
  if (!h) return RRG_EINVAL;
  if (!(tol > 0.0) || max_iter < 1) return set_err(h, RRG_EINVAL, "tol > 0 and max_iter >= 1 needed");
  if (h->cfg.max_candidates < 3)
    return set_err(h, RRG_EINVAL, "the search needs max_candidates >= 3");
  if (!x_ok(x_t) || !is_fin(v_prev) || !is_fin(r_t) || !(v_prev > 0.0) || !(r_t > 0.0))
    return set_err(h, RRG_EINVAL, "x_t, v_prev, r_t must be finite and v_prev, r_t > 0");
  if (checkpoint < 1 || checkpoint > 1 << 16)
    return set_err(h, RRG_EINVAL, "checkpoint must be in [1, 65536]");
  if (precision != RRG_FP64 && precision != RRG_FP32)
    return set_err(h, RRG_EINVAL, "precision must be RRG_FP64 or RRG_FP32");
  DeviceGuard gd(h->device);
  const int M = h->cfg.max_candidates;
  int32_t grads = 0;
  int rc;
  auto done = [&](double k, int32_t fl) {
    if (kappa) *kappa = k;
    if (flags) *flags = fl;
    if (iterations) *iterations = grads;
    return RRG_OK;
  };
  // A. values on the grid j / G, j = 0..G
  int G = 8;
  while (G + 1 > M) G /= 2;
  double kg[9];
  for (int j = 0; j <= G; ++j) kg[j] = static_cast<double>(j) / G;
  rc = adj_enqueue_forward(h, x_t, v_prev, r_t, kg, G + 1, checkpoint, precision);
  if (rc != RRG_OK) return rc;
  std::vector<double> out;
  std::vector<int32_t> ss;
  rc = adj_read(h, G + 1, &out, &ss);
  if (rc != RRG_OK) return rc;
  grads += G + 1;
  auto gval = [&](int j) { return out[static_cast<size_t>(j) * kAdjOutStride]; };
  auto adm_at = [&](int j) { return ss[j] && gval(j) >= 0.0; };
  if (ss[G] && !(gval(G) < -1e-4)) {
    // kappa = 1 is not clearly inadmissible: Alg. 1's first test, judged
    const double one = 1.0;
    uint8_t adm_one = 0;
    rc = rrg_eval_candidates(h, x_t, v_prev, r_t, &one, 1, &adm_one, nullptr, nullptr);
    if (rc != RRG_OK) return rc;
    if (adm_one) return done(1.0, 0);
    // the slots were reused by the evaluation: set the grid up again
    rc = adj_enqueue_forward(h, x_t, v_prev, r_t, kg, G + 1, checkpoint, precision);
    if (rc != RRG_OK) return rc;
    rc = adj_read(h, G + 1, &out, &ss);
    if (rc != RRG_OK) return rc;
  }
  // Alg. 1's walk below kappa = 1 through the grid's levels
  int jlo = 0, jhi = G;
  while (jhi - jlo > 1) {
    const int jm = (jlo + jhi) / 2;
    if (adm_at(jm)) jlo = jm; else jhi = jm;
  }
  double lo = static_cast<double>(jlo) / G, hi = static_cast<double>(jhi) / G;
  // B. the slope at the bracket's upper end (the violating side, whose
  // argmin is the constraint's early dip, so its reverse sweep is short;
  // the admissible end's minimum often comes late in the horizon), and a
  // Newton step from there; the secant through both ends' values guards it
  rc = adj_enqueue_reverse(h, jhi, 1, checkpoint, precision);
  if (rc != RRG_OK) return rc;
  rc = adj_read(h, G + 1, &out, nullptr);
  if (rc != RRG_OK) return rc;
  const double ghi = gval(jhi), dhi = out[static_cast<size_t>(jhi) * kAdjOutStride + 3];
  double k = 0.5 * (lo + hi);
  if (ss[jhi] && ghi < 0.0 && dhi < 0.0 && std::isfinite(dhi)) {
    k = hi - ghi / dhi;
    if (adm_at(jlo) && !(k > lo)) {
      // Newton overshoots below lo: the secant root instead
      const double glo = gval(jlo);
      k = lo + (hi - lo) * glo / (glo - ghi);
    }
  }
  if (!(k > lo && k < hi)) k = 0.5 * (lo + hi);
  double curv = 0.0;  // |g''| estimate from the last two slopes (none yet)
  double k_prev = hi, d_prev = dhi;
  // C. Newton steps inside the bracket
  while (grads < max_iter && hi - lo > tol) {
    double g = 0.0, grad[4 + RRG_NPARAM];
    uint8_t s1 = 0;
    rc = rrg_slack_gradients(h, x_t, v_prev, r_t, &k, 1, checkpoint, precision, &g, grad, nullptr,
                             nullptr, &s1);
    if (rc != RRG_OK) return rc;
    ++grads;
    if (s1 && g >= 0.0) lo = k; else hi = k;
    const double slope = grad[0];
    if (std::isfinite(d_prev) && k != k_prev) curv = std::fabs(slope - d_prev) / std::fabs(k - k_prev);
    k_prev = k;
    d_prev = slope;
    double kn = (s1 && slope < 0.0 && std::isfinite(g)) ? k - g / slope : 0.5 * (lo + hi);
    if (!(kn > lo && kn < hi)) kn = 0.5 * (lo + hi);
    const double step = std::fabs(kn - k);
    const double predicted = (s1 && slope < 0.0 && curv > 0.0) ? curv * step * step / (2.0 * -slope) : step;
    k = kn;
    if (step <= 0.25 * tol || predicted <= 0.25 * tol) break;
  }
  // D. the handle's judgement of [k - tol/2, k + tol/2]
  double lo_j = 0.0, hi_j = 1.0;  // judged: lo_j admissible (or 0), hi_j not
  bool any = false;
  {
    double a = k - 0.5 * tol, b = k + 0.5 * tol;
    if (a < 0.0) a = 0.0;
    if (b > 1.0) b = 1.0;
    const double br[2] = {a, b};
    uint8_t ad[2] = {0, 0};
    rc = rrg_eval_candidates(h, x_t, v_prev, r_t, br, 2, ad, nullptr, nullptr);
    if (rc != RRG_OK) return rc;
    if (ad[1]) {            // b admissible: the boundary lies above it
      lo_j = b;
      any = true;
    } else if (ad[0]) {     // the expected outcome: [a, b], at most tol wide
      lo_j = a;
      hi_j = b;
      any = a > 0.0;
    } else {                // both inadmissible: below a
      hi_j = a;
    }
  }
  // fallback: exact k-section rounds inside the judged bracket
  std::vector<double> pts(static_cast<size_t>(M));
  std::vector<uint8_t> ad(static_cast<size_t>(M));
  while (hi_j - lo_j > tol && hi_j > 0.0) {
    for (int i = 0; i < M; ++i) pts[i] = lo_j + (hi_j - lo_j) * (i + 1) / (M + 1);
    rc = rrg_eval_candidates(h, x_t, v_prev, r_t, pts.data(), M, ad.data(), nullptr, nullptr);
    if (rc != RRG_OK) return rc;
    int best = -1;
    for (int i = 0; i < M; ++i)
      if (ad[i]) best = i;
    // Alg. 3's rule within the bracket: the largest admissible point
    const double nlo = best >= 0 ? pts[best] : lo_j;
    const double nhi = best + 1 < M ? pts[best + 1] : hi_j;
    if (best >= 0) any = true;
    lo_j = nlo;
    hi_j = nhi;
  }
  return done(any ? lo_j : 0.0, any ? 0 : 1);
}

// Speculative-bisection shape: tree width and probe length.  Neither changes
// the result (always Alg. 1's); both change the time per update.
int set_tuning(rrg_ctx* h, int m, int probe) {
  h->scfg.m_cap = m;
  h->scfg.probe_steps = probe;
  fill_launch(h);
  if (h->cl_exec) {  // the cached closed-loop graph holds the old schedule
    cudaGraphExecDestroy(h->cl_exec);
    h->cl_exec = nullptr;
  }
  return RRG_OK;
}

int rrg_set_tuning(rrg_handle h, int m, int probe_steps) {
  if (!h) return RRG_EINVAL;
  if (h->cfg.search != RRG_SEARCH_SPEC_BISECT)
    return set_err(h, RRG_EINVAL, "tuning applies to RRG_SEARCH_SPEC_BISECT");
  if (m < 1 || m > h->cfg.max_candidates)
    return set_err(h, RRG_EINVAL, "m must be in [1, max_candidates]");
  if (probe_steps < 0 || (probe_steps > 0 && !h->lane_state))
    return set_err(h, RRG_EINVAL, "probe_steps must be >= 0, and 0 unless the handle was created with probe_steps > 0");
  DeviceGuard g(h->device);
  CK(cudaStreamSynchronize(h->stream));
  return set_tuning(h, m, probe_steps);
}

int rrg_get_tuning(rrg_handle h, int32_t* m, int32_t* probe_steps) {
  if (!h) return RRG_EINVAL;
  if (m) *m = h->scfg.m_cap;
  if (probe_steps) *probe_steps = h->scfg.probe_steps;
  return RRG_OK;
}

int rrg_autotune(rrg_handle h, const double* x_t, double r_t, double v_prev, int repeats,
                 int32_t* m_out, int32_t* probe_out, double* ms_out) {
  if (!h) return RRG_EINVAL;
  if (h->cfg.search != RRG_SEARCH_SPEC_BISECT)
    return set_err(h, RRG_EINVAL, "the autotuner tunes RRG_SEARCH_SPEC_BISECT");
  if (!x_ok(x_t) || !is_fin(v_prev) || !is_fin(r_t) || !(v_prev > 0.0) || !(r_t > 0.0) || repeats < 1)
    return set_err(h, RRG_EINVAL, "x_t, v_prev, r_t must be finite, v_prev, r_t > 0, repeats >= 1");
  DeviceGuard g(h->device);
  const int cap = h->cfg.max_candidates, H = h->cfg.horizon;
  std::vector<int> ms;
  for (int m = 4; m < cap; m *= 2) ms.push_back(m);
  ms.push_back(cap);
  std::vector<int> probes = {0};
  if (h->lane_state)
    for (int p : {32, 128, 512})
      if (p < H) probes.push_back(p);
  std::memcpy(h->io_h + IO_X, x_t, 3 * sizeof(double));
  h->io_h[IO_R] = r_t;
  h->io_h[IO_V] = v_prev;
  CK(cudaMemcpyAsync(h->io_dev, h->io_h, 5 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  cudaEvent_t a = take_event(h), b = take_event(h);
  if (!a || !b) return set_err(h, RRG_ECUDA, "event creation failed");
  const bool prof = h->profiling;
  h->profiling = false;
  double best = 0.0;
  int best_m = h->scfg.m_cap, best_p = h->scfg.probe_steps, rc = RRG_OK;
  for (int m : ms) {
    for (int p : probes) {
      set_tuning(h, m, p);
      float total = 0.0f;
      for (int rep = 0; rep <= repeats && rc == RRG_OK; ++rep) {
        cudaEventRecord(a, h->stream);
        rc = enqueue_search(h, h->io_dev + IO_X, h->io_dev + IO_R, nullptr, h->io_dev + IO_V,
                            h->io_dev + IO_OUT, h->io_dev + IO_OUT + 1, h->flag_dev);
        cudaEventRecord(b, h->stream);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = RRG_ECUDA;
        float t = 0.0f;
        if (rc == RRG_OK && rep > 0 && cudaEventElapsedTime(&t, a, b) == cudaSuccess) total += t;
      }
      if (rc != RRG_OK) break;
      const double mean = total / repeats;
      if ((m == ms.front() && p == probes.front()) || mean < best) {
        best = mean;
        best_m = m;
        best_p = p;
      }
    }
    if (rc != RRG_OK) break;
  }
  h->ev_free.push_back(a);
  h->ev_free.push_back(b);
  h->profiling = prof;
  set_tuning(h, best_m, best_p);
  if (rc != RRG_OK) return set_err(h, RRG_ECUDA, "autotune: a timed update failed");
  if (m_out) *m_out = best_m;
  if (probe_out) *probe_out = best_p;
  if (ms_out) *ms_out = best;
  return RRG_OK;
}

int rrg_set_pairing(rrg_handle h, int mode) {
  if (!h) return RRG_EINVAL;
  if (mode < RRG_PAIR_NEVER || mode > RRG_PAIR_ALWAYS)
    return set_err(h, RRG_EINVAL, "pairing mode must be RRG_PAIR_NEVER, RRG_PAIR_FILLED or RRG_PAIR_ALWAYS");
  DeviceGuard g(h->device);
  CK(cudaStreamSynchronize(h->stream));
  h->pair = mode;
  fill_launch(h);
  if (h->cl_exec) {  // the cached closed-loop graph holds the old kernels
    cudaGraphExecDestroy(h->cl_exec);
    h->cl_exec = nullptr;
  }
  return RRG_OK;
}

int rrg_set_tma(rrg_handle h, int mode) {
  if (!h) return RRG_EINVAL;
  if (mode < RRG_TMA_NEVER || mode > RRG_TMA_ALWAYS)
    return set_err(h, RRG_EINVAL, "TMA mode must be RRG_TMA_NEVER, RRG_TMA_AUTO or RRG_TMA_ALWAYS");
  if (mode != RRG_TMA_NEVER && !h->tma_ok)
    return set_err(h, RRG_EINVAL, "no TMA ring for this handle (n_scenarios %% 4 != 0, in-register "
                                  "scenarios, or the driver refused the tensor map)");
  DeviceGuard g(h->device);
  CK(cudaStreamSynchronize(h->stream));
  h->tma_mode = mode;
  fill_launch(h);
  if (h->cl_exec) {  // the cached closed-loop graph holds the old kernels
    cudaGraphExecDestroy(h->cl_exec);
    h->cl_exec = nullptr;
  }
  return RRG_OK;
}

int rrg_set_injection(rrg_handle h, int flags) {
  if (!h) return RRG_EINVAL;
  if (flags & ~RRG_INJECT_TMA_NO_COPY) return set_err(h, RRG_EINVAL, "unknown injection flags 0x%x", flags);
  DeviceGuard g(h->device);
  CK(cudaStreamSynchronize(h->stream));
  h->inject = flags;
  fill_launch(h);
  if (h->cl_exec) {
    cudaGraphExecDestroy(h->cl_exec);
    h->cl_exec = nullptr;
  }
  return RRG_OK;
}

int rrg_get_tma(rrg_handle h, int32_t* mode) {
  if (!h || !mode) return RRG_EINVAL;
  *mode = h->tma_ok ? h->tma_mode : RRG_TMA_NEVER;
  return RRG_OK;
}

int rrg_get_pairing(rrg_handle h, int32_t* mode) {
  if (!h || !mode) return RRG_EINVAL;
  *mode = h->pair;
  return RRG_OK;
}

int rrg_autotune_pairing(rrg_handle h, const double* x_t, double r_t, double v_prev, int repeats,
                         int32_t* mode_out, double* ms_out) {
  if (!h) return RRG_EINVAL;
  if (!x_ok(x_t) || !is_fin(v_prev) || !is_fin(r_t) || !(v_prev > 0.0) || !(r_t > 0.0) || repeats < 1)
    return set_err(h, RRG_EINVAL, "x_t, v_prev, r_t must be finite, v_prev, r_t > 0, repeats >= 1");
  DeviceGuard g(h->device);
  std::memcpy(h->io_h + IO_X, x_t, 3 * sizeof(double));
  h->io_h[IO_R] = r_t;
  h->io_h[IO_V] = v_prev;
  CK(cudaMemcpyAsync(h->io_dev, h->io_h, 5 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  cudaEvent_t a = take_event(h), b = take_event(h);
  if (!a || !b) return set_err(h, RRG_ECUDA, "event creation failed");
  const bool prof = h->profiling;
  h->profiling = false;
  const int old = h->pair;
  int best_mode = old, rc = RRG_OK;
  double best = 0.0;
  for (int mode = RRG_PAIR_NEVER; mode <= RRG_PAIR_ALWAYS && rc == RRG_OK; ++mode) {
    h->pair = mode;
    fill_launch(h);
    float total = 0.0f;
    for (int rep = 0; rep <= repeats && rc == RRG_OK; ++rep) {
      cudaEventRecord(a, h->stream);
      rc = enqueue_search(h, h->io_dev + IO_X, h->io_dev + IO_R, nullptr, h->io_dev + IO_V,
                          h->io_dev + IO_OUT, h->io_dev + IO_OUT + 1, h->flag_dev);
      cudaEventRecord(b, h->stream);
      if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = RRG_ECUDA;
      float t = 0.0f;
      if (rc == RRG_OK && rep > 0 && cudaEventElapsedTime(&t, a, b) == cudaSuccess) total += t;
    }
    if (rc != RRG_OK) break;
    const double mean = total / repeats;
    if (ms_out) ms_out[mode] = mean;
    if (mode == RRG_PAIR_NEVER || mean < best) {
      best = mean;
      best_mode = mode;
    }
  }
  h->ev_free.push_back(a);
  h->ev_free.push_back(b);
  h->profiling = prof;
  h->pair = rc == RRG_OK ? best_mode : old;
  fill_launch(h);
  if (h->cl_exec) {
    cudaGraphExecDestroy(h->cl_exec);
    h->cl_exec = nullptr;
  }
  if (rc != RRG_OK) return set_err(h, RRG_ECUDA, "autotune: a timed update failed");
  if (mode_out) *mode_out = best_mode;
  return RRG_OK;
}

int rrg_set_profiling(rrg_handle h, int on) {
  if (!h) return RRG_EINVAL;
  h->profiling = on != 0;
  return RRG_OK;
}

int rrg_get_stats(rrg_handle h, rrg_stats* out) {
  if (!h || !out) return RRG_EINVAL;
  DeviceGuard g(h->device);
  DevStats ds{};
  CK(cudaMemcpyAsync(&ds, h->stats, sizeof ds, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (auto& pr : h->ev_roll) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, pr.first, pr.second));
    h->rollout_ms += ms;
    h->timed_rollouts++;
    h->ev_free.push_back(pr.first);
    h->ev_free.push_back(pr.second);
  }
  h->ev_roll.clear();
  for (auto& pr : h->ev_rec) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, pr.first, pr.second));
    h->recheck_ms += ms;
    h->ev_free.push_back(pr.first);
    h->ev_free.push_back(pr.second);
  }
  h->ev_rec.clear();
  out->launches = h->launches + ds.cond_launches;
  out->rollout_launches = h->rollout_launches + ds.cond_rollouts;
  out->lane_steps = ds.lane_steps;
  out->lane_steps_fp64 = ds.lane_steps_fp64;
  out->rechecked = ds.rechecked;
  out->rounds = h->rounds + ds.cond_rounds;
  out->rollout_ms = h->rollout_ms;
  out->recheck_ms = h->recheck_ms;
  out->timed_rollouts = h->timed_rollouts;
  out->repairs = ds.repairs;
  out->graph_conditional = h->cl_exec != nullptr && h->cl_conditional ? 1 : 0;
  out->lane_steps_paired = ds.lane_steps_paired;
  out->wait_timeouts = ds.wait_timeouts;
  out->lane_steps_tma = ds.lane_steps_tma;
  return RRG_OK;
}

int rrg_reset_stats(rrg_handle h) {
  if (!h) return RRG_EINVAL;
  DeviceGuard g(h->device);
  rrg_stats tmp;
  int rc = rrg_get_stats(h, &tmp);  // drains pending events
  if (rc != RRG_OK) return rc;
  CK(cudaMemsetAsync(h->stats, 0, sizeof(DevStats), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->launches = h->rollout_launches = h->rounds = 0;
  h->rollout_ms = h->recheck_ms = 0.0;
  h->timed_rollouts = 0;
  return RRG_OK;
}

// ---- Alg. 1 rounds for caller-run evaluations ---------------------------
// The speculative bisection's tree on the host: the nodes of the next levels
// of Alg. 1's bisection tree from the current state, in breadth-first order
// (heap numbering: node 2n follows "not admissible" at node n, 2n + 1
// "admissible"; an admissible kappa = 1 ends the search, so it has no
// admissible child), and the walk of Alg. 1's path through their outcomes.
namespace {

struct TreeNode {
  uint32_t heap;
  double lo, hi, kappa;
};

int tree_size(bool root_is_one, int d) { return root_is_one ? (1 << (d - 1)) : ((1 << d) - 1); }

// Levels of the next round: the most that fit in m_max nodes and in the
// iterations Alg. 1 has left (0 when the search is finished).
int tree_depth(const rrg_bisect_state* s, int m_max) {
  if (s->done || s->iter >= s->n_bisect || m_max < 1) return 0;
  const bool one = s->kappa == 1.0;
  int d = 1;
  while (d < 20 && d + 1 <= s->n_bisect - s->iter && tree_size(one, d + 1) <= m_max) ++d;
  return d;
}

int build_nodes(const rrg_bisect_state* s, int d, TreeNode* out) {
  int n = 0;
  out[n++] = TreeNode{1u, s->lo, s->hi, s->kappa};
  for (int q = 0; q < n; ++q) {
    const TreeNode a = out[q];
    int depth = 0;
    for (uint32_t h = a.heap; h > 1u; h >>= 1) ++depth;
    if (depth + 1 >= d) continue;
    out[n++] = TreeNode{2u * a.heap, a.lo, a.kappa, (a.lo + a.kappa) / 2.0};
    if (a.kappa != 1.0) out[n++] = TreeNode{2u * a.heap + 1u, a.kappa, a.hi, (a.kappa + a.hi) / 2.0};
  }
  return n;
}

}  // namespace

int rrg_bisect_init(rrg_bisect_state* s, int n_bisect) {
  if (!s || n_bisect < 1 || n_bisect > 62) return RRG_EINVAL;
  s->lo = 0.0;
  s->hi = 1.0;
  s->kappa = 1.0;
  s->kappa_opt = 0.0;
  s->iter = 0;
  s->n_bisect = n_bisect;
  s->any = 0;
  s->done = 0;
  return RRG_OK;
}

int rrg_bisect_plan(const rrg_bisect_state* s, int m_max, double* kappas, int32_t* m) {
  if (!s || !m || m_max < 1 || (m_max > 0 && !kappas)) return RRG_EINVAL;
  if (s->n_bisect < 1 || s->n_bisect > 62) return RRG_EINVAL;
  const int d = tree_depth(s, m_max > RRG_MAX_CANDIDATES ? RRG_MAX_CANDIDATES : m_max);
  if (d == 0) {
    *m = 0;
    return RRG_OK;
  }
  std::vector<TreeNode> nodes(static_cast<size_t>(tree_size(s->kappa == 1.0, d)));
  const int n = build_nodes(s, d, nodes.data());
  for (int i = 0; i < n; ++i) kappas[i] = nodes[i].kappa;
  *m = n;
  return RRG_OK;
}

int rrg_bisect_decide(rrg_bisect_state* s, const uint8_t* admissible, int m) {
  if (!s || !admissible || m < 1 || s->done) return RRG_EINVAL;
  const bool one = s->kappa == 1.0;
  int d = 0;
  for (int k = 1; k <= 20; ++k)
    if (tree_size(one, k) == m) d = k;
  if (d == 0 || d > s->n_bisect - s->iter) return RRG_EINVAL;
  std::vector<TreeNode> nodes(static_cast<size_t>(m));
  build_nodes(s, d, nodes.data());
  uint32_t heap = 1u;
  for (;;) {
    int pos = -1;
    for (int i = 0; i < m; ++i)
      if (nodes[i].heap == heap) pos = i;
    if (pos < 0) break;  // past the round's levels
    const bool ok = admissible[pos] != 0;
    s->iter += 1;
    if (ok) {
      s->kappa_opt = s->kappa;
      s->any = 1;
      if (s->kappa == 1.0) {
        s->done = 1;
        break;
      }
      s->lo = s->kappa;
    } else {
      s->hi = s->kappa;
    }
    s->kappa = (s->lo + s->hi) / 2.0;
    if (s->iter >= s->n_bisect) {
      s->done = 1;
      break;
    }
    heap = 2u * heap + (ok ? 1u : 0u);
  }
  return RRG_OK;
}

}  // extern "C"

namespace rrg {
// Used by the handle-less entry point in rrg_static.cu.
int check_config(const rrg_config* c) { return validate_cfg(c); }
void set_thread_error(const char* msg) { g_create_error = msg; }
}  // namespace rrg
