// rrg_static.cu -- rrg_eval_candidates_static: candidate evaluation that
// allocates nothing.  Its working memory is one file-scope device array of
// fixed size; everything else is the caller's.  The paper has no counterpart
// of this entry point: it exists for callers that cannot allocate device
// memory while they run (see include/rrg.h).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda.h>  // driver types only (CUcontext); the calls go through cudaGetDriverEntryPoint

#include "rrg_internal.h"

namespace rrg {
namespace {

constexpr int kStaticMaxCand = RRG_STATIC_MAX_CANDIDATES;
constexpr size_t kStaticMaxLanes = RRG_STATIC_MAX_LANES;

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t align256(size_t n) { return (n + 255) & ~static_cast<size_t>(255); }
constexpr size_t kOffState = 0;
constexpr size_t kOffParams = kOffState + align256(sizeof(SearchState));
constexpr size_t kOffPws = kOffParams + align256(RRG_NPARAM * sizeof(double));
constexpr size_t kOffKappa = kOffPws + align256(sizeof(PowSeries));
constexpr size_t kOffV = kOffKappa + align256(kStaticMaxCand * sizeof(double));
constexpr size_t kOffK64 = kOffV + align256(kStaticMaxCand * sizeof(double));
constexpr size_t kOffK32 = kOffK64 + align256(kStaticMaxCand * sizeof(RhsC<double>));
constexpr size_t kOffOk = kOffK32 + align256(kStaticMaxCand * sizeof(RhsC<float>));
constexpr size_t kOffDead = kOffOk + align256(kStaticMaxCand * sizeof(int32_t));
constexpr size_t kOffSs = kOffDead + align256(kStaticMaxCand * sizeof(int32_t));
constexpr size_t kOffMin = kOffSs + align256(kStaticMaxCand * sizeof(int32_t));
constexpr size_t kOffCount = kOffMin + align256(kStaticMaxCand * sizeof(unsigned long long));
constexpr size_t kOffStats = kOffCount + align256(sizeof(uint32_t));
constexpr size_t kOffList = kOffStats + align256(sizeof(DevStats));
constexpr size_t kOffJlast = kOffList + align256(kStaticMaxLanes * sizeof(uint32_t));
constexpr size_t kScratchBytes = kOffJlast + align256(kStaticMaxLanes * sizeof(uint32_t));
static_assert(kScratchBytes <= RRG_STATIC_SCRATCH_BYTES, "scratch layout exceeds its stated size");

// The scratch itself: held by every device that loads the library.
__device__ __align__(256) unsigned char g_rrg_static_scratch[RRG_STATIC_SCRATCH_BYTES];

struct ParamBlock {
  double v[RRG_NPARAM];
  PowSeries pws;   // binary64 x^e - 1 series of the model's exponent (as rrg_create builds it)
};

// Writes the parameter vector and the x^e - 1 series (passed by value) into
// the scratch and clears the scratch's step counters.
__global__ void static_params_kernel(ParamBlock pb, double* params, PowSeries* pws,
                                     DevStats* stats, SearchState* st) {
  const int i = threadIdx.x;
  if (i < RRG_NPARAM) params[i] = pb.v[i];
  if (i == 0) *pws = pb.pws;
  if (i == 0) {
    st->src[0].d64_valid = 1;  // the caller's binary64 array holds the values
    st->src[1].d64_valid = 1;
    stats->lane_steps = 0ull;
    stats->lane_steps_fp64 = 0ull;
    stats->rechecked = 0ull;
  }
}

// Device address of the scratch, looked up once per device and context: a
// device reset or a recreated primary context loads the module again, and
// the array may then sit at another address, so each cached address is kept
// with the id of the context it was looked up in (cuCtxGetId, reached through
// cudaGetDriverEntryPointByVersion so that the library needs no link to the
// driver library).  The SM count is cached beside it.
std::mutex g_mu;
constexpr int kMaxDevices = 64;
struct ScratchEntry {
  unsigned long long ctx_id;
  unsigned char* ptr;
  int sms;
};
ScratchEntry g_scratch[kMaxDevices] = {};
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_thread_error(buf);
  return code;
}

// Id of the calling thread's current context (0 if none is current yet).
int current_context_id(unsigned long long* id) {
  if (g_ctx_get_current == nullptr || g_ctx_get_id == nullptr) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    const cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    const cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
        q2 != cudaDriverEntryPointSuccess || f1 == nullptr || f2 == nullptr)
      return fail(RRG_ECUDA, "the driver's cuCtxGetCurrent / cuCtxGetId are not available");
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return fail(RRG_ECUDA, "cuCtxGetCurrent failed");
  *id = 0;
  if (ctx != nullptr && g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return fail(RRG_ECUDA, "cuCtxGetId failed");
  return RRG_OK;
}

int scratch_for_current_device(unsigned char** out, int* sms) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(RRG_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(RRG_EINVAL, "device ordinal %d not supported", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long ctx = 0;
  int rc = current_context_id(&ctx);
  if (rc != RRG_OK) return rc;
  ScratchEntry& c = g_scratch[dev];
  if (c.ptr == nullptr || ctx == 0 || c.ctx_id != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_rrg_static_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(RRG_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || n < 1)
      return fail(RRG_ECUDA, "cudaDeviceGetAttribute(SM count): %s", cudaGetErrorString(e));
    // the look-up made the primary context current if none was
    rc = current_context_id(&ctx);
    if (rc != RRG_OK) return rc;
    c.ctx_id = ctx;
    c.ptr = static_cast<unsigned char*>(p);
    c.sms = n;
  }
  *out = c.ptr;
  *sms = c.sms;
  return RRG_OK;
}

}  // namespace
}  // namespace rrg

using namespace rrg;

extern "C" int rrg_eval_candidates_static(const double* model_params, int n_params,
                                          const rrg_config* cfg, void* cuda_stream,
                                          const double* d_scen64, const float* d_scen32,
                                          const double* d_x_t, double v_prev, double r_t,
                                          const double* d_kappas, int m, uint8_t* d_admissible,
                                          double* d_min_slack) {
  if (!model_params || n_params != RRG_NPARAM)
    return fail(RRG_EINVAL, "model_params must hold %d values", RRG_NPARAM);
  for (int i = 0; i < RRG_NPARAM; ++i)
    if (!std::isfinite(model_params[i])) return fail(RRG_EINVAL, "model_params[%d] not finite", i);
  int rc = check_config(cfg);
  if (rc != RRG_OK) return rc;
  if (cfg->param_unc_rel != 0.0 || cfg->scenarios_in_register != 0)
    return fail(RRG_ENOTIMPL, "the allocation-free evaluation has no parametric uncertainty "
                "and reads the caller's scenarios (param_unc_rel and scenarios_in_register must be 0)");
  if (m < 1 || m > cfg->max_candidates || m > kStaticMaxCand)
    return fail(RRG_EINVAL, "m = %d: the allocation-free evaluation takes 1..%d candidates "
                "(and at most max_candidates)", m, kStaticMaxCand);
  const size_t lanes = static_cast<size_t>(m) * static_cast<size_t>(cfg->n_scenarios);
  if (lanes > kStaticMaxLanes)
    return fail(RRG_EINVAL, "m * n_scenarios = %zu exceeds the scratch limit of %zu trajectories",
                lanes, kStaticMaxLanes);
  if (!std::isfinite(v_prev) || !std::isfinite(r_t) || !(v_prev > 0.0) || !(r_t > 0.0))
    return fail(RRG_EINVAL, "v_prev and r_t must be finite and > 0");
  if (!d_x_t || !d_kappas || !d_admissible)
    return fail(RRG_EINVAL, "d_x_t, d_kappas and d_admissible must be non-NULL");
  const bool need64 = cfg->precision != RRG_FP32, need32 = cfg->precision != RRG_FP64;
  if ((need64 && !d_scen64) || (need32 && !d_scen32))
    return fail(RRG_EINVAL, "precision %d needs the %s scenario array(s)", cfg->precision,
                cfg->precision == RRG_FP64 ? "binary64" : (cfg->precision == RRG_FP32 ? "binary32" : "binary64 and binary32"));

  unsigned char* base = nullptr;
  int sms = 0;
  rc = scratch_for_current_device(&base, &sms);
  if (rc != RRG_OK) return rc;

  Launch L{};
  L.stream = static_cast<cudaStream_t>(cuda_stream);
  L.N = cfg->n_scenarios;
  L.H = cfg->horizon;
  L.precision = cfg->precision;
  L.early_exit = cfg->early_exit;
  L.m_cap = m;
  L.dt = cfg->dt;
  L.y_min = cfg->y_min;
  L.eps_abs = cfg->precision == RRG_FP32_RECHECK ? cfg->recheck_eps_rel * std::fabs(cfg->y_min) : 0.0;
  L.scfg.search = cfg->search;
  L.scfg.m_cap = m;
  L.scfg.n_bisect = cfg->n_bisect;
  L.scfg.n_rounds = cfg->n_rounds;
  L.scfg.ss_check = cfg->ss_check;
  L.scfg.y_min = cfg->y_min;
  L.scfg.eps_ss = cfg->eps_ss;
  L.scfg.y_c = cfg->y_c;
  fold_constants(model_params, &L.k64, &L.k32);
  // the binary64 rollouts and the recheck evaluate x^e - 1 by the same series
  // as a handle's, so both give the same bits
  L.k64.pws = reinterpret_cast<const PowSeries*>(base + kOffPws);
  fold_rhs(L.k64, &L.u64, &L.u32);
  L.params = reinterpret_cast<double*>(base + kOffParams);
  L.d64 = const_cast<double*>(d_scen64);
  L.d32 = const_cast<float*>(d_scen32);
  L.st = reinterpret_cast<SearchState*>(base + kOffState);
  L.cand_kappa = reinterpret_cast<double*>(base + kOffKappa);
  L.cand_v = reinterpret_cast<double*>(base + kOffV);
  L.cand_c64 = reinterpret_cast<RhsC<double>*>(base + kOffK64);
  L.cand_c32 = reinterpret_cast<RhsC<float>*>(base + kOffK32);
  L.cand_ok = reinterpret_cast<int32_t*>(base + kOffOk);
  L.cand_dead = reinterpret_cast<int32_t*>(base + kOffDead);
  L.cand_ss = reinterpret_cast<int32_t*>(base + kOffSs);
  L.cand_min = reinterpret_cast<unsigned long long*>(base + kOffMin);
  L.recheck_count = reinterpret_cast<uint32_t*>(base + kOffCount);
  L.stats = reinterpret_cast<DevStats*>(base + kOffStats);
  L.recheck_list = reinterpret_cast<uint32_t*>(base + kOffList);
  L.recheck_jlast = reinterpret_cast<uint32_t*>(base + kOffJlast);
  L.P = nullptr;
  L.sms = sms;
  L.recheck_blocks = 2 * sms;

  ParamBlock pb;
  std::memcpy(pb.v, model_params, sizeof pb.v);
  make_pow_series((model_params[P_GAMMA] - 1.0) / model_params[P_GAMMA], &pb.pws);
  static_params_kernel<<<1, 32, 0, L.stream>>>(pb, const_cast<double*>(L.params),
                                               const_cast<PowSeries*>(L.k64.pws), L.stats, L.st);
  cudaError_t e = cudaGetLastError();
  // the prepare kernel rewrites every per-candidate flag, key and the recheck
  // count, so nothing left in the scratch by an earlier call is read
  if (e == cudaSuccess) e = launch_eval_prepare(L, d_x_t, v_prev, r_t, d_kappas, m);
  if (e == cudaSuccess) e = launch_prepare(L, m);
  if (e == cudaSuccess)
    e = launch_rollout(L, m, cfg->precision == RRG_FP64, cfg->early_exit,
                       cfg->precision == RRG_FP32_RECHECK);
  if (e == cudaSuccess && cfg->precision == RRG_FP32_RECHECK) e = launch_recheck(L, cfg->early_exit);
  if (e == cudaSuccess) e = launch_eval_finish(L, m, d_admissible, d_min_slack);
  if (e != cudaSuccess) return fail(RRG_ECUDA, "launch: %s", cudaGetErrorString(e));
  return RRG_OK;
}
