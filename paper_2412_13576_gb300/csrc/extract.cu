// mape_extract: argument checks and dispatch by precision; library-wide
// helpers (default configuration, version, CUDA error record).
#include "common.cuh"
#include "extract_internal.cuh"

#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>

namespace mape_detail {

static std::mutex g_err_mu;
static char g_last_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void record_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  std::snprintf(g_last_err, sizeof(g_last_err), "%s (%d) at %s:%d in %s", cudaGetErrorString(e), (int)e,
                file, line, what);
}

}  // namespace mape_detail

extern "C" const char* mape_last_cuda_error(void) { return mape_detail::g_last_err; }

extern "C" unsigned long long mape_launch_count(void) { return mape_detail::g_launches.load(); }

extern "C" const char* mape_version(void) { return "mape-gb300 0.1 (sm_103a)"; }

extern "C" void mape_default_config(mape_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->lambda1 = 0.85f;
  cfg->lambda2 = 1.0f;
  cfg->lr = 0.003f;
  cfg->beta1 = 0.9;
  cfg->beta2 = 0.999;
  cfg->eps = 1e-8f;
  cfg->T = 1000;
  cfg->period = 1;
  cfg->precision = MAPE_PREC_BF16;
  cfg->cand_capacity = 0;
  cfg->max_aug_iters = 1000000;
}

namespace {
bool valid_precision(int32_t precision) {
  const int32_t base = precision & MAPE_PREC_MASK, extra = precision & ~MAPE_PREC_MASK;
  if (base == MAPE_PREC_FP32) return extra == 0;
  return (base == MAPE_PREC_BF16 || base == MAPE_PREC_BF16X1) && (extra & ~MAPE_PREC_STREAMED) == 0;
}
}  // namespace

extern "C" size_t mape_extract_workspace_bytes(int32_t n, int32_t d, int32_t P, int32_t precision) {
  if (n <= 0 || d <= 0 || P < 0 || !valid_precision(precision)) return 0;
  const int32_t base = precision & MAPE_PREC_MASK;
  if (base == MAPE_PREC_FP32) return mape_detail::extract_fp32_workspace(n, d, P);
  // the streamed path also serves a general B of a shape whose resident tile
  // fits only when B is identity-topped, so its workspace is always included
  size_t w = mape_detail::extract_stream_workspace(n, d, P);
  if (!(precision & MAPE_PREC_STREAMED)) {
    const size_t t = mape_detail::extract_tc_workspace(n, d, P, base);
    if (t > w) w = t;
  }
  return w;
}

extern "C" int mape_extract(const mape_extract_args* a, void* stream) {
  if (!a) return MAPE_ERR_INVALID_ARG;
  if (a->n <= 0 || a->d <= 0 || a->d > a->n || a->P < 0 || a->T < 0 || a->t0 < 0 || a->period <= 0)
    return MAPE_ERR_INVALID_ARG;
  if (!a->B || !a->span || !a->cand_count || !a->flags) return MAPE_ERR_INVALID_ARG;
  if (a->P > 0 && (!a->Z || !a->M || !a->V)) return MAPE_ERR_INVALID_ARG;
  if (a->ldc < a->n || a->ldc % 16 != 0 || a->cand_cap < 0 || (a->cand_cap > 0 && !a->cand))
    return MAPE_ERR_INVALID_ARG;
  if (!valid_precision(a->precision)) return MAPE_ERR_INVALID_ARG;
  if (a->P == 0 || a->T == 0) return MAPE_OK;
  cudaStream_t st = mape_detail::as_stream(stream);
  const int32_t base = a->precision & MAPE_PREC_MASK;
  if (base != MAPE_PREC_FP32) {
    if (!mape_detail::extract_stream_supported(a->n, a->d)) return MAPE_ERR_SHAPE;
    if (a->workspace_bytes < mape_extract_workspace_bytes(a->n, a->d, a->P, a->precision)) return MAPE_ERR_CAPACITY;
    mape_extract_args b = *a;
    b.precision = base;
    if (!(a->precision & MAPE_PREC_STREAMED) && mape_detail::extract_tc_supported(a->n, a->d, base)) {
      const int rc = mape_detail::extract_tc(&b, st);
      if (rc != MAPE_ERR_SHAPE) return rc;  // SHAPE: a general B that only the streamed path takes
    }
    return mape_detail::extract_stream(&b, st);
  }
  if (a->workspace_bytes < mape_detail::extract_fp32_workspace(a->n, a->d, a->P)) return MAPE_ERR_CAPACITY;
  return mape_detail::extract_fp32(a, st);
}
