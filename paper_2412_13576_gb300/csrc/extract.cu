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

extern "C" size_t mape_extract_workspace_bytes(int32_t n, int32_t d, int32_t P, int32_t precision) {
  if (n <= 0 || d <= 0 || P < 0) return 0;
  if (precision == MAPE_PREC_BF16 || precision == MAPE_PREC_BF16X1)
    return mape_detail::extract_tc_workspace(n, d, P, precision);
  return mape_detail::extract_fp32_workspace(n, d, P);
}

extern "C" int mape_extract(const mape_extract_args* a, void* stream) {
  if (!a) return MAPE_ERR_INVALID_ARG;
  if (a->n <= 0 || a->d <= 0 || a->d > a->n || a->P < 0 || a->T < 0 || a->t0 < 0 || a->period <= 0)
    return MAPE_ERR_INVALID_ARG;
  if (!a->B || !a->span || !a->cand_count || !a->flags) return MAPE_ERR_INVALID_ARG;
  if (a->P > 0 && (!a->Z || !a->M || !a->V)) return MAPE_ERR_INVALID_ARG;
  if (a->ldc < a->n || a->ldc % 16 != 0 || a->cand_cap < 0 || (a->cand_cap > 0 && !a->cand))
    return MAPE_ERR_INVALID_ARG;
  if (a->precision != MAPE_PREC_FP32 && a->precision != MAPE_PREC_BF16 && a->precision != MAPE_PREC_BF16X1)
    return MAPE_ERR_INVALID_ARG;
  if (a->P == 0 || a->T == 0) return MAPE_OK;
  cudaStream_t st = mape_detail::as_stream(stream);
  if (a->precision != MAPE_PREC_FP32) {
    if (!mape_detail::extract_tc_supported(a->n, a->d, a->precision)) return MAPE_ERR_SHAPE;
    if (a->workspace_bytes < mape_detail::extract_tc_workspace(a->n, a->d, a->P, a->precision))
      return MAPE_ERR_CAPACITY;
    return mape_detail::extract_tc(a, st);
  }
  if (a->workspace_bytes < mape_detail::extract_fp32_workspace(a->n, a->d, a->P)) return MAPE_ERR_CAPACITY;
  return mape_detail::extract_fp32(a, st);
}
