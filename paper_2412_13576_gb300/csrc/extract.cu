// mape_extract: argument checks and dispatch by precision; library-wide
// helpers (default configuration, version, CUDA error record).
#include "common.cuh"
#include "extract_internal.cuh"

#include <memory>

#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <vector>

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
  if (base == MAPE_PREC_FP32 || base == MAPE_PREC_SPARSE) return extra == 0;
  return (base == MAPE_PREC_BF16 || base == MAPE_PREC_BF16X1) && (extra & ~MAPE_PREC_STREAMED) == 0;
}
}  // namespace

extern "C" size_t mape_extract_workspace_bytes(int32_t n, int32_t d, int32_t P, int32_t precision) {
  if (n <= 0 || d <= 0 || P < 0 || !valid_precision(precision)) return 0;
  const int32_t base = precision & MAPE_PREC_MASK;
  if (base == MAPE_PREC_FP32) return mape_detail::extract_fp32_workspace(n, d, P);
  if (base == MAPE_PREC_SPARSE) return mape_detail::extract_sparse_workspace(n, d, P);
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
  if (base == MAPE_PREC_SPARSE) {
    if (!mape_detail::extract_sparse_supported(a->n, a->d)) return MAPE_ERR_SHAPE;
    if (a->workspace_bytes < mape_detail::extract_sparse_workspace(a->n, a->d, a->P)) return MAPE_ERR_CAPACITY;
    return mape_detail::extract_sparse(a, st);
  }
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

namespace {

int check_item(const mape_extract_args* a) {
  if (a->n <= 0 || a->d <= 0 || a->d > a->n || a->P < 0 || a->T < 0 || a->t0 < 0 || a->period <= 0)
    return MAPE_ERR_INVALID_ARG;
  if (!a->B || !a->span || !a->cand_count || !a->flags) return MAPE_ERR_INVALID_ARG;
  if (a->P > 0 && (!a->Z || !a->M || !a->V)) return MAPE_ERR_INVALID_ARG;
  if (a->ldc < a->n || a->ldc % 16 != 0 || a->cand_cap < 0 || (a->cand_cap > 0 && !a->cand))
    return MAPE_ERR_INVALID_ARG;
  const int32_t base = a->precision & MAPE_PREC_MASK;
  if (!valid_precision(a->precision) || base == MAPE_PREC_FP32 || base == MAPE_PREC_SPARSE)
    return MAPE_ERR_INVALID_ARG;
  if (!mape_detail::extract_stream_supported(a->n, a->d)) return MAPE_ERR_SHAPE;
  if (a->workspace_bytes < mape_extract_workspace_bytes(a->n, a->d, a->P, a->precision)) return MAPE_ERR_CAPACITY;
  return MAPE_OK;
}

}  // namespace

extern "C" size_t mape_extract_batch_workspace_bytes(const mape_extract_args* items, int32_t count) {
  if (!items || count <= 0) return 0;
  std::vector<const mape_extract_args*> ptrs;
  for (int i = 0; i < count; ++i) ptrs.push_back(&items[i]);
  mape_detail::Sizer s;
  s.take<int32_t>((size_t)count);
  s.take<char>(mape_detail::extract_tc_batch_workspace(ptrs.data(), count));
  s.take<char>(mape_detail::extract_stream_batch_workspace(ptrs.data(), count));
  return s.bytes();
}

extern "C" int mape_extract_batch(const mape_extract_args* items, int32_t count, void* workspace,
                                  size_t workspace_bytes, void* stream) {
  using namespace mape_detail;
  if (!items || count < 0) return MAPE_ERR_INVALID_ARG;
  if (count == 0) return MAPE_OK;
  std::vector<const mape_extract_args*> live;
  for (int i = 0; i < count; ++i) {
    const mape_extract_args* a = &items[i];
    int rc = check_item(a);
    if (rc != MAPE_OK) return rc;
    if (a->T != items[0].T || a->t0 != items[0].t0 || a->period != items[0].period ||
        (a->precision & MAPE_PREC_MASK) != (items[0].precision & MAPE_PREC_MASK))
      return MAPE_ERR_INVALID_ARG;
    if (a->P > 0 && a->T > 0) live.push_back(a);
  }
  if (live.empty()) return MAPE_OK;
  if (workspace_bytes < mape_extract_batch_workspace_bytes(items, count)) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  // the per-call precision word carries only the base precision into the kernels
  std::vector<mape_extract_args> calls;
  calls.reserve(live.size());
  for (auto* a : live) {
    calls.push_back(*a);
    calls.back().precision = a->precision & MAPE_PREC_MASK;
  }
  const int nl = (int)calls.size();
  std::vector<const mape_extract_args*> cp;
  for (auto& c : calls) cp.push_back(&c);
  Carver cv(workspace, workspace_bytes);
  int32_t* dflags = cv.take<int32_t>((size_t)count);
  const size_t tws = extract_tc_batch_workspace(cp.data(), nl), sws = extract_stream_batch_workspace(cp.data(), nl);
  char* tw = cv.take<char>(tws);
  char* sw = cv.take<char>(sws);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  std::vector<bool> ids;
  int rc = identity_tops(cp.data(), nl, dflags, st, ids);
  if (rc != MAPE_OK) return rc;
  std::vector<const mape_extract_args*> res_items, st_items;
  std::vector<char> res_ids, st_ids;
  for (int i = 0; i < nl; ++i) {
    const bool forced = (live[i]->precision & MAPE_PREC_STREAMED) != 0;
    if (!forced && extract_tc_fits(cp[i], ids[i])) {
      res_items.push_back(cp[i]);
      res_ids.push_back(ids[i]);
    } else {
      st_items.push_back(cp[i]);
      st_ids.push_back(ids[i]);
    }
  }
  std::vector<bool> rb(res_ids.begin(), res_ids.end()), sb(st_ids.begin(), st_ids.end());
  std::unique_ptr<bool[]> rba(new bool[rb.size() + 1]), sba(new bool[sb.size() + 1]);
  for (size_t i = 0; i < rb.size(); ++i) rba[i] = rb[i];
  for (size_t i = 0; i < sb.size(); ++i) sba[i] = sb[i];
  TcBatch* tplan = nullptr;
  StBatch* splan = nullptr;
  auto cleanup = [&]() {
    if (tplan) extract_tc_batch_free(tplan);
    if (splan) extract_stream_batch_free(splan);
  };
  if (!res_items.empty() &&
      (rc = extract_tc_batch_prepare(res_items.data(), rba.get(), (int)res_items.size(), tw, tws, st, &tplan))) {
    cleanup();
    return rc;
  }
  if (!st_items.empty() &&
      (rc = extract_stream_batch_prepare(st_items.data(), sba.get(), (int)st_items.size(), sw, sws, st, &splan))) {
    cleanup();
    return rc;
  }
  if (st == nullptr) {  // the legacy default stream cannot be captured: launch directly
    if (tplan) rc = extract_tc_batch_enqueue(tplan, st);
    if (rc == MAPE_OK && splan) rc = extract_stream_batch_enqueue(splan, st);
    cleanup();
    return rc;
  }
  // the resident launches and the streamed steps are independent: they run as
  // two branches (a second stream forked from and joined back into `st`), so
  // the SMs one leaves idle take the other's CTAs
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  if (tplan && splan) {
    if (cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess) {
      if (aux) cudaStreamDestroy(aux);
      if (ev_fork) cudaEventDestroy(ev_fork);
      cleanup();
      return MAPE_ERR_CUDA;
    }
  }
  auto enqueue = [&]() -> int {
    int r = MAPE_OK;
    cudaStream_t tst = st;
    if (aux) {
      if (cudaEventRecord(ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(aux, ev_fork, 0) != cudaSuccess)
        return MAPE_ERR_CUDA;
      tst = aux;
    }
    if (tplan && (r = extract_tc_batch_enqueue(tplan, tst)) != MAPE_OK) return r;
    if (splan && (r = extract_stream_batch_enqueue(splan, st)) != MAPE_OK) return r;
    if (aux) {
      if (cudaEventRecord(ev_join, aux) != cudaSuccess || cudaStreamWaitEvent(st, ev_join, 0) != cudaSuccess)
        return MAPE_ERR_CUDA;
    }
    return MAPE_OK;
  };
  // every step of every call in one CUDA graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    record_cuda_error(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
    cleanup();
    return MAPE_ERR_CUDA;
  }
  rc = enqueue();
  e = cudaStreamEndCapture(st, &graph);
  if (rc == MAPE_OK && e != cudaSuccess) {
    record_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    rc = MAPE_ERR_CUDA;
  }
  if (rc == MAPE_OK && (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
    record_cuda_error(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    rc = MAPE_ERR_CUDA;
  }
  if (rc == MAPE_OK && (e = cudaGraphLaunch(exec, st)) != cudaSuccess) {
    record_cuda_error(e, "cudaGraphLaunch", __FILE__, __LINE__);
    rc = MAPE_ERR_CUDA;
  }
  if (rc == MAPE_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) {
    record_cuda_error(e, "batch graph", __FILE__, __LINE__);
    rc = MAPE_ERR_CUDA;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (aux) cudaStreamDestroy(aux);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  cleanup();
  return rc;
}
