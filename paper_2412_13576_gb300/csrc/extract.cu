// mape_extract: argument checks and dispatch by precision; library-wide
// helpers (default configuration, version, CUDA error record).
#include "common.cuh"
#include "extract_internal.cuh"

#include <map>
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

int allow_max_dynamic_smem(const void* func, size_t* limit) {
  int dev = 0, optin = 0;
  MAPE_CUDA_TRY(cudaGetDevice(&dev));
  MAPE_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  MAPE_CUDA_TRY(cudaFuncGetAttributes(&fa, func));
  const int v = optin - (int)fa.sharedSizeBytes;
  MAPE_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
  if (limit) *limit = (size_t)v;
  return MAPE_OK;
}

void record_message(const char* what) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  std::snprintf(g_last_err, sizeof(g_last_err), "%s", what);
}

// ---- launch timing (measurement only) ----------------------------------------

namespace {
std::mutex g_timing_mu;
std::atomic<bool> g_timing_on{false};
struct TimedPair {
  int kind;
  cudaEvent_t start, stop;
};
std::vector<TimedPair> g_timed;
double g_timed_ms[MAPE_TIMED_KINDS] = {};
int64_t g_timed_count[MAPE_TIMED_KINDS] = {};

void drop_pending() {
  for (auto& t : g_timed) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  g_timed.clear();
}
}  // namespace

bool launch_timing_on() { return g_timing_on.load(std::memory_order_relaxed); }

void timed_record(int kind, cudaEvent_t start, cudaEvent_t stop) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  g_timed.push_back({kind, start, stop});
}

}  // namespace mape_detail

extern "C" int mape_launch_timing(int32_t enable) {
  using namespace mape_detail;
  std::lock_guard<std::mutex> lk(g_timing_mu);
  drop_pending();
  for (int k = 0; k < MAPE_TIMED_KINDS; ++k) {
    g_timed_ms[k] = 0.0;
    g_timed_count[k] = 0;
  }
  g_timing_on.store(enable != 0);
  return MAPE_OK;
}

extern "C" int mape_launch_timing_read(double* ms, int64_t* launches) {
  using namespace mape_detail;
  if (!ms || !launches) return MAPE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_timing_mu);
  int rc = MAPE_OK;
  for (auto& t : g_timed) {
    cudaError_t e = cudaEventSynchronize(t.stop);
    float v = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&v, t.start, t.stop);
    if (e != cudaSuccess) {
      record_cuda_error(e, "mape_launch_timing_read", __FILE__, __LINE__);
      rc = MAPE_ERR_CUDA;
      continue;
    }
    if (t.kind >= 0 && t.kind < MAPE_TIMED_KINDS) {
      g_timed_ms[t.kind] += v;
      g_timed_count[t.kind] += 1;
    }
  }
  drop_pending();
  for (int k = 0; k < MAPE_TIMED_KINDS; ++k) {
    ms[k] = g_timed_ms[k];
    launches[k] = g_timed_count[k];
  }
  return rc;
}

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
  if (base == MAPE_PREC_FP8)  // streamed only; the tile widths may be autotuned
    return (extra & ~(MAPE_PREC_STREAMED | MAPE_PREC_AUTOTUNE)) == 0 &&
           !((extra & MAPE_PREC_STREAMED) && (extra & MAPE_PREC_AUTOTUNE));
  if ((extra & MAPE_PREC_STREAMED) && (extra & MAPE_PREC_AUTOTUNE)) return false;
  if ((extra & MAPE_PREC_SPARSE_FWD) && ((extra & MAPE_PREC_AUTOTUNE) || base != MAPE_PREC_BF16)) return false;
  return (base == MAPE_PREC_BF16 || base == MAPE_PREC_BF16X1) &&
         (extra & ~(MAPE_PREC_STREAMED | MAPE_PREC_AUTOTUNE | MAPE_PREC_SPARSE_FWD)) == 0;
}

// ---- autotuning of the implementation (BF16) and the streamed tile widths (BF16, FP8) ----

struct TuneKey {
  int32_t n, d, pb, base;
  bool operator<(const TuneKey& o) const {
    if (n != o.n) return n < o.n;
    if (d != o.d) return d < o.d;
    if (pb != o.pb) return pb < o.pb;
    return base < o.base;
  }
};

std::mutex g_tune_mu;
std::map<TuneKey, mape_tune_info> g_tuned;

int32_t p_bucket(int32_t P) {
  int32_t b = 1;
  while (b < P && b < (1 << 30)) b <<= 1;
  return b;
}

constexpr int kProbeSteps = 6;

// scratch the probes need beyond the implementation's own workspace
size_t tune_scratch_bytes(int32_t n, int32_t d, int32_t P) {
  mape_detail::Sizer s;
  for (int k = 0; k < 3; ++k) s.take<float>((size_t)P * d);
  s.take<int8_t>((size_t)(P + 16) * mape_detail::align_up((size_t)n, 16));
  s.take<unsigned long long>(1);
  s.take<int32_t>(1);
  return s.bytes();
}

int run_choice(const mape_extract_args* a, cudaStream_t st, const mape_tune_info& c) {
  if (c.path == 0) return mape_detail::extract_tc(a, st);
  return mape_detail::extract_stream_widths(a, st, c.wF, c.wG,
                                            c.path == 2 ? mape_detail::kFwdSparse : mape_detail::kFwdDense);
}

}  // namespace

// Times kProbeSteps steps of every candidate from the call's state on scratch
// copies (the call's own arrays are not touched) and caches the fastest.
static int autotune(const mape_extract_args* a, cudaStream_t st, size_t impl_bytes, mape_tune_info& out) {
  using namespace mape_detail;
  const int n = a->n, d = a->d, P = a->P;
  const size_t ldc = align_up((size_t)n, 16);
  Carver cv(static_cast<char*>(a->workspace) + impl_bytes, a->workspace_bytes - impl_bytes);
  float* Zs = cv.take<float>((size_t)P * d);
  float* Ms = cv.take<float>((size_t)P * d);
  float* Vs = cv.take<float>((size_t)P * d);
  int8_t* cs = cv.take<int8_t>((size_t)(P + 16) * ldc);
  unsigned long long* cnt = cv.take<unsigned long long>(1);
  int32_t* fl = cv.take<int32_t>(1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  std::vector<mape_tune_info> cands;
  mape_tune_info c{};
  const bool f8 = (a->precision & MAPE_PREC_MASK) == MAPE_PREC_FP8;  // streamed dense forward only
  if (!f8 && extract_tc_supported(n, d, a->precision & MAPE_PREC_MASK)) {
    c.path = 0;
    cands.push_back(c);
  }
  for (int wf : {64, 128, 256})
    for (int wg : {64, 128, 256}) {
      c.path = 1; c.wF = wf; c.wG = wg;
      cands.push_back(c);
    }
  // the sparse forward (refused with SHAPE, and so skipped, when B does not qualify)
  for (int wg : {64, 128, 256}) {
    if (f8) break;
    c.path = 2; c.wF = 256; c.wG = wg;
    cands.push_back(c);
  }
  cudaEvent_t e0, e1;
  MAPE_CUDA_TRY(cudaEventCreate(&e0));
  MAPE_CUDA_TRY(cudaEventCreate(&e1));
  mape_extract_args b = *a;
  b.precision = a->precision & MAPE_PREC_MASK;
  b.Z = Zs; b.M = Ms; b.V = Vs;
  b.cand = cs; b.ldc = (int32_t)ldc; b.cand_cap = P + 16; b.cand_count = cnt; b.flags = fl;
  b.dbg_phi = nullptr; b.dbg_grad = nullptr;
  b.T = a->T < kProbeSteps ? a->T : kProbeSteps;
  b.workspace_bytes = impl_bytes;
  float best = 1e30f;
  int nc = 0;
  out = mape_tune_info{};
  for (const auto& k : cands) {
    int rc = MAPE_OK;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && rc == MAPE_OK; ++rep) {  // the first run loads the kernels
      MAPE_CUDA_TRY(cudaMemcpyAsync(Zs, a->Z, sizeof(float) * (size_t)P * d, cudaMemcpyDeviceToDevice, st));
      MAPE_CUDA_TRY(cudaMemcpyAsync(Ms, a->M, sizeof(float) * (size_t)P * d, cudaMemcpyDeviceToDevice, st));
      MAPE_CUDA_TRY(cudaMemcpyAsync(Vs, a->V, sizeof(float) * (size_t)P * d, cudaMemcpyDeviceToDevice, st));
      MAPE_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
      MAPE_CUDA_TRY(cudaMemsetAsync(fl, 0, sizeof(int32_t), st));
      MAPE_CUDA_TRY(cudaEventRecord(e0, st));
      rc = run_choice(&b, st, k);
      MAPE_CUDA_TRY(cudaEventRecord(e1, st));
      MAPE_CUDA_TRY(cudaEventSynchronize(e1));
      MAPE_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    }
    if (rc != MAPE_OK) continue;  // e.g. a general B the resident tile cannot take
    if (nc < 16) {
      out.cand_path[nc] = k.path; out.cand_wF[nc] = k.wF; out.cand_wG[nc] = k.wG; out.probe_ms[nc] = ms;
      ++nc;
    }
    if (ms < best) {
      best = ms;
      out.path = k.path; out.wF = k.wF; out.wG = k.wG;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  out.candidates = nc;
  out.probe_steps = b.T;
  return nc > 0 ? MAPE_OK : MAPE_ERR_SHAPE;
}

extern "C" int mape_autotune_lookup(int32_t n, int32_t d, int32_t P, int32_t precision, mape_tune_info* out) {
  if (!out) return MAPE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(TuneKey{n, d, p_bucket(P), precision & MAPE_PREC_MASK});
  if (it == g_tuned.end()) return MAPE_ERR_STATE;
  *out = it->second;
  return MAPE_OK;
}

extern "C" void mape_autotune_clear(void) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
  }
  mape_detail::augment_tune_clear();
}

extern "C" size_t mape_extract_workspace_bytes(int32_t n, int32_t d, int32_t P, int32_t precision) {
  if (n <= 0 || d <= 0 || P < 0 || !valid_precision(precision)) return 0;
  if (precision & MAPE_PREC_AUTOTUNE) {
    const size_t w = mape_extract_workspace_bytes(n, d, P, precision & ~MAPE_PREC_AUTOTUNE);
    return w ? mape_detail::align_up(w, 256) + tune_scratch_bytes(n, d, P) : 0;
  }
  const int32_t base = precision & MAPE_PREC_MASK;
  if (base == MAPE_PREC_FP32) return mape_detail::extract_fp32_workspace(n, d, P);
  if (base == MAPE_PREC_SPARSE) return mape_detail::extract_sparse_workspace(n, d, P);
  if (base == MAPE_PREC_FP8) return mape_detail::extract_stream_workspace(n, d, P);
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
    if (base == MAPE_PREC_FP8 && !(a->precision & MAPE_PREC_AUTOTUNE))
      return mape_detail::extract_stream(&b, st, mape_detail::kFwdDense);
    if (a->precision & MAPE_PREC_AUTOTUNE) {
      const size_t impl = mape_detail::align_up(mape_extract_workspace_bytes(a->n, a->d, a->P, base), 256);
      const TuneKey key{a->n, a->d, p_bucket(a->P), base};
      mape_tune_info choice{};
      bool have = false;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) { choice = it->second; have = true; }
      }
      if (!have) {
        int rc = autotune(a, st, impl, choice);
        if (rc != MAPE_OK) return rc;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = choice;
      }
      b.workspace_bytes = impl;
      return run_choice(&b, st, choice);
    }
    if (a->precision & MAPE_PREC_SPARSE_FWD) return mape_detail::extract_stream(&b, st, mape_detail::kFwdSparse);
    if (!(a->precision & MAPE_PREC_STREAMED) && mape_detail::extract_tc_supported(a->n, a->d, base)) {
      const int rc = mape_detail::extract_tc(&b, st);
      if (rc != MAPE_ERR_SHAPE) return rc;  // SHAPE: a general B that only the streamed path takes
    }
    return mape_detail::extract_stream(&b, st, mape_detail::kFwdDense);
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
