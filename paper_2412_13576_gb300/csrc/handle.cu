// The instance handle: create_instance / extract_directions / augment /
// poll / wait / get_* / destroy.  Host arrays are copied in the calling
// thread; device buffers are allocated there too (so an allocator hook runs on
// the caller's thread), and the stage pipeline then runs on one worker thread
// per handle, which only launches kernels and synchronises its stream.
//
// Extraction memory is bounded: candidates go to a buffer of `cap` rows laid
// out as [distinct rows so far | rows of the current chunk]; each chunk runs
// at most (cap - distinct) / P collection steps (steps whose number is a
// multiple of the period), which append at most one row per start each, so the
// buffer cannot overflow; after each chunk mape_dedup merges
// the buffer into the other buffer of the pair and the two swap.
#include "common.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

namespace {

std::mutex g_alloc_mu;
mape_alloc_fn g_alloc = nullptr;
mape_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

// Default allocation: a stream-ordered memory pool per device owned by the
// library, whose release threshold keeps freed memory reserved, so that
// handles created one after another (a request per handle) reuse it instead
// of mapping new pages; mape_trim_memory hands it back.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};

cudaMemPool_t library_pool(int dev) {
  if (dev < 0 || dev >= kMaxPoolDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}

__global__ void basis_check_kernel(const int32_t* __restrict__ A, const int32_t* __restrict__ B, int m, int n,
                                   int d, int32_t* __restrict__ bad) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (j >= d) return;
  long long acc = 0;
  for (int i = 0; i < n; ++i) acc += (long long)A[(int64_t)r * n + i] * B[(int64_t)i * d + j];
  if (acc != 0) atomicOr(bad, 1);
}

__global__ void feasible_check_kernel(const int32_t* __restrict__ A, const int64_t* __restrict__ b,
                                      const int32_t* __restrict__ X, int m, int n, int S, int32_t* __restrict__ bad) {
  int s = blockIdx.x;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    long long acc = 0;
    for (int i = 0; i < n; ++i) acc += (long long)A[(int64_t)r * n + i] * X[(int64_t)s * n + i];
    if (acc != b[r]) atomicOr(bad, 1);
  }
}

__global__ void i8_to_i32_kernel(const int8_t* __restrict__ G, int64_t K, int n, int ldg, int32_t* __restrict__ out) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= K * n) return;
  int64_t k = t / n;
  int i = (int)(t % n);
  out[t] = G[k * ldg + i];
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct mape_instance {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n = 0, m = 0, d = 0, ldg = 0;
  mape_config cfg{};
  bool has_w = false;
  int nnz = 0;

  // device buffers owned by the handle, with their sizes (for the free hook)
  std::vector<std::pair<void*, size_t>> owned;
  int32_t *dA = nullptr, *dB = nullptr, *dl = nullptr, *du = nullptr, *dspan = nullptr;
  int64_t* db = nullptr;
  int32_t *dc = nullptr, *dw = nullptr, *dqr = nullptr, *dqc = nullptr, *dqv = nullptr;
  float* dWproj = nullptr;  // B (B^T B)^{-1}, computed once per instance for the start projection
  char* dWprojWork = nullptr;
  bool proj_ready = false;  // dWproj holds W (formed at the first call with G0 starts)

  // extraction job buffers (replaced per extract call)
  std::vector<std::pair<void*, size_t>> job_bufs;
  int P = 0;
  float *dZ = nullptr, *dM = nullptr, *dV = nullptr, *dG0 = nullptr;
  int8_t *dBuf0 = nullptr, *dBuf1 = nullptr;
  int64_t cap = 0;
  uint8_t *dOk = nullptr, *dKeep = nullptr;
  int64_t *da = nullptr, *dq4 = nullptr;
  void* dWork = nullptr;
  size_t work_bytes = 0;
  unsigned long long* dCount = nullptr;
  int32_t* dFlags = nullptr;
  int8_t* dirs = nullptr;  // current direction set (the candidate buffer free after the last merge)
  int64_t K = 0;

  // augmentation buffers
  std::vector<std::pair<void*, size_t>> aug_bufs;
  int S = 0;
  int32_t* dX = nullptr;
  int64_t* dF = nullptr;
  void* dAugWork = nullptr;
  size_t aug_work_bytes = 0;

  std::mutex mu;
  std::condition_variable cv;
  mape_status st{};
  bool busy = false;
  std::thread worker;
  std::atomic<bool> cancel{false};
  std::vector<int32_t> best_x;
  int64_t best_f = 0;

  void* alloc(size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    {
      std::lock_guard<std::mutex> lk(g_alloc_mu);
      if (g_alloc) {
        p = g_alloc(bytes, stream, g_alloc_ctx);
        return p;
      }
    }
    cudaMemPool_t pool = library_pool(dev);
    if (!pool || cudaMallocFromPoolAsync(&p, bytes, pool, stream) != cudaSuccess) return nullptr;
    return p;
  }
  void release(void* p, size_t bytes) {
    if (!p) return;
    {
      std::lock_guard<std::mutex> lk(g_alloc_mu);
      if (g_free) {
        g_free(p, bytes, stream, g_alloc_ctx);
        return;
      }
    }
    cudaFreeAsync(p, stream);
  }
  template <typename T>
  T* take(std::vector<std::pair<void*, size_t>>& list, size_t count) {
    size_t bytes = std::max<size_t>(16, count * sizeof(T));
    void* p = alloc(bytes);
    if (p) list.push_back({p, bytes});
    return static_cast<T*>(p);
  }
  void release_all(std::vector<std::pair<void*, size_t>>& list) {
    for (auto& pr : list) release(pr.first, pr.second);
    list.clear();
  }
  void join() {
    if (worker.joinable()) worker.join();
  }
  void set_phase(int ph) {
    std::lock_guard<std::mutex> lk(mu);
    st.phase = ph;
  }
  void finish(int err) {
    std::lock_guard<std::mutex> lk(mu);
    st.error = err;
    st.phase = err == MAPE_OK ? MAPE_PHASE_DONE : MAPE_PHASE_ERROR;
    busy = false;
    cv.notify_all();
  }

  // extraction progress (the parts of run_extract, also driven by a batch)
  double ex_start = 0;
  int64_t ex_U = 0, ex_total = 0;
  int ex_done = 0;
  int8_t *ex_cur = nullptr, *ex_other = nullptr;
  int extract_begin();
  int extract_chunk_steps(int* chunk) const;
  int extract_chunk_args(int chunk, mape_extract_args* a);
  int extract_chunk_done(int chunk);
  int chunk_candidates(cudaStream_t s, int64_t* cnt);
  void chunk_merged(int chunk, int64_t cnt, int64_t K_new);
  int extract_filter();
  int filter_done(int64_t fails, int64_t Kk, double t_ext, double t_fil);

  int run_extract();
  // Algorithm 1 (the parts of run_augment, also driven by a batch)
  void augment_args(mape_augment_args* a);
  int augment_end(int64_t it1, int64_t it2, double t0, double t1);
  int run_augment(int64_t max_iters);
};

#define H_TRY(expr)                 \
  do {                              \
    int _rc = (expr);               \
    if (_rc != MAPE_OK) return _rc; \
  } while (0)

// Algorithm 2 in three parts, so that a batch of handles can run the
// extraction steps of all of them as one mape_extract_batch call per chunk:
// begin (starts, Adam moments), chunks (each: the steps, then the merge of the
// chunk's candidates into the distinct set), filter (kernel test, minimality,
// coefficients).
int mape_instance::extract_begin() {
  ex_start = now_ms();
  set_phase(MAPE_PHASE_EXTRACTING);
  if (dG0) H_TRY(mape_project_apply(dWproj, n, d, dG0, P, dZ, stream));
  MAPE_CUDA_TRY(cudaMemsetAsync(dM, 0, sizeof(float) * (size_t)P * d, stream));
  MAPE_CUDA_TRY(cudaMemsetAsync(dV, 0, sizeof(float) * (size_t)P * d, stream));
  ex_U = 0;
  ex_total = 0;
  ex_done = 0;
  ex_cur = dBuf0;
  ex_other = dBuf1;
  return MAPE_OK;
}

// The longest chunk from ex_done: it may hold as many collections (steps
// whose number is a multiple of the period) as there is room for one row per
// start each, and ends just before the first collection that would not fit.
int mape_instance::extract_chunk_steps(int* chunk) const {
  const int64_t room = cap - ex_U;
  const int64_t fits = room / P;
  const int64_t period = cfg.period;
  const int64_t steps = (ex_done / period + fits + 1) * period - 1 - ex_done;
  if (steps < 1) return MAPE_ERR_CAPACITY;
  *chunk = (int)std::min<int64_t>(steps, cfg.T - ex_done);
  return MAPE_OK;
}

// The arguments of the next `chunk` steps (counter and flags cleared).
int mape_instance::extract_chunk_args(int chunk, mape_extract_args* a) {
  MAPE_CUDA_TRY(cudaMemsetAsync(dCount, 0, sizeof(unsigned long long), stream));
  MAPE_CUDA_TRY(cudaMemsetAsync(dFlags, 0, sizeof(int32_t), stream));
  *a = mape_extract_args{};
  a->n = n; a->d = d; a->P = P; a->B = dB; a->span = dspan; a->Z = dZ; a->M = dM; a->V = dV;
  a->t0 = ex_done; a->T = chunk; a->period = cfg.period; a->precision = cfg.precision;
  a->lambda1 = cfg.lambda1; a->lambda2 = cfg.lambda2; a->lr = cfg.lr; a->beta1 = cfg.beta1;
  a->beta2 = cfg.beta2; a->eps = cfg.eps;
  a->cand = ex_cur + ex_U * ldg; a->ldc = ldg; a->cand_cap = cap - ex_U; a->cand_count = dCount; a->flags = dFlags;
  a->workspace = dWork; a->workspace_bytes = work_bytes;
  return MAPE_OK;
}

// After the steps of a chunk: its candidates are merged into the distinct set.
int mape_instance::extract_chunk_done(int chunk) {
  int64_t cnt = 0;
  H_TRY(chunk_candidates(stream, &cnt));
  int64_t K_new = 0;
  H_TRY(mape_dedup(ex_cur, ex_U + cnt, n, ldg, ex_other, cap, &K_new, dWork, work_bytes, stream));
  chunk_merged(chunk, cnt, K_new);
  return MAPE_OK;
}

// The candidates the chunk appended (read on stream s).
int mape_instance::chunk_candidates(cudaStream_t s, int64_t* cnt) {
  unsigned long long c = 0;
  int32_t flags = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&c, dCount, sizeof(c), cudaMemcpyDeviceToHost, s));
  MAPE_CUDA_TRY(cudaMemcpyAsync(&flags, dFlags, sizeof(flags), cudaMemcpyDeviceToHost, s));
  MAPE_CUDA_TRY(cudaStreamSynchronize(s));
  if (flags & 1) return MAPE_ERR_CAPACITY;
  *cnt = (int64_t)c;
  return MAPE_OK;
}

// The merge of the chunk's candidates left K_new distinct rows in ex_other.
void mape_instance::chunk_merged(int chunk, int64_t cnt, int64_t K_new) {
  ex_total += cnt;
  ex_U = K_new;
  std::swap(ex_cur, ex_other);
  ex_done += chunk;
  std::lock_guard<std::mutex> lk(mu);
  st.candidates = ex_total;
  st.unique = ex_U;
}

int mape_instance::extract_filter() {
  cudaStream_t s = stream;
  double t_ext = now_ms();
  set_phase(MAPE_PHASE_FILTERING);
  int64_t fails = 0;
  H_TRY(mape_kernel_test(dA, m, n, ex_cur, ex_U, ldg, dOk, &fails, dWork, work_bytes, s));
  int64_t Kk = 0;
  // the kept rows go to the buffer of the pair that the last merge left free
  H_TRY(mape_minimal_filter(ex_cur, ex_U, n, ldg, dOk, dKeep, ex_other, &Kk, dWork, work_bytes, s));
  H_TRY(mape_direction_coeffs(dqr, dqc, dqv, nnz, has_w ? dw : nullptr, n, ex_other, Kk, ldg, da, dq4, s));
  MAPE_CUDA_TRY(cudaStreamSynchronize(s));
  return filter_done(fails, Kk, t_ext, now_ms());
}

// The direction set after the filter stages (kept rows in ex_other).
int mape_instance::filter_done(int64_t fails, int64_t Kk, double t_ext, double t_fil) {
  dirs = ex_other;
  K = Kk;
  std::lock_guard<std::mutex> lk(mu);
  st.kernel_failures = fails;
  st.directions = Kk;
  st.extract_ms = t_ext - ex_start;
  st.filter_ms = t_fil - t_ext;
  return fails ? MAPE_ERR_KERNEL_TEST : MAPE_OK;
}

int mape_instance::run_extract() {
  H_TRY(extract_begin());
  while (ex_done < cfg.T) {
    if (cancel.load()) return MAPE_ERR_CANCELLED;
    int chunk = 0;
    H_TRY(extract_chunk_steps(&chunk));
    mape_extract_args a;
    H_TRY(extract_chunk_args(chunk, &a));
    H_TRY(mape_extract(&a, stream));
    H_TRY(extract_chunk_done(chunk));
  }
  return extract_filter();
}

void mape_instance::augment_args(mape_augment_args* a) {
  *a = mape_augment_args{};
  a->n = n; a->S = S; a->K = K; a->G = dirs; a->ldg = ldg; a->a = da; a->q4 = dq4;
  a->q_row = dqr; a->q_col = dqc; a->q_val = dqv; a->nnz = nnz; a->c = dc; a->w = has_w ? dw : nullptr;
  a->l = dl; a->u = du; a->X = dX; a->fval = dF;
  a->workspace = dAugWork; a->workspace_bytes = aug_work_bytes;
}

int mape_instance::run_augment(int64_t max_iters) {
  set_phase(MAPE_PHASE_AUGMENTING);
  double t0 = now_ms();
  mape_augment_args a;
  augment_args(&a);
  // the first iteration alone: time to the first improving direction
  a.max_iters = std::min<int64_t>(1, max_iters);
  int64_t it1 = 0, it2 = 0;
  H_TRY(mape_augment_run(&a, &it1, stream));
  double t1 = now_ms();
  if (max_iters > 1 && !cancel.load()) {
    a.max_iters = max_iters - 1;
    H_TRY(mape_augment_run(&a, &it2, stream));
  }
  return augment_end(it1, it2, t0, t1);
}

// The best start's point and value, and the status of the run.
int mape_instance::augment_end(int64_t it1, int64_t it2, double t0, double t1) {
  cudaStream_t s = stream;
  std::vector<int64_t> f(S);
  MAPE_CUDA_TRY(cudaMemcpyAsync(f.data(), dF, sizeof(int64_t) * S, cudaMemcpyDeviceToHost, s));
  MAPE_CUDA_TRY(cudaStreamSynchronize(s));
  int bi = (int)(std::min_element(f.begin(), f.end()) - f.begin());
  best_x.assign(n, 0);
  MAPE_CUDA_TRY(cudaMemcpyAsync(best_x.data(), dX + (int64_t)bi * n, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  MAPE_CUDA_TRY(cudaStreamSynchronize(s));
  best_f = f[bi];
  double t2 = now_ms();
  std::lock_guard<std::mutex> lk(mu);
  st.aug_iters = it1 + it2;
  st.best_f = best_f;
  st.best_start = bi;
  st.augment_ms = t2 - t0;
  st.first_improve_ms = t1 - t0;
  return MAPE_OK;
}

namespace {

int upload(mape_instance* h, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return MAPE_OK;
  MAPE_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->stream));
  return MAPE_OK;
}

int set_objective(mape_instance* h, const mape_problem* f) {
  const int n = h->n;
  if (!f->Q || !f->c) return MAPE_ERR_INVALID_ARG;
  // Q must be symmetric: compared in 64 x 64 blocks, so that the transposed
  // reads stay within a few cache lines per row of a block
  constexpr int kSymBlock = 64;
  for (int i0 = 0; i0 < n; i0 += kSymBlock)
    for (int j0 = i0; j0 < n; j0 += kSymBlock)
      for (int i = i0; i < std::min(i0 + kSymBlock, n); ++i)
        for (int j = std::max(j0, i + 1); j < std::min(j0 + kSymBlock, n); ++j)
          if (f->Q[(int64_t)i * n + j] != f->Q[(int64_t)j * n + i]) return MAPE_ERR_INVALID_ARG;
  std::vector<int32_t> qr, qc, qv;  // the upper triangle in COO form, row by row
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) {
      const int32_t v = f->Q[(int64_t)i * n + j];
      if (v != 0) { qr.push_back(i); qc.push_back(j); qv.push_back(v); }
    }
  if (f->w)
    for (int i = 0; i < n; ++i)
      if (f->w[i] < 0) return MAPE_ERR_INVALID_ARG;
  h->nnz = (int)qv.size();
  h->dqr = h->take<int32_t>(h->owned, qr.size());
  h->dqc = h->take<int32_t>(h->owned, qc.size());
  h->dqv = h->take<int32_t>(h->owned, qv.size());
  h->dc = h->take<int32_t>(h->owned, n);
  h->dw = h->take<int32_t>(h->owned, n);
  if (!h->dqr || !h->dqc || !h->dqv || !h->dc || !h->dw) return MAPE_ERR_OOM;
  H_TRY(upload(h, h->dqr, qr.data(), qr.size() * 4));
  H_TRY(upload(h, h->dqc, qc.data(), qc.size() * 4));
  H_TRY(upload(h, h->dqv, qv.data(), qv.size() * 4));
  H_TRY(upload(h, h->dc, f->c, (size_t)n * 4));
  h->has_w = f->w != nullptr;
  if (f->w) H_TRY(upload(h, h->dw, f->w, (size_t)n * 4));
  MAPE_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return MAPE_OK;
}

bool idle(mape_instance* h) {
  std::lock_guard<std::mutex> lk(h->mu);
  return !h->busy;
}

}  // namespace

extern "C" int mape_set_allocator(mape_alloc_fn a, mape_free_fn f, void* ctx) {
  if ((a == nullptr) != (f == nullptr)) return MAPE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = a;
  g_free = f;
  g_alloc_ctx = ctx;
  return MAPE_OK;
}

extern "C" int mape_trim_memory(void) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxPoolDevices) return MAPE_ERR_CUDA;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    pool = g_pool[dev];
  }
  if (!pool) return MAPE_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
  if (e != cudaSuccess) {
    mape_detail::record_cuda_error(e, "mape_trim_memory", __FILE__, __LINE__);
    return MAPE_ERR_CUDA;
  }
  return MAPE_OK;
}

extern "C" int mape_create_instance(const int32_t* A, const int64_t* b, const int32_t* l, const int32_t* u,
                                    const mape_problem* f, const int32_t* B, const mape_config* cfg,
                                    void* stream, mape_handle* out) {
  if (!out) return MAPE_ERR_INVALID_ARG;
  *out = nullptr;
  if (!A || !b || !l || !u || !f || !B || !cfg) return MAPE_ERR_INVALID_ARG;
  const int n = f->n, m = f->m;
  if (n <= 0 || m <= 0 || m >= n) return MAPE_ERR_SHAPE;
  if (n > 4096) return MAPE_ERR_SHAPE;
  if (cfg->T < 0 || cfg->period <= 0 || cfg->lr <= 0.f || cfg->max_aug_iters < 0) return MAPE_ERR_INVALID_ARG;
  if (mape_extract_workspace_bytes(n, n - m, 1, cfg->precision) == 0) return MAPE_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (u[i] < l[i] || (int64_t)u[i] - l[i] > 127) return MAPE_ERR_BOUNDS;
  auto* h = new mape_instance();
  h->n = n;
  h->m = m;
  h->d = n - m;
  h->ldg = (int)mape_detail::align_up((size_t)n, 16);
  h->cfg = *cfg;
  if (cudaGetDevice(&h->dev) != cudaSuccess) { delete h; return MAPE_ERR_CUDA; }
  if (stream) {
    h->stream = mape_detail::as_stream(stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) { delete h; return MAPE_ERR_CUDA; }
    h->own_stream = true;
  }
  auto fail = [&](int rc) {
    mape_destroy(h);
    return rc;
  };
  const int d = h->d;
  h->dA = h->take<int32_t>(h->owned, (size_t)m * n);
  h->dB = h->take<int32_t>(h->owned, (size_t)n * d);
  h->db = h->take<int64_t>(h->owned, (size_t)m);
  h->dl = h->take<int32_t>(h->owned, n);
  h->du = h->take<int32_t>(h->owned, n);
  h->dspan = h->take<int32_t>(h->owned, n);
  int32_t* dbad = h->take<int32_t>(h->owned, 1);
  if (!h->dA || !h->dB || !h->db || !h->dl || !h->du || !h->dspan || !dbad) return fail(MAPE_ERR_OOM);
  std::vector<int32_t> span(n);
  for (int i = 0; i < n; ++i) span[i] = u[i] - l[i];
  int rc;
  if ((rc = upload(h, h->dA, A, (size_t)m * n * 4)) || (rc = upload(h, h->dB, B, (size_t)n * d * 4)) ||
      (rc = upload(h, h->db, b, (size_t)m * 8)) || (rc = upload(h, h->dl, l, (size_t)n * 4)) ||
      (rc = upload(h, h->du, u, (size_t)n * 4)) || (rc = upload(h, h->dspan, span.data(), (size_t)n * 4)))
    return fail(rc);
  if (cudaMemsetAsync(dbad, 0, 4, h->stream) != cudaSuccess) return fail(MAPE_ERR_CUDA);
  mape_detail::launch(basis_check_kernel, dim3((unsigned)mape_detail::ceil_div(d, 128), (unsigned)m), 128, 0, h->stream, 
      h->dA, h->dB, m, n, d, dbad);
  int32_t bad = 0;
  if (cudaMemcpyAsync(&bad, dbad, 4, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return fail(MAPE_ERR_CUDA);
  if (bad) return fail(MAPE_ERR_NOT_KERNEL_BASIS);
  if ((rc = set_objective(h, f))) return fail(rc);
  h->st.phase = MAPE_PHASE_IDLE;
  *out = h;
  return MAPE_OK;
}

namespace {

// W = B (B^T B)^{-1} for the projection of G0 starts (a2), formed once per
// instance, at its first job with G0 starts: a job given z0 directly never
// needs it.  Synchronous on the handle's stream; the handle must be idle.
int prepare_projection(mape_handle h) {
  if (h->proj_ready) return MAPE_OK;
  const size_t pb = mape_project_prepare_workspace_bytes(h->n, h->d);
  if (!h->dWproj) h->dWproj = h->take<float>(h->owned, (size_t)h->n * h->d);
  if (!h->dWprojWork) h->dWprojWork = h->take<char>(h->owned, pb);
  if (!h->dWproj || !h->dWprojWork) return MAPE_ERR_OOM;
  H_TRY(mape_project_prepare(h->dB, h->n, h->d, h->dWproj, h->dWprojWork, pb, h->stream));
  h->proj_ready = true;
  return MAPE_OK;
}

// The buffers of an extraction job of P starts and the upload of its starts;
// the handle must be idle.
int prepare_job(mape_handle h, int32_t P, const float* Z0, const float* G0) {
  using namespace mape_detail;
  if (P <= 0 || (Z0 == nullptr) == (G0 == nullptr)) return MAPE_ERR_INVALID_ARG;
  if (!idle(h)) return MAPE_ERR_STATE;
  h->join();
  if (G0) H_TRY(prepare_projection(h));
  if (mape_extract_workspace_bytes(h->n, h->d, P, h->cfg.precision) == 0) return MAPE_ERR_SHAPE;
  h->release_all(h->job_bufs);
  h->K = 0;
  h->dirs = nullptr;
  const int n = h->n, d = h->d, ldg = h->ldg;
  const int64_t T = h->cfg.T;
  int64_t cap = h->cfg.cand_capacity > 0 ? h->cfg.cand_capacity
                                         : default_cand_capacity(P, T / h->cfg.period, ldg);
  cap = std::max<int64_t>(cap, (int64_t)P + 1);
  h->cap = cap;
  h->P = P;
  h->dZ = h->take<float>(h->job_bufs, (size_t)P * d);
  h->dM = h->take<float>(h->job_bufs, (size_t)P * d);
  h->dV = h->take<float>(h->job_bufs, (size_t)P * d);
  h->dG0 = G0 ? h->take<float>(h->job_bufs, (size_t)P * n) : nullptr;
  h->dBuf0 = h->take<int8_t>(h->job_bufs, (size_t)cap * ldg);
  h->dBuf1 = h->take<int8_t>(h->job_bufs, (size_t)cap * ldg);
  h->dOk = h->take<uint8_t>(h->job_bufs, (size_t)cap);
  h->dKeep = h->take<uint8_t>(h->job_bufs, (size_t)cap);
  h->da = h->take<int64_t>(h->job_bufs, (size_t)cap);
  h->dq4 = h->take<int64_t>(h->job_bufs, (size_t)cap);
  h->dCount = h->take<unsigned long long>(h->job_bufs, 1);
  h->dFlags = h->take<int32_t>(h->job_bufs, 1);
  size_t w = 0;
  w = std::max(w, mape_extract_workspace_bytes(n, d, P, h->cfg.precision));
  w = std::max(w, mape_dedup_workspace_bytes(cap, ldg));
  w = std::max(w, mape_kernel_test_workspace_bytes(h->m, n));
  w = std::max(w, mape_minimal_workspace_bytes(cap, n));
  h->work_bytes = w;
  h->dWork = h->take<char>(h->job_bufs, w);
  if (!h->dZ || !h->dM || !h->dV || (G0 && !h->dG0) || !h->dBuf0 || !h->dBuf1 || !h->dOk ||
      !h->dKeep || !h->da || !h->dq4 || !h->dCount || !h->dFlags || !h->dWork)
    return MAPE_ERR_OOM;
  int rc = G0 ? upload(h, h->dG0, G0, sizeof(float) * (size_t)P * n) : upload(h, h->dZ, Z0, sizeof(float) * (size_t)P * d);
  if (rc) return rc;
  MAPE_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return MAPE_OK;
}

void mark_busy(mape_handle h) {
  std::lock_guard<std::mutex> lk(h->mu);
  h->busy = true;
  h->st = mape_status{};
  h->st.phase = MAPE_PHASE_EXTRACTING;
  h->cancel.store(false);
}

// A batch of extraction jobs: the first handle's worker runs the steps of
// every handle, chunk by chunk, as one mape_extract_batch call each; the
// other workers wait for it and then filter their own sets in parallel.
struct ExtractBatch {
  std::vector<mape_handle> hs;
  std::mutex mu;
  std::condition_variable cv;
  bool done = false;
  int rc = MAPE_OK;
  std::vector<int> rcs;  // per handle
};

int run_batch_steps(ExtractBatch& b) {
  const int count = (int)b.hs.size();
  for (int i = 0; i < count; ++i) {
    mape_handle h = b.hs[i];
    if (h->dev != b.hs[0]->dev) return MAPE_ERR_INVALID_ARG;
    H_TRY(h->extract_begin());
  }
  for (auto h : b.hs) MAPE_CUDA_TRY(cudaStreamSynchronize(h->stream));
  mape_handle h0 = b.hs[0];
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* dws = nullptr;  // the dedup batch's tables
  size_t dws_bytes = 0;
  std::vector<mape_extract_args> items((size_t)count);
  while (h0->ex_done < h0->cfg.T) {
    int chunk = h0->cfg.T - h0->ex_done;
    for (auto h : b.hs) {
      if (h->cancel.load()) return MAPE_ERR_CANCELLED;
      int c = 0;
      H_TRY(h->extract_chunk_steps(&c));
      chunk = std::min(chunk, c);
    }
    for (int i = 0; i < count; ++i) H_TRY(b.hs[i]->extract_chunk_args(chunk, &items[(size_t)i]));
    for (auto h : b.hs) MAPE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    const size_t need = mape_extract_batch_workspace_bytes(items.data(), count);
    if (need > ws_bytes) {
      ws = h0->take<char>(h0->job_bufs, need);
      if (!ws) return MAPE_ERR_OOM;
      ws_bytes = need;
    }
    H_TRY(mape_extract_batch(items.data(), count, ws, ws_bytes, h0->stream));
    // every handle's candidates merged into its set by one mape_dedup_batch
    std::vector<mape_dedup_item> dd((size_t)count);
    std::vector<int64_t> cnt((size_t)count, 0);
    for (int i = 0; i < count; ++i) {
      mape_handle h = b.hs[i];
      H_TRY(h->chunk_candidates(h0->stream, &cnt[(size_t)i]));
      mape_dedup_item& it = dd[(size_t)i];
      it = mape_dedup_item{};
      it.cand = h->ex_cur; it.count = h->ex_U + cnt[(size_t)i]; it.n = h->n; it.ldc = h->ldg;
      it.uniq = h->ex_other; it.uniq_cap = h->cap; it.workspace = h->dWork; it.workspace_bytes = h->work_bytes;
    }
    if (!dws) {
      dws_bytes = mape_dedup_batch_workspace_bytes(count);
      dws = h0->take<char>(h0->job_bufs, dws_bytes);
      if (!dws) return MAPE_ERR_OOM;
    }
    H_TRY(mape_dedup_batch(dd.data(), count, dws, dws_bytes, h0->stream));
    for (int i = 0; i < count; ++i) b.hs[i]->chunk_merged(chunk, cnt[(size_t)i], dd[(size_t)i].K);
  }
  return MAPE_OK;
}

// The filter stages of every handle of the batch, each as one batched call:
// the kernel test, the minimality filter and the coefficients.
int run_batch_filter(ExtractBatch& b) {
  const int count = (int)b.hs.size();
  mape_handle h0 = b.hs[0];
  const double t_ext = now_ms();
  for (auto h : b.hs) h->set_phase(MAPE_PHASE_FILTERING);
  std::vector<mape_kernel_test_item> kt((size_t)count);
  std::vector<mape_minimal_item> mi((size_t)count);
  std::vector<mape_coeffs_item> ci((size_t)count);
  for (int i = 0; i < count; ++i) {
    mape_handle h = b.hs[i];
    kt[(size_t)i] = mape_kernel_test_item{h->dA, h->m, h->n, h->ex_cur, h->ex_U, h->ldg, 0, h->dOk, 0,
                                          h->dWork, h->work_bytes};
    // the kept rows go to the buffer of the pair that the last merge left free
    mi[(size_t)i] = mape_minimal_item{h->ex_cur, h->ex_U, h->n, h->ldg, h->dOk, h->dKeep, h->ex_other, 0,
                                      h->dWork, h->work_bytes};
  }
  const size_t b1 = mape_kernel_test_batch_workspace_bytes(count);
  const size_t b2 = mape_minimal_filter_batch_workspace_bytes(mi.data(), count);
  const size_t b3 = mape_direction_coeffs_batch_workspace_bytes(count);
  const size_t wb = std::max(b1, std::max(b2, b3));
  void* ws = h0->take<char>(h0->job_bufs, wb);
  if (!ws) return MAPE_ERR_OOM;
  H_TRY(mape_kernel_test_batch(kt.data(), count, ws, wb, h0->stream));
  H_TRY(mape_minimal_filter_batch(mi.data(), count, ws, wb, h0->stream));
  for (int i = 0; i < count; ++i) {
    mape_handle h = b.hs[i];
    ci[(size_t)i] = mape_coeffs_item{h->dqr, h->dqc, h->dqv, h->nnz, h->n, h->has_w ? h->dw : nullptr, h->ex_other,
                                     mi[(size_t)i].K_out, h->ldg, 0, h->da, h->dq4};
  }
  H_TRY(mape_direction_coeffs_batch(ci.data(), count, ws, wb, h0->stream));
  MAPE_CUDA_TRY(cudaStreamSynchronize(h0->stream));
  const double t_fil = now_ms();
  for (int i = 0; i < count; ++i) b.rcs[(size_t)i] = b.hs[i]->filter_done(kt[(size_t)i].fail_count, mi[(size_t)i].K_out,
                                                                           t_ext, t_fil);
  return MAPE_OK;
}

}  // namespace

extern "C" int mape_extract_directions(mape_handle h, int32_t P, const float* Z0, const float* G0) {
  if (!h) return MAPE_ERR_INVALID_ARG;
  int rc = prepare_job(h, P, Z0, G0);
  if (rc) return rc;
  mark_busy(h);
  h->worker = std::thread([h]() {
    cudaSetDevice(h->dev);
    int r = h->run_extract();
    h->finish(r);
  });
  return MAPE_OK;
}

extern "C" int mape_extract_directions_batch(mape_handle* hs, int32_t count, const int32_t* P, const float* const* Z0,
                                             const float* const* G0) {
  if (!hs || count <= 0 || !P) return MAPE_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return MAPE_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return MAPE_ERR_INVALID_ARG;
    const mape_config& c = hs[i]->cfg;
    const int32_t base = c.precision & MAPE_PREC_MASK;
    if ((base != MAPE_PREC_BF16 && base != MAPE_PREC_BF16X1) || (c.precision & MAPE_PREC_SPARSE_FWD) ||
        c.T != hs[0]->cfg.T || c.period != hs[0]->cfg.period ||
        (c.precision & MAPE_PREC_MASK) != (hs[0]->cfg.precision & MAPE_PREC_MASK))
      return MAPE_ERR_INVALID_ARG;
    if (!idle(hs[i])) return MAPE_ERR_STATE;
  }
  for (int i = 0; i < count; ++i) {
    int rc = prepare_job(hs[i], P[i], Z0 ? Z0[i] : nullptr, G0 ? G0[i] : nullptr);
    if (rc) return rc;
  }
  auto b = std::make_shared<ExtractBatch>();
  b->hs.assign(hs, hs + count);
  for (int i = 0; i < count; ++i) mark_busy(hs[i]);
  for (int i = 0; i < count; ++i) {
    mape_handle h = hs[i];
    h->worker = std::thread([h, b, i]() {
      cudaSetDevice(h->dev);
      int r = MAPE_OK;
      if (i == 0) {
        b->rcs.assign(b->hs.size(), MAPE_OK);
        r = run_batch_steps(*b);
        if (r == MAPE_OK) r = run_batch_filter(*b);
        std::lock_guard<std::mutex> lk(b->mu);
        b->rc = r;
        b->done = true;
        b->cv.notify_all();
      } else {
        std::unique_lock<std::mutex> lk(b->mu);
        b->cv.wait(lk, [&] { return b->done; });
        r = b->rc;
      }
      if (r == MAPE_OK) r = b->rcs[(size_t)i];
      h->finish(r);
    });
  }
  return MAPE_OK;
}

namespace {

// The starts of an augmentation job are uploaded and checked (A x = b, box).
int prepare_augment(mape_handle h, const int32_t* X0, int32_t S, const mape_problem* f) {
  using namespace mape_detail;
  if (!h || !X0 || S <= 0) return MAPE_ERR_INVALID_ARG;
  if (!idle(h)) return MAPE_ERR_STATE;
  h->join();
  {
    std::lock_guard<std::mutex> lk(h->mu);
    if (h->st.phase != MAPE_PHASE_DONE || h->dirs == nullptr) return MAPE_ERR_STATE;
  }
  if (f) {
    if (f->n != h->n || f->m != h->m) return MAPE_ERR_SHAPE;
    int rc = set_objective(h, f);
    if (rc) return rc;
    MAPE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (h->K > 0)
      if ((rc = mape_direction_coeffs(h->dqr, h->dqc, h->dqv, h->nnz, h->has_w ? h->dw : nullptr, h->n, h->dirs,
                                      h->K, h->ldg, h->da, h->dq4, h->stream)))
        return rc;
  }
  const int n = h->n;
  h->release_all(h->aug_bufs);
  h->S = S;
  h->dX = h->take<int32_t>(h->aug_bufs, (size_t)S * n);
  h->dF = h->take<int64_t>(h->aug_bufs, (size_t)S);
  int32_t* dbad = h->take<int32_t>(h->aug_bufs, 1);
  h->aug_work_bytes = mape_augment_workspace_bytes(n, S, h->K);
  h->dAugWork = h->take<char>(h->aug_bufs, h->aug_work_bytes);
  if (!h->dX || !h->dF || !dbad || !h->dAugWork) return MAPE_ERR_OOM;
  int rc = upload(h, h->dX, X0, sizeof(int32_t) * (size_t)S * n);
  if (rc) return rc;
  MAPE_CUDA_TRY(cudaMemsetAsync(dbad, 0, 4, h->stream));
  mape_detail::launch(feasible_check_kernel, S, 128, 0, h->stream, h->dA, h->db, h->dX, h->m, n, S, dbad);
  MAPE_LAUNCH_CHECK();
  int32_t bad = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&bad, dbad, 4, cudaMemcpyDeviceToHost, h->stream));
  MAPE_CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (bad) return MAPE_ERR_INFEASIBLE;
  return MAPE_OK;
}

void mark_augmenting(mape_handle h) {
  {
    std::lock_guard<std::mutex> lk(h->mu);
    h->busy = true;
    h->st.phase = MAPE_PHASE_AUGMENTING;
  }
  h->cancel.store(false);
}

// A batch of augmentation jobs: the first handle's worker runs Algorithm 1
// for every handle as mape_augment_run_batch calls (the first iteration
// alone, then the rest, as run_augment does for one); every worker then reads
// back its own best start.
struct AugmentBatch {
  std::vector<mape_handle> hs;
  std::mutex mu;
  std::condition_variable cv;
  bool done = false;
  int rc = MAPE_OK;
  std::vector<int64_t> it1, it2;
  std::vector<char> fin;  // per handle: its iterations are over (it2 set), before the whole batch ends
  double t0 = 0, t1 = 0;
};

// Called by mape_augment_run_batch as each handle's iterations end, so that
// its worker reads back its result while the others still iterate.
void augment_item_done(int32_t item, int64_t iters, void* ctx) {
  AugmentBatch* b = static_cast<AugmentBatch*>(ctx);
  std::lock_guard<std::mutex> lk(b->mu);
  b->it2[(size_t)item] = iters;
  b->fin[(size_t)item] = 1;
  b->cv.notify_all();
}

int run_augment_batch(AugmentBatch& b) {
  const int count = (int)b.hs.size();
  mape_handle h0 = b.hs[0];
  for (auto h : b.hs) {
    if (h->dev != h0->dev) return MAPE_ERR_INVALID_ARG;
    h->set_phase(MAPE_PHASE_AUGMENTING);
  }
  std::vector<mape_augment_args> items((size_t)count);
  std::vector<int64_t> max_iters((size_t)count);
  for (int i = 0; i < count; ++i) {
    b.hs[i]->augment_args(&items[(size_t)i]);
    max_iters[(size_t)i] = b.hs[i]->cfg.max_aug_iters;
  }
  const size_t ws_bytes = mape_augment_run_batch_workspace_bytes(count);
  void* ws = h0->take<char>(h0->aug_bufs, ws_bytes);
  if (!ws) return MAPE_ERR_OOM;
  b.t0 = now_ms();
  for (int i = 0; i < count; ++i) items[(size_t)i].max_iters = std::min<int64_t>(1, max_iters[(size_t)i]);
  H_TRY(mape_augment_run_batch(items.data(), count, b.it1.data(), ws, ws_bytes, h0->stream, nullptr, nullptr));
  b.t1 = now_ms();
  bool more = false;
  for (int i = 0; i < count; ++i) {
    mape_augment_args& a = items[(size_t)i];
    if (max_iters[(size_t)i] > 1 && !b.hs[i]->cancel.load()) {
      a.max_iters = max_iters[(size_t)i] - 1;
      more = true;
    } else {
      a.S = 0;  // as run_augment: no second call for this handle
    }
  }
  std::vector<int64_t> it2((size_t)count, 0);
  if (more) H_TRY(mape_augment_run_batch(items.data(), count, it2.data(), ws, ws_bytes, h0->stream,
                                         augment_item_done, &b));
  return MAPE_OK;
}

}  // namespace

extern "C" int mape_augment(mape_handle h, const int32_t* X0, int32_t S, const mape_problem* f) {
  int rc = prepare_augment(h, X0, S, f);
  if (rc) return rc;
  mark_augmenting(h);
  int64_t iters = h->cfg.max_aug_iters;
  h->worker = std::thread([h, iters]() {
    cudaSetDevice(h->dev);
    int r = h->run_augment(iters);
    h->finish(r);
  });
  return MAPE_OK;
}

extern "C" int mape_augment_batch(mape_handle* hs, int32_t count, const int32_t* const* X0, const int32_t* S) {
  if (!hs || count <= 0 || !X0 || !S) return MAPE_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return MAPE_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return MAPE_ERR_INVALID_ARG;
    if (hs[i]->dev != hs[0]->dev) return MAPE_ERR_INVALID_ARG;
    if (!idle(hs[i])) return MAPE_ERR_STATE;
  }
  for (int i = 0; i < count; ++i) {
    int rc = prepare_augment(hs[i], X0[i], S[i], nullptr);
    if (rc) return rc;
  }
  auto b = std::make_shared<AugmentBatch>();
  b->hs.assign(hs, hs + count);
  b->it1.assign((size_t)count, 0);
  b->it2.assign((size_t)count, 0);
  b->fin.assign((size_t)count, 0);
  for (int i = 0; i < count; ++i) mark_augmenting(hs[i]);
  for (int i = 0; i < count; ++i) {
    mape_handle h = hs[i];
    h->worker = std::thread([h, b, i]() {
      cudaSetDevice(h->dev);
      int r = MAPE_OK;
      if (i == 0) {
        r = run_augment_batch(*b);
        std::lock_guard<std::mutex> lk(b->mu);
        b->rc = r;
        b->done = true;
        b->cv.notify_all();
      } else {
        // this handle's iterations end (reported by the batch), or the batch does
        std::unique_lock<std::mutex> lk(b->mu);
        b->cv.wait(lk, [&] { return b->fin[(size_t)i] || b->done; });
        r = b->fin[(size_t)i] ? MAPE_OK : b->rc;
      }
      if (r == MAPE_OK) r = h->augment_end(b->it1[(size_t)i], b->it2[(size_t)i], b->t0, b->t1);
      h->finish(r);
    });
  }
  return MAPE_OK;
}

extern "C" int mape_poll(mape_handle h, mape_status* st) {
  if (!h || !st) return MAPE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  *st = h->st;
  return MAPE_OK;
}

extern "C" int mape_wait(mape_handle h, int64_t timeout_ns) {
  if (!h) return MAPE_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(h->mu);
  bool done = h->cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns < 0 ? 0 : timeout_ns), [h] { return !h->busy; });
  if (!done) return MAPE_ERR_TIMEOUT;
  return h->st.error;
}

extern "C" int mape_cancel(mape_handle h) {
  if (!h) return MAPE_ERR_INVALID_ARG;
  h->cancel.store(true);
  return MAPE_OK;
}

extern "C" int mape_get_directions(mape_handle h, int32_t* G, int64_t cap, int64_t* K) {
  using namespace mape_detail;
  if (!h || !K) return MAPE_ERR_INVALID_ARG;
  if (!idle(h)) return MAPE_ERR_STATE;
  *K = h->K;
  if (h->dirs == nullptr) return MAPE_ERR_STATE;
  if (cap < h->K) return MAPE_ERR_CAPACITY;
  if (h->K == 0) return MAPE_OK;
  if (!G) return MAPE_ERR_INVALID_ARG;
  int32_t* tmp = static_cast<int32_t*>(h->alloc(sizeof(int32_t) * (size_t)h->K * h->n));
  if (!tmp) return MAPE_ERR_OOM;
  int64_t tot = h->K * h->n;
  mape_detail::launch(i8_to_i32_kernel, (unsigned)ceil_div(tot, 256), 256, 0, h->stream, h->dirs, h->K, h->n, h->ldg, tmp);
  cudaError_t e = cudaMemcpyAsync(G, tmp, sizeof(int32_t) * (size_t)tot, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  h->release(tmp, sizeof(int32_t) * (size_t)tot);
  if (e != cudaSuccess) {
    record_cuda_error(e, "get_directions", __FILE__, __LINE__);
    return MAPE_ERR_CUDA;
  }
  return MAPE_OK;
}

extern "C" int mape_get_directions_i8(mape_handle h, int8_t* G, int64_t cap, int64_t ldg_out, int64_t* K) {
  using namespace mape_detail;
  if (!h || !K) return MAPE_ERR_INVALID_ARG;
  if (!idle(h)) return MAPE_ERR_STATE;
  *K = h->K;
  if (h->dirs == nullptr) return MAPE_ERR_STATE;
  if (cap < h->K) return MAPE_ERR_CAPACITY;
  if (h->K == 0) return MAPE_OK;
  if (!G || ldg_out < h->n) return MAPE_ERR_INVALID_ARG;
  // one contiguous copy when both pitches equal the row length, else by rows
  cudaError_t e = (ldg_out == h->n && h->ldg == h->n)
                      ? cudaMemcpyAsync(G, h->dirs, (size_t)h->K * h->n, cudaMemcpyDeviceToHost, h->stream)
                      : cudaMemcpy2DAsync(G, (size_t)ldg_out, h->dirs, (size_t)h->ldg, (size_t)h->n, (size_t)h->K,
                                          cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    record_cuda_error(e, "get_directions_i8", __FILE__, __LINE__);
    return MAPE_ERR_CUDA;
  }
  return MAPE_OK;
}

extern "C" int mape_get_solution(mape_handle h, int32_t* x, int64_t* fval) {
  if (!h || !x || !fval) return MAPE_ERR_INVALID_ARG;
  if (!idle(h)) return MAPE_ERR_STATE;
  if ((int)h->best_x.size() != h->n) return MAPE_ERR_STATE;
  std::memcpy(x, h->best_x.data(), sizeof(int32_t) * h->n);
  *fval = h->best_f;
  return MAPE_OK;
}

extern "C" int mape_get_solutions(mape_handle h, int32_t* X, int64_t* fval, int32_t S) {
  if (!h || !X || !fval) return MAPE_ERR_INVALID_ARG;
  if (!idle(h)) return MAPE_ERR_STATE;
  if (h->dX == nullptr || S != h->S) return MAPE_ERR_STATE;
  MAPE_CUDA_TRY(cudaMemcpyAsync(X, h->dX, sizeof(int32_t) * (size_t)S * h->n, cudaMemcpyDeviceToHost, h->stream));
  MAPE_CUDA_TRY(cudaMemcpyAsync(fval, h->dF, sizeof(int64_t) * (size_t)S, cudaMemcpyDeviceToHost, h->stream));
  MAPE_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return MAPE_OK;
}

namespace {
__global__ void sol_rows_kernel(const int8_t* __restrict__ rows, int64_t K, int n, int lds,
                                const int32_t* __restrict__ l, int32_t* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= K * n) return;
  const int64_t k = t / n;
  const int i = (int)(t % n);
  out[t] = (int32_t)(uint8_t)rows[k * lds + i] + l[i];
}
}  // namespace

extern "C" int mape_find_initial_solutions(mape_handle h, int32_t P, const float* X0, int32_t T, int32_t period,
                                           int32_t* X_out, int32_t cap, int32_t* S_out) {
  using namespace mape_detail;
  if (!h || !X0 || !S_out || P <= 0 || T < 0 || period <= 0 || cap < 0 || (cap > 0 && !X_out))
    return MAPE_ERR_INVALID_ARG;
  if (!idle(h)) return MAPE_ERR_STATE;
  h->join();
  const int n = h->n, m = h->m, lds = h->ldg;
  const int64_t rows = std::max<int64_t>(1, std::min<int64_t>((int64_t)P * (T / period + 1), (int64_t)1 << 22));
  std::vector<std::pair<void*, size_t>> bufs;
  auto cleanup = [&]() { h->release_all(bufs); };
  float* dX = h->take<float>(bufs, (size_t)P * n);
  float* dM = h->take<float>(bufs, (size_t)P * n);
  float* dV = h->take<float>(bufs, (size_t)P * n);
  int8_t* dSol = h->take<int8_t>(bufs, (size_t)rows * lds);
  int8_t* dUniq = h->take<int8_t>(bufs, (size_t)rows * lds);
  unsigned long long* dCount = h->take<unsigned long long>(bufs, 1);
  int32_t* dFlags = h->take<int32_t>(bufs, 1);
  const size_t iw = mape_initial_solutions_workspace_bytes(n, m, T);
  const size_t dw = mape_dedup_workspace_bytes(rows, lds);
  char* dWork = h->take<char>(bufs, std::max(iw, dw));
  if (!dX || !dM || !dV || !dSol || !dUniq || !dCount || !dFlags || !dWork) { cleanup(); return MAPE_ERR_OOM; }
  cudaStream_t s = h->stream;
  int rc = upload(h, dX, X0, sizeof(float) * (size_t)P * n);
  if (rc) { cleanup(); return rc; }
  if (cudaMemsetAsync(dM, 0, sizeof(float) * (size_t)P * n, s) != cudaSuccess ||
      cudaMemsetAsync(dV, 0, sizeof(float) * (size_t)P * n, s) != cudaSuccess ||
      cudaMemsetAsync(dSol, 0, (size_t)rows * lds, s) != cudaSuccess ||
      cudaMemsetAsync(dCount, 0, sizeof(unsigned long long), s) != cudaSuccess ||
      cudaMemsetAsync(dFlags, 0, sizeof(int32_t), s) != cudaSuccess) { cleanup(); return MAPE_ERR_CUDA; }
  mape_init_args a{};
  a.n = n; a.m = m; a.P = P; a.A = h->dA; a.b = h->db; a.l = h->dl; a.u = h->du; a.X = dX; a.M = dM; a.V = dV;
  a.t0 = 0; a.T = T; a.period = period; a.lambda3 = 0.1f; a.lr = h->cfg.lr; a.eps = h->cfg.eps;
  a.beta1 = h->cfg.beta1; a.beta2 = h->cfg.beta2;
  a.sol = reinterpret_cast<uint8_t*>(dSol); a.lds = lds; a.sol_cap = rows; a.sol_count = dCount; a.flags = dFlags;
  a.workspace = dWork; a.workspace_bytes = std::max(iw, dw);
  if ((rc = mape_initial_solutions(&a, s))) { cleanup(); return rc; }
  unsigned long long cnt = 0;
  int32_t flags = 0;
  if (cudaMemcpyAsync(&cnt, dCount, sizeof(cnt), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&flags, dFlags, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) { cleanup(); return MAPE_ERR_CUDA; }
  const int64_t got = std::min<int64_t>((int64_t)cnt, rows);
  int64_t K = 0;
  if (got > 0 && (rc = mape_dedup(dSol, got, n, lds, dUniq, rows, &K, dWork, std::max(iw, dw), s))) {
    cleanup();
    return rc;
  }
  *S_out = (int32_t)K;
  if (K > cap) { cleanup(); return MAPE_ERR_CAPACITY; }
  if (K > 0) {
    int32_t* dOut = h->take<int32_t>(bufs, (size_t)K * n);
    if (!dOut) { cleanup(); return MAPE_ERR_OOM; }
    launch(sol_rows_kernel, (unsigned)ceil_div(K * n, 256), 256, 0, s, dUniq, K, n, lds, h->dl, dOut);
    if (cudaMemcpyAsync(X_out, dOut, sizeof(int32_t) * (size_t)K * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { cleanup(); return MAPE_ERR_CUDA; }
  }
  cleanup();
  return (flags & 1) ? MAPE_ERR_CAPACITY : MAPE_OK;
}

extern "C" void mape_destroy(mape_handle h) {
  if (!h) return;
  h->cancel.store(true);
  h->join();
  h->release_all(h->aug_bufs);
  h->release_all(h->job_bufs);
  h->release_all(h->owned);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}
