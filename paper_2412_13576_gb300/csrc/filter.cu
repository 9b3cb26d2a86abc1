// a9: condition C1 (A g = 0, §3) and a11: condition C3 within the collected
// set (⊑-minimality, §1 and §3).
//
// Minimality: h ⊑ g with h != g implies ||h||_1 < ||g||_1, so a row g is
// only compared with strictly shorter rows.  Each row carries its l1 norm and
// sign-support bitmasks (pos, neg; 64 coordinates per word).  h ⊑ g needs
// pos(h) ⊆ pos(g) and neg(h) ⊆ neg(g); -h ⊑ g needs pos(h) ⊆ neg(g) and
// neg(h) ⊆ pos(g).  The first mask word rejects almost every pair; survivors
// get the remaining words and then the magnitude test |h_i| <= |g_i|.
#include "common.cuh"

namespace {

__global__ void kernel_test_kernel(const int32_t* __restrict__ A, int m, int n, const int8_t* __restrict__ G,
                                   int64_t K, int ldg, uint8_t* __restrict__ ok,
                                   unsigned long long* __restrict__ fails) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int8_t* g = G + k * ldg;
  bool good = true;
  for (int r = 0; r < m && good; ++r) {
    const int32_t* a = A + (int64_t)r * n;
    int acc = 0;
    for (int i = 0; i < n; ++i) acc += a[i] * (int)g[i];
    good = (acc == 0);
  }
  ok[k] = good ? 1 : 0;
  if (!good) atomicAdd(fails, 1ull);
}

constexpr int kTile = 256;

// l1 norm and sign masks per row; invalid rows get l1 = INT_MAX.
__global__ void prep_kernel(const int8_t* __restrict__ G, int64_t K, int n, int ldg, int W,
                            const uint8_t* __restrict__ valid, int32_t* __restrict__ l1,
                            uint64_t* __restrict__ masks) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int8_t* g = G + k * ldg;
  int s = 0;
  uint64_t* pm = masks + k * 2 * W;
  for (int w = 0; w < W; ++w) {
    uint64_t pos = 0, neg = 0;
    for (int b = 0; b < 64; ++b) {
      int i = w * 64 + b;
      if (i >= n) break;
      int v = g[i];
      s += abs(v);
      if (v > 0) pos |= 1ull << b;
      if (v < 0) neg |= 1ull << b;
    }
    pm[w] = pos;
    pm[W + w] = neg;
  }
  bool v_ok = valid == nullptr || valid[k] != 0;
  l1[k] = v_ok ? s : 0x7fffffff;
}

__device__ __forceinline__ bool magnitudes_fit(const int8_t* h, const int8_t* g, int n) {
  for (int i = 0; i < n; ++i)
    if (abs((int)h[i]) > abs((int)g[i])) return false;
  return true;
}

__global__ void dominance_kernel(const int8_t* __restrict__ G, int64_t K, int n, int ldg, int W,
                                 const int32_t* __restrict__ l1, const uint64_t* __restrict__ masks,
                                 uint8_t* __restrict__ keep) {
  __shared__ int32_t s_l1[kTile];
  __shared__ uint64_t s_pos[kTile], s_neg[kTile];
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool active = k < K;
  int32_t my_l1 = active ? l1[k] : 0x7fffffff;
  if (my_l1 == 0x7fffffff) active = false;
  uint64_t gp = 0, gn = 0;
  if (active) {
    gp = masks[k * 2 * W];
    gn = masks[k * 2 * W + W];
  }
  bool dominated = false;
  for (int64_t base = 0; base < K; base += kTile) {
    __syncthreads();
    for (int t = threadIdx.x; t < kTile; t += blockDim.x) {
      int64_t h = base + t;
      if (h < K) {
        s_l1[t] = l1[h];
        s_pos[t] = masks[h * 2 * W];
        s_neg[t] = masks[h * 2 * W + W];
      } else {
        s_l1[t] = 0x7fffffff;
      }
    }
    __syncthreads();
    if (!active || dominated) continue;
    int lim = (K - base) < kTile ? (int)(K - base) : kTile;
    for (int t = 0; t < lim; ++t) {
      if (s_l1[t] >= my_l1) continue;
      uint64_t hp = s_pos[t], hn = s_neg[t];
      bool same = ((hp & ~gp) | (hn & ~gn)) == 0;
      bool flip = ((hp & ~gn) | (hn & ~gp)) == 0;
      if (!same && !flip) continue;
      int64_t h = base + t;
      const uint64_t* hm = masks + h * 2 * W;
      const uint64_t* gm = masks + k * 2 * W;
      for (int w = 1; w < W && (same || flip); ++w) {
        uint64_t a = hm[w], b = hm[W + w], c = gm[w], e = gm[W + w];
        same = same && ((a & ~c) | (b & ~e)) == 0;
        flip = flip && ((a & ~e) | (b & ~c)) == 0;
      }
      if ((same || flip) && magnitudes_fit(G + h * ldg, G + k * ldg, n)) {
        dominated = true;
        break;
      }
    }
  }
  if (k < K) keep[k] = (active && !dominated) ? 1 : 0;
}

// Order-preserving compaction of kept rows by one block (exclusive scan).
__global__ void compact_kept_kernel(const int8_t* __restrict__ G, int64_t K, int ldg, const uint8_t* __restrict__ keep,
                                    int8_t* __restrict__ out, unsigned long long* __restrict__ Kout) {
  __shared__ int64_t s_base;
  __shared__ int s_warp[32];
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t start = 0; start < K; start += blockDim.x) {
    int64_t k = start + threadIdx.x;
    int f = (k < K && keep[k]) ? 1 : 0;
    unsigned bal = __ballot_sync(0xffffffffu, f);
    int before = __popc(bal & ((1u << lane) - 1));
    if (lane == 0) s_warp[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { int c = s_warp[w]; s_warp[w] = acc; acc += c; }
    }
    __syncthreads();
    if (f) {
      int64_t dst = s_base + s_warp[wid] + before;
      const uint4* src = reinterpret_cast<const uint4*>(G + k * ldg);
      uint4* d4 = reinterpret_cast<uint4*>(out + dst * ldg);
      for (int c = 0; c < ldg / 16; ++c) d4[c] = src[c];
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_base += s_warp[wid] + before + f;
    __syncthreads();
  }
  if (threadIdx.x == 0) *Kout = (unsigned long long)s_base;
}

}  // namespace

extern "C" size_t mape_kernel_test_workspace_bytes(void) {
  mape_detail::Sizer s;
  s.take<unsigned long long>(1);
  return s.bytes();
}

extern "C" int mape_kernel_test(const int32_t* A, int32_t m, int32_t n, const int8_t* G, int64_t K, int32_t ldg,
                                uint8_t* ok, int64_t* fail_count, void* workspace, size_t workspace_bytes,
                                void* stream) {
  using namespace mape_detail;
  if (!A || m <= 0 || n <= 0 || ldg < n || K < 0 || !fail_count || (K > 0 && (!G || !ok)))
    return MAPE_ERR_INVALID_ARG;
  if (n > 4096) return MAPE_ERR_SHAPE;
  *fail_count = 0;
  if (K == 0) return MAPE_OK;
  Carver cv(workspace, workspace_bytes);
  unsigned long long* d_fail = cv.take<unsigned long long>(1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  MAPE_CUDA_TRY(cudaMemsetAsync(d_fail, 0, sizeof(unsigned long long), st));
  mape_detail::launch(kernel_test_kernel, (unsigned)ceil_div(K, 128), 128, 0, st, A, m, n, G, K, ldg, ok, d_fail);
  MAPE_LAUNCH_CHECK();
  unsigned long long f = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&f, d_fail, sizeof(f), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  *fail_count = (int64_t)f;
  return MAPE_OK;
}

extern "C" size_t mape_minimal_workspace_bytes(int64_t K, int32_t n) {
  if (K < 0 || n <= 0) return 0;
  int W = (n + 63) / 64;
  mape_detail::Sizer s;
  s.take<int32_t>((size_t)K);
  s.take<uint64_t>((size_t)K * 2 * W);
  s.take<unsigned long long>(1);
  return s.bytes();
}

extern "C" int mape_minimal_filter(const int8_t* G, int64_t K, int32_t n, int32_t ldg, const uint8_t* valid,
                                   uint8_t* keep, int8_t* out, int64_t* K_out, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  using namespace mape_detail;
  if (K < 0 || n <= 0 || ldg < n || ldg % 16 != 0 || !K_out || (K > 0 && (!G || !keep || !out)))
    return MAPE_ERR_INVALID_ARG;
  if (n > 4096) return MAPE_ERR_SHAPE;
  *K_out = 0;
  if (K == 0) return MAPE_OK;
  int W = (n + 63) / 64;
  Carver cv(workspace, workspace_bytes);
  int32_t* l1 = cv.take<int32_t>((size_t)K);
  uint64_t* masks = cv.take<uint64_t>((size_t)K * 2 * W);
  unsigned long long* dK = cv.take<unsigned long long>(1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  unsigned g = (unsigned)ceil_div(K, kTile);
  mape_detail::launch(prep_kernel, g, kTile, 0, st, G, K, n, ldg, W, valid, l1, masks);
  mape_detail::launch(dominance_kernel, g, kTile, 0, st, G, K, n, ldg, W, l1, masks, keep);
  mape_detail::launch(compact_kept_kernel, 1, 1024, 0, st, G, K, ldg, keep, out, dK);
  MAPE_LAUNCH_CHECK();
  unsigned long long kk = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&kk, dK, sizeof(kk), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  *K_out = (int64_t)kk;
  return MAPE_OK;
}
