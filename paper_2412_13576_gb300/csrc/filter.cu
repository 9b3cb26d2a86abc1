// a9: condition C1 (A g = 0, §3) and a11: condition C3 within the collected
// set (⊑-minimality, §1 and §3).
//
// Minimality: h ⊑ g with h != g implies ||h||_1 < ||g||_1, so a row g is only
// compared with strictly shorter rows.  Rows are counting-sorted by l1 norm
// (bins 0 .. 127 n), and the row at sorted position q scans exactly the
// positions below the start of its own bin.  Each row carries sign-support
// bitmasks (pos, neg; 64 coordinates per word): h ⊑ g needs pos(h) ⊆ pos(g)
// and neg(h) ⊆ neg(g); -h ⊑ g needs pos(h) ⊆ neg(g) and neg(h) ⊆ pos(g).  The
// first mask word rejects almost every pair; survivors get the remaining words
// and then the magnitude test |h_i| <= |g_i|.  Kept rows are compacted in
// their input order.
#include "common.cuh"

#include <algorithm>

namespace {

constexpr int kInvalidL1 = 0x7fffffff;

// ---- a9 -----------------------------------------------------------------------

constexpr int kMaxRegRow = 256;  // rows up to this pitch are held in registers

// A g over int8 rows.  When A's entries fit in int8 and A (m x ldg bytes)
// fits in shared memory, the row is held in 16 uint4 registers and each
// constraint is 4 dp4a per 16 bytes (exact: |sum| <= 127 * 127 * n < 2^31);
// otherwise plain int32 products from global memory.
__global__ void kernel_test_kernel(const int32_t* __restrict__ A, int m, int n, const int8_t* __restrict__ G,
                                   int64_t K, int ldg, int stage8, uint8_t* __restrict__ ok,
                                   unsigned long long* __restrict__ fails) {
  extern __shared__ int8_t s_A8[];  // m x ldg
  int bad = 0;
  if (stage8) {
    for (int e = threadIdx.x; e < m * ldg; e += blockDim.x) {
      int r = e / ldg, i = e % ldg;
      int v = i < n ? A[(int64_t)r * n + i] : 0;
      if (v > 127 || v < -127) bad = 1;
      s_A8[e] = (int8_t)v;
    }
  }
  const bool use8 = stage8 && !__syncthreads_or(bad);
  const int nv = ldg / 16;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
    const int8_t* g = G + k * ldg;
    bool good = true;
    if (use8) {
      uint4 gv[kMaxRegRow / 16];
#pragma unroll
      for (int w = 0; w < kMaxRegRow / 16; ++w)
        gv[w] = w < nv ? reinterpret_cast<const uint4*>(g)[w] : make_uint4(0, 0, 0, 0);
      for (int r = 0; r < m && good; ++r) {
        const uint4* a4 = reinterpret_cast<const uint4*>(s_A8 + (int64_t)r * ldg);
        int acc = 0;
#pragma unroll
        for (int w = 0; w < kMaxRegRow / 16; ++w) {
          if (w < nv) {
            const uint4 a = a4[w];
            acc = __dp4a((int)a.x, (int)gv[w].x, acc);
            acc = __dp4a((int)a.y, (int)gv[w].y, acc);
            acc = __dp4a((int)a.z, (int)gv[w].z, acc);
            acc = __dp4a((int)a.w, (int)gv[w].w, acc);
          }
        }
        good = (acc == 0);
      }
    } else {
      for (int r = 0; r < m && good; ++r) {
        const int32_t* a = A + (int64_t)r * n;
        long long acc = 0;
        for (int i = 0; i < n; ++i) acc += (long long)a[i] * g[i];
        good = (acc == 0);
      }
    }
    ok[k] = good ? 1 : 0;
    if (!good) atomicAdd(fails, 1ull);
  }
}

// ---- a11 ----------------------------------------------------------------------

// l1 norm and sign masks per row; rows with valid == 0 get l1 = kInvalidL1
__global__ void prep_kernel(const int8_t* __restrict__ G, int64_t K, int n, int ldg, int W,
                            const uint8_t* __restrict__ valid, int32_t* __restrict__ l1,
                            uint64_t* __restrict__ masks, uint32_t* __restrict__ hist) {
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
  l1[k] = v_ok ? s : kInvalidL1;
  if (v_ok) atomicAdd(&hist[s], 1u);
}

// exclusive prefix over bins (one block); cursor receives a copy of the starts
__global__ void bin_scan_kernel(const uint32_t* __restrict__ hist, int nbins, uint32_t* __restrict__ start,
                                uint32_t* __restrict__ cursor) {
  __shared__ uint32_t s_part[1024];
  __shared__ uint32_t s_base;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nbins; b0 += blockDim.x) {
    int b = b0 + threadIdx.x;
    uint32_t v = b < nbins ? hist[b] : 0;
    s_part[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {  // Hillis-Steele inclusive scan
      uint32_t add = threadIdx.x >= (unsigned)off ? s_part[threadIdx.x - off] : 0;
      __syncthreads();
      s_part[threadIdx.x] += add;
      __syncthreads();
    }
    uint32_t excl = s_base + s_part[threadIdx.x] - v;
    __syncthreads();
    if (b < nbins) {
      start[b] = excl;
      cursor[b] = excl;
    }
    if (threadIdx.x == blockDim.x - 1) s_base += s_part[threadIdx.x];
    __syncthreads();
  }
}

// sorted arrays: row index, first mask words, and the number of strictly
// shorter rows (the start of the row's bin)
__global__ void scatter_kernel(const int32_t* __restrict__ l1, const uint64_t* __restrict__ masks, int64_t K, int W,
                               const uint32_t* __restrict__ start, uint32_t* __restrict__ cursor,
                               uint32_t* __restrict__ s_idx, uint64_t* __restrict__ s_pk,
                               ulonglong2* __restrict__ s_sig, uint32_t* __restrict__ s_lim) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= K || l1[k] == kInvalidL1) return;
  uint32_t q = atomicAdd(&cursor[l1[k]], 1u);
  s_idx[q] = (uint32_t)k;
  // sign masks of coordinates 0..31: pos in the low half, neg in the high half
  s_pk[q] = (masks[k * 2 * W] & 0xffffffffull) | (masks[k * 2 * W + W] << 32);
  // second filter: every coordinate i folded onto bit i mod 64 (OR of the
  // mask words), pos and neg apart; support and signs of h within those of
  // +-g imply the same for these signatures
  uint64_t pos = 0, neg = 0;
  for (int w = 0; w < W; ++w) {
    pos |= masks[k * 2 * W + w];
    neg |= masks[k * 2 * W + W + w];
  }
  s_sig[q] = make_ulonglong2(pos, neg);
  s_lim[q] = start[l1[k]];
}

constexpr int kTile = 256;

__device__ __forceinline__ bool magnitudes_fit(const int8_t* h, const int8_t* g, int n) {
  for (int i = 0; i < n; ++i)
    if (abs((int)h[i]) > abs((int)g[i])) return false;
  return true;
}

// full test of h against g once the 32-coordinate prefilter passed
__device__ __forceinline__ bool dominates(const int8_t* __restrict__ G, int n, int ldg, int W,
                                          const uint64_t* __restrict__ masks, uint32_t h, uint32_t k) {
  const uint64_t* hm = masks + (int64_t)h * 2 * W;
  const uint64_t* gm = masks + (int64_t)k * 2 * W;
  bool same = true, flip = true;
  for (int w = 0; w < W && (same || flip); ++w) {
    uint64_t a = hm[w], b = hm[W + w], c = gm[w], e = gm[W + w];
    same = same && ((a & ~c) | (b & ~e)) == 0;
    flip = flip && ((a & ~e) | (b & ~c)) == 0;
  }
  return (same || flip) && magnitudes_fit(G + (int64_t)h * ldg, G + (int64_t)k * ldg, n);
}

constexpr int kChunk = 4096;  // shorter rows scanned by one block

// Work unit (blockIdx.x, blockIdx.y): the 256 sorted rows of row block x
// against the shorter rows [y * kChunk, (y + 1) * kChunk).  Every unit has
// the same size, so the quadratic work spreads evenly over the SMs however the
// rows' limits grow along the l1 order.  Prefilters per pair: sign masks of
// coordinates 0..31 packed in one word (pos | neg << 32), then, for the pairs
// that pass, the folded 64-bit signatures of all coordinates, before the full
// test.  A dominated row gets dom[k] = 1 (several units may write it).
__global__ void dominance_kernel(const int8_t* __restrict__ G, int n, int ldg, int W, const uint64_t* __restrict__ masks,
                                 int64_t nvalid, const uint32_t* __restrict__ s_idx, const uint64_t* __restrict__ s_pk,
                                 const ulonglong2* __restrict__ s_sig, const uint32_t* __restrict__ s_lim,
                                 uint8_t* __restrict__ dom) {
  __shared__ uint64_t t_pk[kTile];
  __shared__ ulonglong2 t_sig[kTile];
  __shared__ uint32_t s_blim;
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const uint32_t lo = blockIdx.y * (uint32_t)kChunk;
  if (threadIdx.x == 0) {
    int64_t last = blockIdx.x * (int64_t)blockDim.x + blockDim.x - 1;
    if (last >= nvalid) last = nvalid - 1;
    s_blim = s_lim[last];  // rows are in l1 order: the last has the largest limit
  }
  __syncthreads();
  const uint32_t blim = s_blim;
  if (lo >= blim) return;  // uniform over the block
  const uint32_t hi = (lo + kChunk < blim) ? lo + kChunk : blim;
  const bool mine = q < nvalid;
  const uint32_t lim = mine ? s_lim[q] : 0;
  const uint32_t k = mine ? s_idx[q] : 0;
  const uint64_t pk = mine ? s_pk[q] : 0;
  const uint32_t np = ~(uint32_t)pk, nn = ~(uint32_t)(pk >> 32);
  const ulonglong2 gs = mine ? s_sig[q] : make_ulonglong2(0, 0);
  const uint64_t gsp = ~gs.x, gsn = ~gs.y;
  bool done = !mine || lim <= lo || dom[k];
  for (uint32_t base = lo; base < hi; base += kTile) {
    __syncthreads();
    for (int t = threadIdx.x; t < kTile; t += blockDim.x) {
      uint32_t h = base + t;
      if (h < hi) {
        t_pk[t] = s_pk[h];
        t_sig[t] = s_sig[h];
      }
    }
    __syncthreads();
    if (done) continue;
    const uint32_t stop = lim < hi ? lim : hi;
    const int cnt = stop > base ? (int)((stop - base) < (uint32_t)kTile ? (stop - base) : (uint32_t)kTile) : 0;
#pragma unroll 4
    for (int t = 0; t < cnt; ++t) {
      const uint64_t hk = t_pk[t];
      const uint32_t hp = (uint32_t)hk, hn = (uint32_t)(hk >> 32);
      const bool cand = (((hp & np) | (hn & nn)) == 0) || (((hp & nn) | (hn & np)) == 0);
      if (!cand) continue;
      const ulonglong2 hs = t_sig[t];
      const bool cand2 = (((hs.x & gsp) | (hs.y & gsn)) == 0) || (((hs.x & gsn) | (hs.y & gsp)) == 0);
      if (cand2 && dominates(G, n, ldg, W, masks, s_idx[base + t], k)) {
        done = true;
        dom[k] = 1;
        break;
      }
    }
  }
}

// keep = valid and not dominated
__global__ void finalize_keep_kernel(const int32_t* __restrict__ l1, const uint8_t* __restrict__ dom, int64_t K,
                                     uint8_t* __restrict__ keep) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < K) keep[k] = (l1[k] != kInvalidL1 && !dom[k]) ? 1 : 0;
}

__global__ void clear_keep_kernel(uint8_t* keep, int64_t K) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < K) keep[k] = 0;
}

constexpr int kCompact = 1024;

__global__ void count_kept_kernel(const uint8_t* __restrict__ keep, int64_t K, uint32_t* __restrict__ block_count) {
  __shared__ uint32_t s_c;
  if (threadIdx.x == 0) s_c = 0;
  __syncthreads();
  int64_t k = blockIdx.x * (int64_t)kCompact + threadIdx.x;
  unsigned bal = __ballot_sync(0xffffffffu, k < K && keep[k]);
  if ((threadIdx.x & 31) == 0) atomicAdd(&s_c, (uint32_t)__popc(bal));
  __syncthreads();
  if (threadIdx.x == 0) block_count[blockIdx.x] = s_c;
}

__global__ void write_kept_kernel(const int8_t* __restrict__ G, int64_t K, int ldg, const uint8_t* __restrict__ keep,
                                  const uint32_t* __restrict__ block_start, int8_t* __restrict__ out) {
  __shared__ uint32_t s_warp[kCompact / 32];
  int64_t k = blockIdx.x * (int64_t)kCompact + threadIdx.x;
  int f = (k < K && keep[k]) ? 1 : 0;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned bal = __ballot_sync(0xffffffffu, f);
  if (lane == 0) s_warp[wid] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int w = 0; w < kCompact / 32; ++w) { uint32_t c = s_warp[w]; s_warp[w] = acc; acc += c; }
  }
  __syncthreads();
  if (!f) return;
  int64_t dst = (int64_t)block_start[blockIdx.x] + s_warp[wid] + __popc(bal & ((1u << lane) - 1));
  const uint4* src = reinterpret_cast<const uint4*>(G + k * ldg);
  uint4* d4 = reinterpret_cast<uint4*>(out + dst * ldg);
  for (int c = 0; c < ldg / 16; ++c) d4[c] = src[c];
}

int64_t l1_bins(int32_t n) { return (int64_t)127 * n + 1; }

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
  const int stage8 = ((int64_t)m * ldg <= 48 * 1024 && ldg <= kMaxRegRow) ? 1 : 0;
  MAPE_CUDA_TRY(cudaMemsetAsync(d_fail, 0, sizeof(unsigned long long), st));
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(K, 128), 152 * 4);
  mape_detail::launch(kernel_test_kernel, grid, 128, stage8 ? (size_t)m * ldg : 0, st, A, m, n, G, K, ldg, stage8, ok,
                      d_fail);
  MAPE_LAUNCH_CHECK();
  unsigned long long f = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&f, d_fail, sizeof(f), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  *fail_count = (int64_t)f;
  return MAPE_OK;
}

extern "C" size_t mape_minimal_workspace_bytes(int64_t K, int32_t n) {
  using namespace mape_detail;
  if (K < 0 || n <= 0) return 0;
  int W = (n + 63) / 64;
  int64_t nb = l1_bins(n);
  Sizer s;
  s.take<int32_t>((size_t)K);                 // l1
  s.take<uint64_t>((size_t)K * 2 * W);        // masks
  s.take<uint32_t>((size_t)nb);               // histogram
  s.take<uint32_t>((size_t)nb);               // bin starts
  s.take<uint32_t>((size_t)nb);               // cursors
  s.take<uint32_t>((size_t)K);                // sorted row index
  s.take<uint64_t>((size_t)K);                // sorted packed sign masks
  s.take<ulonglong2>((size_t)K);              // sorted folded signatures
  s.take<uint32_t>((size_t)K);                // sorted limits
  s.take<uint32_t>((size_t)ceil_div(K, kCompact) + 1);  // block counts
  s.take<uint32_t>((size_t)ceil_div(K, kCompact) + 1);  // block starts
  return s.bytes();
}

extern "C" int mape_minimal_filter(const int8_t* G, int64_t K, int32_t n, int32_t ldg, const uint8_t* valid,
                                   uint8_t* keep, int8_t* out, int64_t* K_out, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  using namespace mape_detail;
  if (K < 0 || n <= 0 || ldg < n || ldg % 16 != 0 || !K_out || (K > 0 && (!G || !keep || !out)))
    return MAPE_ERR_INVALID_ARG;
  if (n > 4096) return MAPE_ERR_SHAPE;
  if (K >= ((int64_t)1 << 31)) return MAPE_ERR_SHAPE;
  *K_out = 0;
  if (K == 0) return MAPE_OK;
  const int W = (n + 63) / 64;
  const int64_t nb = l1_bins(n);
  const int64_t nblk = ceil_div(K, kCompact);
  Carver cv(workspace, workspace_bytes);
  int32_t* l1 = cv.take<int32_t>((size_t)K);
  uint64_t* masks = cv.take<uint64_t>((size_t)K * 2 * W);
  uint32_t* hist = cv.take<uint32_t>((size_t)nb);
  uint32_t* start = cv.take<uint32_t>((size_t)nb);
  uint32_t* cursor = cv.take<uint32_t>((size_t)nb);
  uint32_t* s_idx = cv.take<uint32_t>((size_t)K);
  uint64_t* s_pk = cv.take<uint64_t>((size_t)K);
  ulonglong2* s_sig = cv.take<ulonglong2>((size_t)K);
  uint32_t* s_lim = cv.take<uint32_t>((size_t)K);
  uint32_t* bcount = cv.take<uint32_t>((size_t)nblk + 1);
  uint32_t* bstart = cv.take<uint32_t>((size_t)nblk + 1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  MAPE_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nb, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(bcount, 0, sizeof(uint32_t) * (nblk + 1), st));
  const unsigned g = (unsigned)ceil_div(K, kTile);
  mape_detail::launch(prep_kernel, g, kTile, 0, st, G, K, n, ldg, W, valid, l1, masks, hist);
  mape_detail::launch(bin_scan_kernel, 1, 1024, 0, st, hist, (int)nb, start, cursor);
  mape_detail::launch(scatter_kernel, g, kTile, 0, st, l1, masks, K, W, start, cursor, s_idx, s_pk, s_sig, s_lim);
  mape_detail::launch(clear_keep_kernel, g, kTile, 0, st, keep, K);
  MAPE_LAUNCH_CHECK();
  // number of valid rows = end of the last bin
  uint32_t last_start = 0, last_count = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&last_start, start + nb - 1, 4, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(&last_count, hist + nb - 1, 4, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  const int64_t nvalid = (int64_t)last_start + last_count;
  if (nvalid > 0)
    mape_detail::launch(dominance_kernel, dim3((unsigned)ceil_div(nvalid, kTile), (unsigned)ceil_div(nvalid, kChunk)),
                        kTile, 0, st, G, n, ldg, W, masks, nvalid, s_idx, s_pk, s_sig, s_lim, keep);
  mape_detail::launch(finalize_keep_kernel, g, kTile, 0, st, l1, keep, K, keep);
  mape_detail::launch(count_kept_kernel, (unsigned)nblk, kCompact, 0, st, keep, K, bcount);
  // block starts: exclusive prefix of the counts, entry nblk = total
  mape_detail::launch(bin_scan_kernel, 1, 1024, 0, st, bcount, (int)nblk + 1, bstart, bstart);
  mape_detail::launch(write_kept_kernel, (unsigned)nblk, kCompact, 0, st, G, K, ldg, keep, bstart, out);
  MAPE_LAUNCH_CHECK();
  uint32_t total = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&total, bstart + nblk, 4, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  *K_out = (int64_t)total;
  return MAPE_OK;
}
