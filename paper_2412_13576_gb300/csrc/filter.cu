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
#include <vector>

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

// A in compressed rows (CSR), for the test of rows too long for the dp4a path:
// row r's nonzeros are col[rowptr[r] .. rowptr[r+1]), val[...] in column order.
// One warp per row of A.
__global__ void csr_count_kernel(const int32_t* __restrict__ A, int m, int n, uint32_t* __restrict__ rowcnt) {
  const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= m) return;
  uint32_t c = 0;
  for (int i = lane; i < n; i += 32) c += A[(int64_t)r * n + i] != 0;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if (lane == 0) rowcnt[r] = c;
}

__global__ void csr_fill_kernel(const int32_t* __restrict__ A, int m, int n, const uint32_t* __restrict__ rowptr,
                                uint16_t* __restrict__ col, int32_t* __restrict__ val) {
  const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= m) return;
  uint32_t pos = rowptr[r];
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    const int v = i < n ? A[(int64_t)r * n + i] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, v != 0);
    if (v != 0) {
      const uint32_t q = pos + __popc(bal & ((1u << lane) - 1));
      col[q] = (uint16_t)i;
      val[q] = v;
    }
    pos += __popc(bal);
  }
}

// A g over rows staged in shared memory, one warp per group of candidate
// rows: lane j takes the rows j, j + 32, ... of A through their nonzeros
// (int64 sums, exact for every int32 A and int8 g).  Each candidate row is
// read once, with 16-byte loads.
constexpr int kCsrWarps = 8;
constexpr int kCsrMaxRow = 4096;

// cnt <= kCsrRows candidate rows k0 .. k0 + cnt - 1 by the calling warp
// (rows: its kCsrRows shared-memory rows, ldg bytes apart): every nonzero of A
// is loaded once for all of them, and their sums are independent chains.
constexpr int kCsrRows = 4;

__device__ __forceinline__ void csr_test_rows(const uint32_t* __restrict__ rowptr, const uint16_t* __restrict__ col,
                                              const int32_t* __restrict__ val, int m, const int8_t* __restrict__ G,
                                              int64_t k0, int cnt, int ldg, int8_t* rows, uint8_t* __restrict__ ok,
                                              unsigned long long* __restrict__ fails) {
  const int lane = threadIdx.x & 31;
  const int nv = ldg / 16;
  for (int q = 0; q < cnt; ++q) {
    const uint4* src = reinterpret_cast<const uint4*>(G + (k0 + q) * ldg);
    for (int c = lane; c < nv; c += 32) reinterpret_cast<uint4*>(rows + q * ldg)[c] = src[c];
  }
  __syncwarp();
  bool good[kCsrRows];
#pragma unroll
  for (int q = 0; q < kCsrRows; ++q) good[q] = true;
  for (int r = lane; r < m; r += 32) {
    long long acc[kCsrRows] = {0, 0, 0, 0};
    const uint32_t e1 = rowptr[r + 1];
    for (uint32_t e = rowptr[r]; e < e1; ++e) {
      const long long v = val[e];
      const int c = col[e];
#pragma unroll
      for (int q = 0; q < kCsrRows; ++q) acc[q] += v * rows[q * ldg + c];  // rows past cnt: unused
    }
#pragma unroll
    for (int q = 0; q < kCsrRows; ++q) good[q] &= (acc[q] == 0);
  }
#pragma unroll
  for (int q = 0; q < kCsrRows; ++q) {
    const bool g = __all_sync(0xffffffffu, good[q]);
    if (lane == 0 && q < cnt) {
      ok[k0 + q] = g ? 1 : 0;
      if (!g) atomicAdd(fails, 1ull);
    }
  }
  __syncwarp();
}

// dynamic shared memory: kCsrWarps x kCsrRows rows of ldg bytes
__global__ void __launch_bounds__(32 * kCsrWarps)
kernel_test_csr_kernel(const uint32_t* __restrict__ rowptr, const uint16_t* __restrict__ col,
                       const int32_t* __restrict__ val, int m, const int8_t* __restrict__ G, int64_t K,
                       int ldg, uint8_t* __restrict__ ok, unsigned long long* __restrict__ fails) {
  extern __shared__ __align__(16) int8_t s_rows[];
  const int w = threadIdx.x >> 5;
  int8_t* rows = s_rows + (size_t)w * kCsrRows * ldg;
  for (int64_t k0 = (blockIdx.x * (int64_t)kCsrWarps + w) * kCsrRows; k0 < K;
       k0 += (int64_t)gridDim.x * kCsrWarps * kCsrRows)
    csr_test_rows(rowptr, col, val, m, G, k0, (int)(K - k0 < kCsrRows ? K - k0 : kCsrRows), ldg, rows, ok, fails);
}

// ---- a11 ----------------------------------------------------------------------

// l1 norm and sign masks per row; rows with valid == 0 get l1 = kInvalidL1
__device__ __forceinline__ void prep_row(const int8_t* __restrict__ G, int64_t k, int n, int ldg, int W,
                                         const uint8_t* __restrict__ valid, int32_t* __restrict__ l1,
                                         uint64_t* __restrict__ masks, uint32_t* __restrict__ hist) {
  const int8_t* g = G + k * ldg;
  int s = 0;
  uint64_t* pm = masks + k * 2 * W;
  // rows 16-byte aligned (ldg a multiple of 16, G aligned): 16-byte loads,
  // four per mask word (a piece starting below n ends within the pitch)
  const bool vec = (ldg & 15) == 0 && (reinterpret_cast<uintptr_t>(G) & 15) == 0;
  for (int w = 0; w < W; ++w) {
    uint64_t pos = 0, neg = 0;
    if (vec) {
      for (int q = 0; q < 4; ++q) {
        const int i0 = w * 64 + q * 16;
        if (i0 >= n) break;
        const int4 pc = *reinterpret_cast<const int4*>(g + i0);
        const uint32_t wd[4] = {(uint32_t)pc.x, (uint32_t)pc.y, (uint32_t)pc.z, (uint32_t)pc.w};
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          const int v = (i0 + b < n) ? (int)(int8_t)(wd[b >> 2] >> (8 * (b & 3))) : 0;
          s += abs(v);
          if (v > 0) pos |= 1ull << (q * 16 + b);
          if (v < 0) neg |= 1ull << (q * 16 + b);
        }
      }
    } else {
      for (int b = 0; b < 64; ++b) {
        int i = w * 64 + b;
        if (i >= n) break;
        int v = g[i];
        s += abs(v);
        if (v > 0) pos |= 1ull << b;
        if (v < 0) neg |= 1ull << b;
      }
    }
    pm[w] = pos;
    pm[W + w] = neg;
  }
  bool v_ok = valid == nullptr || valid[k] != 0;
  l1[k] = v_ok ? s : kInvalidL1;
  if (v_ok) atomicAdd(&hist[s], 1u);
}

__global__ void prep_kernel(const int8_t* __restrict__ G, int64_t K, int n, int ldg, int W,
                            const uint8_t* __restrict__ valid, int32_t* __restrict__ l1,
                            uint64_t* __restrict__ masks, uint32_t* __restrict__ hist) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= K) return;
  prep_row(G, k, n, ldg, W, valid, l1, masks, hist);
}

// exclusive prefix over bins (one block of 1024); cursor receives a copy of
// the starts.  Warp w owns a contiguous segment; its lanes read it 32
// consecutive words at a time (coalesced): a first sweep sums the segment, the
// 32 segment sums are scanned by warp 0, and a second sweep scans the
// segment with warp shuffles and writes it.
__device__ __forceinline__ void bin_scan_block(const uint32_t* __restrict__ hist, int nbins,
                                               uint32_t* __restrict__ start, uint32_t* __restrict__ cursor) {
  __shared__ uint32_t s_warp[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  const int per = (nbins + nw - 1) / nw;
  const int b0 = wid * per, b1 = min(b0 + per, nbins);
  uint32_t sum = 0;
  for (int b = b0 + lane; b < b1; b += 32) sum += hist[b];
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) s_warp[wid] = sum;
  __syncthreads();
  if (wid == 0) {
    uint32_t x = lane < nw ? s_warp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_warp[lane] = x;  // inclusive over warps
  }
  __syncthreads();
  uint32_t run = wid > 0 ? s_warp[wid - 1] : 0;  // exclusive start of the segment
  for (int base = b0; base < b1; base += 32) {
    const int b = base + lane;
    const uint32_t v = b < b1 ? hist[b] : 0;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (b < b1) {
      start[b] = run + x - v;
      cursor[b] = run + x - v;
    }
    run += __shfl_sync(0xffffffffu, x, 31);
  }
}

__global__ void bin_scan_kernel(const uint32_t* __restrict__ hist, int nbins, uint32_t* __restrict__ start,
                                uint32_t* __restrict__ cursor) {
  bin_scan_block(hist, nbins, start, cursor);
}

// sorted arrays: row index, first mask words, folded signatures, l1
__device__ __forceinline__ void scatter_row(const int32_t* __restrict__ l1, const uint64_t* __restrict__ masks,
                                            int64_t k, int W, uint32_t* __restrict__ cursor,
                                            uint32_t* __restrict__ s_idx, uint64_t* __restrict__ s_pk,
                                            ulonglong2* __restrict__ s_sig, int32_t* __restrict__ s_l1) {
  if (l1[k] == kInvalidL1) return;
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
  s_l1[q] = l1[k];
}

__global__ void scatter_kernel(const int32_t* __restrict__ l1, const uint64_t* __restrict__ masks, int64_t K, int W,
                               uint32_t* __restrict__ cursor, uint32_t* __restrict__ s_idx,
                               uint64_t* __restrict__ s_pk, ulonglong2* __restrict__ s_sig,
                               int32_t* __restrict__ s_l1) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= K) return;
  scatter_row(l1, masks, k, W, cursor, s_idx, s_pk, s_sig, s_l1);
}

// ---- sign patterns -------------------------------------------------------------
//
// The pairwise test is pruned by the signs on kb key coordinates (the
// densest, at most 6).  Each row has a pattern there: t_b = 0 (zero), 1
// (positive), 2 (negative) on key coordinate b, index sum_b t_b 3^b.  h ⊑ g
// needs, on every key coordinate, h zero or of g's sign (and h zero where g
// is); -h ⊑ g the same with h's signs reversed.  So for g the candidate rows
// h lie in the 2^|nz(g)| lists whose pattern keeps a subset N of g's nonzero
// key coordinates, with g's signs (h ⊑ g) or the reversed ones (-h ⊑ g), and
// zero elsewhere.  Rows are split into the 3^kb pattern lists, each kept in l1
// order, and every row is compared only with the shorter rows of those
// lists.  Only pairs that cannot dominate are skipped, so the kept set is the
// one all pairs give.

constexpr int kKeyCoords = 6;
constexpr int kLists = 729;       // 3^kKeyCoords pattern lists
constexpr int kPartBlock = 1024;  // positions per block of the stable partition
constexpr int64_t kDensitySample = 16384;  // rows that choose the key coordinates

// per-coordinate nonzero counts of the valid rows among the first rows (64
// rows per block); any choice of key coordinates gives the same kept set, so
// a sample is enough to find the densest
__device__ __forceinline__ void coord_count_block(const int8_t* __restrict__ G, int64_t K, int n, int ldg,
                                                  const int32_t* __restrict__ l1, uint32_t* __restrict__ cnt,
                                                  int64_t bx) {
  extern __shared__ uint32_t s_cnt[];  // n
  for (int i = threadIdx.x; i < n; i += blockDim.x) s_cnt[i] = 0;
  __syncthreads();
  const int64_t r0 = bx * 64;
  for (int64_t e = threadIdx.x; e < 64 * (int64_t)n; e += blockDim.x) {
    const int64_t k = r0 + e / n;
    const int i = (int)(e % n);
    if (k < K && l1[k] != kInvalidL1 && G[k * ldg + i] != 0) atomicAdd(&s_cnt[i], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(&cnt[i], s_cnt[i]);
}

__global__ void coord_count_kernel(const int8_t* __restrict__ G, int64_t K, int n, int ldg,
                                   const int32_t* __restrict__ l1, uint32_t* __restrict__ cnt) {
  coord_count_block(G, K, n, ldg, l1, cnt, blockIdx.x);
}

// the kb densest coordinates (ties to the lower index); one block of 1024
__device__ __forceinline__ void select_keys_block(const uint32_t* __restrict__ cnt, int n, int kb,
                                                  int32_t* __restrict__ keys) {
  __shared__ unsigned long long s_best[32];
  __shared__ int s_taken[kKeyCoords];
  for (int b = 0; b < kb; ++b) {
    // count in the high word, ~index in the low word: the maximum is the
    // largest count with the lowest index
    unsigned long long best = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      bool taken = false;
      for (int c = 0; c < b; ++c) taken |= s_taken[c] == i;
      if (taken) continue;
      const unsigned long long v = ((unsigned long long)cnt[i] << 32) | (0xffffffffu - (uint32_t)i) | (1ull << 63);
      best = v > best ? v : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
      best = w > best ? w : best;
    }
    if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = s_best[w] > m ? s_best[w] : m;
      const int idx = (int)(0xffffffffu - (uint32_t)(m & 0xffffffffull));
      s_taken[b] = idx;
      keys[b] = idx;
    }
    __syncthreads();
  }
}

__global__ void select_keys_kernel(const uint32_t* __restrict__ cnt, int n, int kb, int32_t* __restrict__ keys) {
  select_keys_block(cnt, n, kb, keys);
}

// pattern list of the row at sorted position q
__device__ __forceinline__ void key_row(const int8_t* __restrict__ G, int ldg, const uint32_t* __restrict__ s_idx,
                                        int64_t q, const int32_t* __restrict__ keys, int kb,
                                        uint16_t* __restrict__ s_list) {
  const int8_t* g = G + (int64_t)s_idx[q] * ldg;
  int idx = 0, p3 = 1;
  for (int b = 0; b < kb; ++b) {
    const int v = g[keys[b]];
    idx += (v > 0 ? 1 : (v < 0 ? 2 : 0)) * p3;
    p3 *= 3;
  }
  s_list[q] = (uint16_t)idx;
}

__global__ void key_kernel(const int8_t* __restrict__ G, int ldg, const uint32_t* __restrict__ s_idx, int64_t nvalid,
                           const int32_t* __restrict__ keys, int kb, uint16_t* __restrict__ s_list) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nvalid) return;
  key_row(G, ldg, s_idx, q, keys, kb, s_list);
}

// stable partition by list, step 1: counts per (list, block of positions)
__device__ __forceinline__ void part_count_block(const uint16_t* __restrict__ s_list, int64_t nvalid, int nlists,
                                                 int nblk, uint32_t* __restrict__ bc, int64_t bx) {
  __shared__ uint32_t s_c[kLists];
  for (int L = threadIdx.x; L < nlists; L += blockDim.x) s_c[L] = 0;
  __syncthreads();
  const int64_t q = bx * kPartBlock + threadIdx.x;
  if (q < nvalid) atomicAdd(&s_c[s_list[q]], 1u);
  __syncthreads();
  for (int L = threadIdx.x; L < nlists; L += blockDim.x) bc[(int64_t)L * nblk + bx] = s_c[L];
}

__global__ void part_count_kernel(const uint16_t* __restrict__ s_list, int64_t nvalid, int nlists, int nblk,
                                  uint32_t* __restrict__ bc) {
  part_count_block(s_list, nvalid, nlists, nblk, bc, blockIdx.x);
}

// step 2 (one warp per block of positions, in position order): rank among
// the earlier rows of the same list, then move the row's sorted data
__device__ __forceinline__ void part_scatter_block(const uint16_t* __restrict__ s_list, int64_t nvalid, int nlists,
                                                   int nblk, const uint32_t* __restrict__ boff,
                                                   const uint32_t* __restrict__ s_idx, const uint64_t* __restrict__ s_pk,
                                                   const ulonglong2* __restrict__ s_sig,
                                                   const int32_t* __restrict__ s_l1, uint32_t* __restrict__ p_idx,
                                                   uint64_t* __restrict__ p_pk, ulonglong2* __restrict__ p_sig,
                                                   int32_t* __restrict__ p_l1, int64_t bx) {
  __shared__ uint32_t s_run[kLists];
  const int lane = threadIdx.x;
  for (int L = lane; L < nlists; L += 32) s_run[L] = boff[(int64_t)L * nblk + bx];
  __syncwarp();
  for (int it = 0; it < kPartBlock / 32; ++it) {
    const int64_t q = bx * kPartBlock + it * 32 + lane;
    const int L = q < nvalid ? (int)s_list[q] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, L);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1));
    uint32_t dst = 0;
    if (L >= 0) dst = s_run[L] + rank;
    __syncwarp();
    if (L >= 0 && (32 - __clz(peers)) - 1 == lane) s_run[L] += __popc(peers);
    __syncwarp();
    if (L >= 0) {
      p_idx[dst] = s_idx[q];
      p_pk[dst] = s_pk[q];
      p_sig[dst] = s_sig[q];
      p_l1[dst] = s_l1[q];
    }
  }
}

__global__ void part_scatter_kernel(const uint16_t* __restrict__ s_list, int64_t nvalid, int nlists, int nblk,
                                    const uint32_t* __restrict__ boff, const uint32_t* __restrict__ s_idx,
                                    const uint64_t* __restrict__ s_pk, const ulonglong2* __restrict__ s_sig,
                                    const int32_t* __restrict__ s_l1, uint32_t* __restrict__ p_idx,
                                    uint64_t* __restrict__ p_pk, ulonglong2* __restrict__ p_sig,
                                    int32_t* __restrict__ p_l1) {
  part_scatter_block(s_list, nvalid, nlists, nblk, boff, s_idx, s_pk, s_sig, s_l1, p_idx, p_pk, p_sig, p_l1,
                     blockIdx.x);
}

// list starts: lstart[L] = boff[L * nblk], lstart[nlists] = nvalid
__global__ void list_start_kernel(const uint32_t* __restrict__ boff, int nlists, int nblk, int64_t nvalid,
                                  uint32_t* __restrict__ lstart) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L < nlists) lstart[L] = boff[(int64_t)L * nblk];
  if (L == nlists) lstart[L] = (uint32_t)nvalid;
}

constexpr int kTile = 256;

__device__ __forceinline__ bool magnitudes_fit(const int8_t* h, const int8_t* g, int n) {
  for (int i = 0; i < n; ++i)
    if (abs((int)h[i]) > abs((int)g[i])) return false;
  return true;
}

// full test of h against g once the prefilters passed
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

constexpr int kChunk = 4096;  // rows of a source list scanned by one block

// Work unit (blockIdx.x, .y, .z): the up to 256 rows of g-block x (a run of
// one pattern list) against chunk z of one source list.  y = o 2^kb + N: N
// the key coordinates where the source rows are nonzero (a subset of g's
// nonzero key coordinates, else the unit is empty), o = 0 for h ⊑ g (g's
// signs) and o = 1 for -h ⊑ g (reversed signs); N = 0 takes both
// orientations at once.  Lists are in l1 order, so a row stops at the first
// source row that is not shorter.  Prefilters per pair: sign masks of
// coordinates 0..31 packed in one word (pos | neg << 32), then the folded
// 64-bit signatures of all coordinates, before the full test.  A dominated
// row gets dom[k] = 1 (several units may write it).
__device__ __forceinline__ void dominance_block(const int8_t* __restrict__ G, int n, int ldg, int W,
                                                const uint64_t* __restrict__ masks, const int4 gb,
                                                const uint32_t* __restrict__ lstart, int kb,
                                                const uint32_t* __restrict__ p_idx, const uint64_t* __restrict__ p_pk,
                                                const ulonglong2* __restrict__ p_sig, const int32_t* __restrict__ p_l1,
                                                uint8_t* __restrict__ dom, int by, int bz) {
  __shared__ int s_maxl1;
  const int nsub = 1 << kb;
  if (by >= 2 * nsub) return;  // batch: a unit beyond this instance's orientations and subsets
  const int o = by / nsub, N = by % nsub;
  // g's pattern digits; the source pattern keeps digits in N (reversed for o = 1)
  int nzmask = 0, S = 0;
  {
    int rest = gb.z, p3 = 1;
    for (int b = 0; b < kb; ++b) {
      const int t = rest % 3;
      rest /= 3;
      if (t != 0) nzmask |= 1 << b;
      if ((N >> b) & 1) S += (o == 0 ? t : 3 - t) * p3;
      p3 *= 3;
    }
  }
  if ((N & ~nzmask) != 0 || (N == 0 && o == 1)) return;  // uniform over the block
  const int mode = N == 0 ? 3 : (o == 0 ? 1 : 2);  // bit 0: h ⊑ g, bit 1: -h ⊑ g
  const uint32_t lo = lstart[S] + (uint32_t)bz * (uint32_t)kChunk, s_end = lstart[S + 1];
  if (lo >= s_end) return;
  const uint32_t hi = lo + kChunk < s_end ? lo + kChunk : s_end;
  const bool mine = (int)threadIdx.x < gb.y;
  const uint32_t q = (uint32_t)gb.x + threadIdx.x;
  const int32_t gl1 = mine ? p_l1[q] : 0;
  if (threadIdx.x == 0) s_maxl1 = 0;
  __syncthreads();
  if (mine) atomicMax(&s_maxl1, gl1);
  __syncthreads();
  if (p_l1[lo] >= s_maxl1) return;  // no source row of the chunk is shorter than any g
  const uint32_t k = mine ? p_idx[q] : 0;
  const uint64_t pk = mine ? p_pk[q] : 0;
  const uint32_t np = ~(uint32_t)pk, nn = ~(uint32_t)(pk >> 32);
  const ulonglong2 gs = mine ? p_sig[q] : make_ulonglong2(0, 0);
  const uint64_t gsp = ~gs.x, gsn = ~gs.y;
  const bool want_same = (mode & 1) != 0, want_flip = (mode & 2) != 0;
  if (!mine || dom[k]) return;
  // every thread of the block reads the same source rows at the same time:
  // the loads are L1 broadcasts, and no block barrier is needed; four rows'
  // words are loaded at once
  for (uint32_t h0 = lo; h0 < hi; h0 += 4) {
    int32_t l1v[4];
    uint64_t pkv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool in = h0 + u < hi;
      l1v[u] = in ? p_l1[h0 + u] : 0x7fffffff;
      pkv[u] = in ? p_pk[h0 + u] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (l1v[u] >= gl1) return;  // the rest of the list is not shorter (or past its end)
      const uint32_t hp = (uint32_t)pkv[u], hn = (uint32_t)(pkv[u] >> 32);
      const bool cand = (want_same && ((hp & np) | (hn & nn)) == 0) || (want_flip && ((hp & nn) | (hn & np)) == 0);
      if (!cand) continue;
      const uint32_t h = h0 + u;
      const ulonglong2 hs = p_sig[h];
      const bool cand2 = (want_same && ((hs.x & gsp) | (hs.y & gsn)) == 0) ||
                         (want_flip && ((hs.x & gsn) | (hs.y & gsp)) == 0);
      if (cand2 && dominates(G, n, ldg, W, masks, p_idx[h], k)) {
        dom[k] = 1;
        return;
      }
    }
  }
}

__global__ void dominance_kernel(const int8_t* __restrict__ G, int n, int ldg, int W, const uint64_t* __restrict__ masks,
                                 const int4* __restrict__ gblk, const uint32_t* __restrict__ lstart, int kb,
                                 const uint32_t* __restrict__ p_idx, const uint64_t* __restrict__ p_pk,
                                 const ulonglong2* __restrict__ p_sig, const int32_t* __restrict__ p_l1,
                                 uint8_t* __restrict__ dom) {
  dominance_block(G, n, ldg, W, masks, gblk[blockIdx.x], lstart, kb, p_idx, p_pk, p_sig, p_l1, dom, blockIdx.y,
                  blockIdx.z);
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

__device__ __forceinline__ void count_kept_block(const uint8_t* __restrict__ keep, int64_t K,
                                                 uint32_t* __restrict__ block_count, int64_t bx) {
  __shared__ uint32_t s_c;
  if (threadIdx.x == 0) s_c = 0;
  __syncthreads();
  int64_t k = bx * (int64_t)kCompact + threadIdx.x;
  unsigned bal = __ballot_sync(0xffffffffu, k < K && keep[k]);
  if ((threadIdx.x & 31) == 0) atomicAdd(&s_c, (uint32_t)__popc(bal));
  __syncthreads();
  if (threadIdx.x == 0) block_count[bx] = s_c;
}

__global__ void count_kept_kernel(const uint8_t* __restrict__ keep, int64_t K, uint32_t* __restrict__ block_count) {
  count_kept_block(keep, K, block_count, blockIdx.x);
}

__device__ __forceinline__ void write_kept_block(const int8_t* __restrict__ G, int64_t K, int ldg,
                                                 const uint8_t* __restrict__ keep,
                                                 const uint32_t* __restrict__ block_start, int8_t* __restrict__ out,
                                                 int64_t bx) {
  __shared__ uint32_t s_warp[kCompact / 32];
  int64_t k = bx * (int64_t)kCompact + threadIdx.x;
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
  int64_t dst = (int64_t)block_start[bx] + s_warp[wid] + __popc(bal & ((1u << lane) - 1));
  const uint4* src = reinterpret_cast<const uint4*>(G + k * ldg);
  uint4* d4 = reinterpret_cast<uint4*>(out + dst * ldg);
  for (int c = 0; c < ldg / 16; ++c) d4[c] = src[c];
}

__global__ void write_kept_kernel(const int8_t* __restrict__ G, int64_t K, int ldg, const uint8_t* __restrict__ keep,
                                  const uint32_t* __restrict__ block_start, int8_t* __restrict__ out) {
  write_kept_block(G, K, ldg, keep, block_start, out, blockIdx.x);
}

int64_t l1_bins(int32_t n) { return (int64_t)127 * n + 1; }

}  // namespace

extern "C" size_t mape_kernel_test_workspace_bytes(int32_t m, int32_t n) {
  if (m <= 0 || n <= 0) return 0;
  mape_detail::Sizer s;
  s.take<unsigned long long>(1);             // failure counter
  s.take<uint32_t>((size_t)m + 1);           // nonzeros per row of A
  s.take<uint32_t>((size_t)m + 1);           // row starts
  s.take<uint16_t>((size_t)m * n);           // column indices
  s.take<int32_t>((size_t)m * n);            // values
  return s.bytes();
}

extern "C" int mape_kernel_test(const int32_t* A, int32_t m, int32_t n, const int8_t* G, int64_t K, int32_t ldg,
                                uint8_t* ok, int64_t* fail_count, void* workspace, size_t workspace_bytes,
                                void* stream) {
  using namespace mape_detail;
  if (!A || m <= 0 || n <= 0 || ldg < n || ldg % 16 != 0 || K < 0 || !fail_count || (K > 0 && (!G || !ok)))
    return MAPE_ERR_INVALID_ARG;
  if (n > 4096 || ldg > kCsrMaxRow) return MAPE_ERR_SHAPE;
  *fail_count = 0;
  if (K == 0) return MAPE_OK;
  Carver cv(workspace, workspace_bytes);
  unsigned long long* d_fail = cv.take<unsigned long long>(1);
  uint32_t* rowcnt = cv.take<uint32_t>((size_t)m + 1);
  uint32_t* rowptr = cv.take<uint32_t>((size_t)m + 1);
  uint16_t* col = cv.take<uint16_t>((size_t)m * n);
  int32_t* val = cv.take<int32_t>((size_t)m * n);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  const int stage8 = ((int64_t)m * ldg <= 48 * 1024 && ldg <= kMaxRegRow) ? 1 : 0;
  MAPE_CUDA_TRY(cudaMemsetAsync(d_fail, 0, sizeof(unsigned long long), st));
  if (stage8) {
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(K, 128), 152 * 4);
    mape_detail::launch(kernel_test_kernel, grid, 128, (size_t)m * ldg, st, A, m, n, G, K, ldg, stage8, ok, d_fail);
  } else {
    const unsigned gw = (unsigned)ceil_div((int64_t)m * 32, 256);
    MAPE_CUDA_TRY(cudaMemsetAsync(rowcnt, 0, sizeof(uint32_t) * ((size_t)m + 1), st));
    mape_detail::launch(csr_count_kernel, gw, 256, 0, st, A, m, n, rowcnt);
    // exclusive prefix over m + 1 entries: entry m = nnz(A)
    mape_detail::launch(bin_scan_kernel, 1, 1024, 0, st, rowcnt, m + 1, rowptr, rowptr);
    mape_detail::launch(csr_fill_kernel, gw, 256, 0, st, A, m, n, rowptr, col, val);
    const size_t smem = (size_t)kCsrWarps * kCsrRows * ldg;
    if (smem > 48 * 1024) {
      size_t lim = 0;
      const int rc = allow_max_dynamic_smem((const void*)kernel_test_csr_kernel, &lim);
      if (rc != MAPE_OK) return rc;
      if (smem > lim) return MAPE_ERR_SHAPE;
    }
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(K, (int64_t)kCsrWarps * kCsrRows), 152 * 4);
    mape_detail::launch(kernel_test_csr_kernel, grid, 32 * kCsrWarps, smem, st, rowptr, col, val, m, G, K, ldg, ok,
                        d_fail);
  }
  MAPE_LAUNCH_CHECK();
  unsigned long long f = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&f, d_fail, sizeof(f), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  *fail_count = (int64_t)f;
  return MAPE_OK;
}

// ---- a9 for many instances at once ---------------------------------------------
//
// Every instance's A goes to compressed rows (one launch per kernel over the
// rows of all the A's, one scan block per instance), then one launch tests
// the candidate rows of all instances, a warp per four rows finding its
// instance by binary search over the launch's prefix table.  The compressed-row test is
// exact for every int32 A, so each instance's flags and count equal those of
// its own mape_kernel_test (whichever path that takes).

namespace {

struct KtView {
  const int32_t* A;
  int m, n, ldg;
  const int8_t* G;
  int64_t K;
  uint8_t* ok;
  uint32_t *rowcnt, *rowptr;
  uint16_t* col;
  int32_t* val;
};

__device__ __forceinline__ int find_inst(const int64_t* __restrict__ prefix, int count, int64_t x) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// prefix: rows of the A's (a warp per row); phase 0 counts, 1 fills
__global__ void csr_batch_kernel(const KtView* __restrict__ v, const int64_t* __restrict__ prefix, int count,
                                 int phase) {
  const int64_t wr = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (wr >= prefix[count]) return;  // warp-uniform
  const int i = find_inst(prefix, count, wr);
  const KtView& d = v[i];
  const int r = (int)(wr - prefix[i]);
  const int lane = threadIdx.x & 31;
  const int32_t* a = d.A + (int64_t)r * d.n;
  if (phase == 0) {
    uint32_t c = 0;
    for (int j = lane; j < d.n; j += 32) c += a[j] != 0;
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if (lane == 0) d.rowcnt[r] = c;
    return;
  }
  uint32_t pos = d.rowptr[r];
  for (int j0 = 0; j0 < d.n; j0 += 32) {
    const int j = j0 + lane;
    const int x = j < d.n ? a[j] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, x != 0);
    if (x != 0) {
      const uint32_t q = pos + __popc(bal & ((1u << lane) - 1));
      d.col[q] = (uint16_t)j;
      d.val[q] = x;
    }
    pos += __popc(bal);
  }
}

// one block per instance: exclusive prefix of its row counts (entry m = nnz)
__global__ void csr_scan_batch_kernel(const KtView* __restrict__ v) {
  const KtView& d = v[blockIdx.x];
  __shared__ uint32_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base <= d.m; base += blockDim.x) {
    const int r = base + threadIdx.x;
    uint32_t x = r < d.m ? d.rowcnt[r] : 0;
    // block-wide inclusive scan of x by warp shuffles and a pass over the warp sums
    __shared__ uint32_t s_w[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t y = x;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += t;
    }
    if (lane == 31) s_w[wid] = y;
    __syncthreads();
    if (wid == 0) {
      uint32_t z = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += t;
      }
      s_w[lane] = z;
    }
    __syncthreads();
    const uint32_t incl = y + (wid > 0 ? s_w[wid - 1] : 0) + s_carry;
    if (r <= d.m) d.rowptr[r] = incl - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = incl;
    __syncthreads();
  }
}

// prefix: groups of kCsrRows candidate rows of every instance (a warp per
// group); dynamic shared memory kCsrWarps x kCsrRows rows of max_ldg bytes
__global__ void __launch_bounds__(32 * kCsrWarps)
kernel_test_batch_kernel(const KtView* __restrict__ v, const int64_t* __restrict__ prefix, int count,
                         int max_ldg, unsigned long long* __restrict__ fails) {
  extern __shared__ __align__(16) int8_t s_rows[];
  const int w = threadIdx.x >> 5;
  const int64_t g = blockIdx.x * (int64_t)kCsrWarps + w;
  if (g >= prefix[count]) return;  // warp-uniform
  const int i = find_inst(prefix, count, g);
  const KtView& d = v[i];
  const int64_t k0 = (g - prefix[i]) * kCsrRows;
  const int cnt = (int)(d.K - k0 < kCsrRows ? d.K - k0 : kCsrRows);
  csr_test_rows(d.rowptr, d.col, d.val, d.m, d.G, k0, cnt, d.ldg, s_rows + (size_t)w * kCsrRows * max_ldg, d.ok,
                fails + i);
}

}  // namespace

extern "C" size_t mape_kernel_test_batch_workspace_bytes(int32_t count) {
  if (count <= 0) return 0;
  mape_detail::Sizer s;
  s.take<KtView>((size_t)count);
  s.take<int64_t>((size_t)2 * (count + 1));    // prefix tables: rows of A, candidate rows
  s.take<unsigned long long>((size_t)count);   // failure counters
  return s.bytes();
}

extern "C" int mape_kernel_test_batch(mape_kernel_test_item* items, int32_t count, void* workspace,
                                      size_t workspace_bytes, void* stream) {
  using namespace mape_detail;
  if (!items || count <= 0) return MAPE_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const mape_kernel_test_item& it = items[i];
    if (!it.A || it.m <= 0 || it.n <= 0 || it.ldg < it.n || it.ldg % 16 != 0 || it.K < 0 ||
        (it.K > 0 && (!it.G || !it.ok)))
      return MAPE_ERR_INVALID_ARG;
    if (it.n > 4096 || it.ldg > kCsrMaxRow) return MAPE_ERR_SHAPE;
  }
  Carver bc(workspace, workspace_bytes);
  KtView* d_views = bc.take<KtView>((size_t)count);
  int64_t* d_px = bc.take<int64_t>((size_t)2 * (count + 1));
  unsigned long long* d_fail = bc.take<unsigned long long>((size_t)count);
  if (!bc.ok) return MAPE_ERR_CAPACITY;
  std::vector<KtView> v((size_t)count);
  std::vector<int64_t> px((size_t)2 * (count + 1), 0);
  int max_ldg = 16;
  for (int i = 0; i < count; ++i) {
    mape_kernel_test_item& it = items[i];
    it.fail_count = 0;
    KtView& d = v[(size_t)i];
    d = KtView{it.A, it.m, it.n, it.ldg, it.G, it.K, it.ok, nullptr, nullptr, nullptr, nullptr};
    // the compressed rows in the instance's own workspace, carved as mape_kernel_test carves it
    Carver cv(it.workspace, it.workspace_bytes);
    cv.take<unsigned long long>(1);
    d.rowcnt = cv.take<uint32_t>((size_t)it.m + 1);
    d.rowptr = cv.take<uint32_t>((size_t)it.m + 1);
    d.col = cv.take<uint16_t>((size_t)it.m * it.n);
    d.val = cv.take<int32_t>((size_t)it.m * it.n);
    if (!cv.ok) return MAPE_ERR_CAPACITY;
    px[(size_t)i + 1] = px[(size_t)i] + it.m;
    px[(size_t)(count + 1) + i + 1] = px[(size_t)(count + 1) + i] + (it.K + kCsrRows - 1) / kCsrRows;
    max_ldg = std::max(max_ldg, it.ldg);
  }
  const int64_t arows = px[(size_t)count], crows = px[(size_t)2 * count + 1];
  cudaStream_t st = as_stream(stream);
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_views, v.data(), sizeof(KtView) * count, cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_px, px.data(), sizeof(int64_t) * px.size(), cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(d_fail, 0, sizeof(unsigned long long) * count, st));
  const unsigned ga = (unsigned)ceil_div(arows * 32, 256);
  launch(csr_batch_kernel, ga, 256, 0, st, (const KtView*)d_views, (const int64_t*)d_px, (int)count, 0);
  launch(csr_scan_batch_kernel, (unsigned)count, 1024, 0, st, (const KtView*)d_views);
  launch(csr_batch_kernel, ga, 256, 0, st, (const KtView*)d_views, (const int64_t*)d_px, (int)count, 1);
  if (crows > 0) {  // crows: groups of kCsrRows candidate rows
    const size_t smem = (size_t)kCsrWarps * kCsrRows * max_ldg;
    if (smem > 48 * 1024) {
      size_t lim = 0;
      const int rc = allow_max_dynamic_smem((const void*)kernel_test_batch_kernel, &lim);
      if (rc != MAPE_OK) return rc;
      if (smem > lim) return MAPE_ERR_SHAPE;
    }
    launch(kernel_test_batch_kernel, (unsigned)ceil_div(crows, kCsrWarps), 32 * kCsrWarps, smem, st,
           (const KtView*)d_views, (const int64_t*)(d_px + count + 1), (int)count, max_ldg, d_fail);
  }
  MAPE_LAUNCH_CHECK();
  std::vector<unsigned long long> f((size_t)count, 0);
  MAPE_CUDA_TRY(cudaMemcpyAsync(f.data(), d_fail, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i) items[i].fail_count = (int64_t)f[(size_t)i];
  return MAPE_OK;
}

extern "C" size_t mape_minimal_workspace_bytes(int64_t K, int32_t n) {
  using namespace mape_detail;
  if (K < 0 || n <= 0) return 0;
  int W = (n + 63) / 64;
  int64_t nb = l1_bins(n);
  const int64_t nblk_part = ceil_div(K, kPartBlock);
  Sizer s;
  s.take<int32_t>((size_t)K);                 // l1
  s.take<uint64_t>((size_t)K * 2 * W);        // masks
  s.take<uint32_t>((size_t)nb);               // histogram
  s.take<uint32_t>((size_t)nb);               // bin starts
  s.take<uint32_t>((size_t)nb);               // cursors
  s.take<uint32_t>((size_t)K);                // l1-sorted: row index
  s.take<uint64_t>((size_t)K);                //   packed sign masks
  s.take<ulonglong2>((size_t)K);              //   folded signatures
  s.take<int32_t>((size_t)K);                 //   l1
  s.take<uint16_t>((size_t)K);                //   list
  s.take<uint32_t>((size_t)K);                // partitioned by list: row index
  s.take<uint64_t>((size_t)K);                //   packed sign masks
  s.take<ulonglong2>((size_t)K);              //   folded signatures
  s.take<int32_t>((size_t)K);                 //   l1
  s.take<uint32_t>((size_t)n);                // coordinate nonzero counts
  s.take<int32_t>((size_t)kKeyCoords);        // key coordinates
  s.take<uint32_t>((size_t)kLists * nblk_part);      // counts per (list, block)
  s.take<uint32_t>((size_t)kLists * nblk_part + 1);  // their exclusive prefix
  s.take<uint32_t>((size_t)kLists + 1);              // list starts
  s.take<int4>((size_t)ceil_div(K, kTile) + kLists);  // g-blocks
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
  const int64_t nblk_part_max = ceil_div(K, kPartBlock);
  const int kb = n < kKeyCoords ? n : kKeyCoords;
  int nlists = 1;
  for (int b = 0; b < kb; ++b) nlists *= 3;
  Carver cv(workspace, workspace_bytes);
  int32_t* l1 = cv.take<int32_t>((size_t)K);
  uint64_t* masks = cv.take<uint64_t>((size_t)K * 2 * W);
  uint32_t* hist = cv.take<uint32_t>((size_t)nb);
  uint32_t* start = cv.take<uint32_t>((size_t)nb);
  uint32_t* cursor = cv.take<uint32_t>((size_t)nb);
  uint32_t* s_idx = cv.take<uint32_t>((size_t)K);
  uint64_t* s_pk = cv.take<uint64_t>((size_t)K);
  ulonglong2* s_sig = cv.take<ulonglong2>((size_t)K);
  int32_t* s_l1 = cv.take<int32_t>((size_t)K);
  uint16_t* s_list = cv.take<uint16_t>((size_t)K);
  uint32_t* p_idx = cv.take<uint32_t>((size_t)K);
  uint64_t* p_pk = cv.take<uint64_t>((size_t)K);
  ulonglong2* p_sig = cv.take<ulonglong2>((size_t)K);
  int32_t* p_l1 = cv.take<int32_t>((size_t)K);
  uint32_t* cnt = cv.take<uint32_t>((size_t)n);
  int32_t* keys = cv.take<int32_t>((size_t)kKeyCoords);
  uint32_t* bc = cv.take<uint32_t>((size_t)kLists * nblk_part_max);
  uint32_t* boff = cv.take<uint32_t>((size_t)kLists * nblk_part_max + 1);
  uint32_t* lstart = cv.take<uint32_t>((size_t)kLists + 1);
  int4* gblk = cv.take<int4>((size_t)ceil_div(K, kTile) + kLists);
  uint32_t* bcount = cv.take<uint32_t>((size_t)nblk + 1);
  uint32_t* bstart = cv.take<uint32_t>((size_t)nblk + 1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  MAPE_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nb, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(bcount, 0, sizeof(uint32_t) * (nblk + 1), st));
  MAPE_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * n, st));
  const unsigned g = (unsigned)ceil_div(K, kTile);
  mape_detail::launch(prep_kernel, g, kTile, 0, st, G, K, n, ldg, W, valid, l1, masks, hist);
  mape_detail::launch(bin_scan_kernel, 1, 1024, 0, st, hist, (int)nb, start, cursor);
  mape_detail::launch(scatter_kernel, g, kTile, 0, st, l1, masks, K, W, cursor, s_idx, s_pk, s_sig, s_l1);
  mape_detail::launch(clear_keep_kernel, g, kTile, 0, st, keep, K);
  const int64_t K_sample = K < kDensitySample ? K : kDensitySample;
  mape_detail::launch(coord_count_kernel, (unsigned)ceil_div(K_sample, 64), 256, sizeof(uint32_t) * n, st, G, K_sample,
                      n, ldg, l1, cnt);
  mape_detail::launch(select_keys_kernel, 1, 1024, 0, st, cnt, n, kb, keys);
  MAPE_LAUNCH_CHECK();
  // number of valid rows = end of the last bin
  uint32_t last_start = 0, last_count = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&last_start, start + nb - 1, 4, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(&last_count, hist + nb - 1, 4, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  const int64_t nvalid = (int64_t)last_start + last_count;
  if (nvalid > 0) {
    // pattern lists, each in l1 order (stable partition of the l1 order)
    const int nblk_part = (int)ceil_div(nvalid, kPartBlock);
    mape_detail::launch(key_kernel, (unsigned)ceil_div(nvalid, kTile), kTile, 0, st, G, ldg, s_idx, nvalid, keys, kb,
                        s_list);
    mape_detail::launch(part_count_kernel, (unsigned)nblk_part, kPartBlock, 0, st, s_list, nvalid, nlists, nblk_part,
                        bc);
    mape_detail::launch(bin_scan_kernel, 1, 1024, 0, st, bc, nlists * nblk_part, boff, boff);
    mape_detail::launch(part_scatter_kernel, (unsigned)nblk_part, 32, 0, st, s_list, nvalid, nlists, nblk_part, boff,
                        s_idx, s_pk, s_sig, s_l1, p_idx, p_pk, p_sig, p_l1);
    mape_detail::launch(list_start_kernel, (unsigned)ceil_div(nlists + 1, 256), 256, 0, st, boff, nlists, nblk_part,
                        nvalid, lstart);
    MAPE_LAUNCH_CHECK();
    std::vector<uint32_t> ls((size_t)nlists + 1);
    MAPE_CUDA_TRY(cudaMemcpyAsync(ls.data(), lstart, sizeof(uint32_t) * ls.size(), cudaMemcpyDeviceToHost, st));
    MAPE_CUDA_TRY(cudaStreamSynchronize(st));
    // g-blocks: runs of at most kTile rows of one list
    std::vector<int4> gb;
    uint32_t max_list = 0;
    for (int L = 0; L < nlists; ++L) {
      const uint32_t a = ls[L], b = ls[L + 1];
      max_list = std::max(max_list, b - a);
      for (uint32_t o = a; o < b; o += kTile) gb.push_back(make_int4((int)o, (int)std::min<uint32_t>(kTile, b - o), L, 0));
    }
    if (!gb.empty()) {
      MAPE_CUDA_TRY(cudaMemcpyAsync(gblk, gb.data(), sizeof(int4) * gb.size(), cudaMemcpyHostToDevice, st));
      const dim3 grid((unsigned)gb.size(), 2u << kb, (unsigned)ceil_div(max_list, kChunk));
      mape_detail::launch(dominance_kernel, grid, kTile, 0, st, G, n, ldg, W, masks, gblk, lstart, kb, p_idx, p_pk,
                          p_sig, p_l1, keep);
    }
  }
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

// ---- a11 for many instances at once --------------------------------------------
//
// Every kernel of the filter runs once over the rows (positions, blocks, g-
// blocks) of all instances, each thread or block finding its instance by
// binary search over the launch's prefix table; the dominance launch covers
// the g-blocks of all instances (each g-block carries its instance).  Every
// instance keeps its own arrays, carved from its own workspace as
// mape_minimal_filter carves them, so its kept set and output equal those of
// its own call.

namespace {

struct MinView {
  const int8_t* G;
  int64_t K;
  int n, ldg, W, kb, nlists, nblk_part;
  const uint8_t* valid;
  uint8_t* keep;
  int8_t* out;
  int64_t nb, nblk, K_sample, nvalid;
  int32_t* l1;
  uint64_t* masks;
  uint32_t *hist, *start, *cursor, *s_idx;
  uint64_t* s_pk;
  ulonglong2* s_sig;
  int32_t* s_l1;
  uint16_t* s_list;
  uint32_t* p_idx;
  uint64_t* p_pk;
  ulonglong2* p_sig;
  int32_t* p_l1;
  uint32_t* cnt;
  int32_t* keys;
  uint32_t *bc, *boff, *lstart;
  int4* gblk;
  uint32_t *bcount, *bstart;
};

// phase 0: l1 and masks; 1: l1-sorted arrays; 2: keep cleared; 3: keep = valid and not dominated
__global__ void min_rows_batch_kernel(const MinView* __restrict__ v, const int64_t* __restrict__ prefix, int count,
                                      int phase) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= prefix[count]) return;
  const int i = find_inst(prefix, count, t);
  const MinView& d = v[i];
  const int64_t k = t - prefix[i];
  if (phase == 0) prep_row(d.G, k, d.n, d.ldg, d.W, d.valid, d.l1, d.masks, d.hist);
  else if (phase == 1) scatter_row(d.l1, d.masks, k, d.W, d.cursor, d.s_idx, d.s_pk, d.s_sig, d.s_l1);
  else if (phase == 2) d.keep[k] = 0;
  else d.keep[k] = (d.l1[k] != kInvalidL1 && !d.keep[k]) ? 1 : 0;
}

// one block per instance: 0 the l1 bins, 1 the partition counts, 2 the kept-row counts
__global__ void min_scan_batch_kernel(const MinView* __restrict__ v, int which) {
  const MinView& d = v[blockIdx.x];
  if (d.K == 0) return;
  if (which == 0) bin_scan_block(d.hist, (int)d.nb, d.start, d.cursor);
  else if (which == 1) {
    if (d.nvalid > 0) bin_scan_block(d.bc, d.nlists * d.nblk_part, d.boff, d.boff);
  } else {
    bin_scan_block(d.bcount, (int)d.nblk + 1, d.bstart, d.bstart);
  }
}

// per instance (one block each): the key coordinates; then the valid-row count
__global__ void min_keys_batch_kernel(const MinView* __restrict__ v, int64_t* __restrict__ nvalid) {
  const MinView& d = v[blockIdx.x];
  if (d.K == 0) {
    if (threadIdx.x == 0) nvalid[blockIdx.x] = 0;
    return;
  }
  select_keys_block(d.cnt, d.n, d.kb, d.keys);
  if (threadIdx.x == 0) nvalid[blockIdx.x] = (int64_t)d.start[d.nb - 1] + d.hist[d.nb - 1];
}

// prefix: blocks of 64 sampled rows
__global__ void min_coord_batch_kernel(const MinView* __restrict__ v, const int64_t* __restrict__ prefix, int count) {
  const int i = find_inst(prefix, count, blockIdx.x);
  const MinView& d = v[i];
  coord_count_block(d.G, d.K_sample, d.n, d.ldg, d.l1, d.cnt, blockIdx.x - prefix[i]);
}

// prefix: valid rows (pattern list of each)
__global__ void min_key_rows_batch_kernel(const MinView* __restrict__ v, const int64_t* __restrict__ prefix,
                                          int count) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= prefix[count]) return;
  const int i = find_inst(prefix, count, t);
  const MinView& d = v[i];
  key_row(d.G, d.ldg, d.s_idx, t - prefix[i], d.keys, d.kb, d.s_list);
}

// prefix: partition blocks; phase 0 counts, 1 scatters
__global__ void min_part_batch_kernel(const MinView* __restrict__ v, const int64_t* __restrict__ prefix, int count,
                                      int phase) {
  const int i = find_inst(prefix, count, blockIdx.x);
  const MinView& d = v[i];
  const int64_t b = blockIdx.x - prefix[i];
  if (phase == 0) part_count_block(d.s_list, d.nvalid, d.nlists, d.nblk_part, d.bc, b);
  else
    part_scatter_block(d.s_list, d.nvalid, d.nlists, d.nblk_part, d.boff, d.s_idx, d.s_pk, d.s_sig, d.s_l1, d.p_idx,
                       d.p_pk, d.p_sig, d.p_l1, b);
}

// prefix: list starts (nlists + 1 per instance)
__global__ void min_list_start_batch_kernel(const MinView* __restrict__ v, const int64_t* __restrict__ prefix,
                                            int count) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= prefix[count]) return;
  const int i = find_inst(prefix, count, t);
  const MinView& d = v[i];
  const int L = (int)(t - prefix[i]);
  d.lstart[L] = L < d.nlists ? d.boff[(int64_t)L * d.nblk_part] : (uint32_t)d.nvalid;
}

// the g-blocks of all instances (.w: instance)
__global__ void min_dominance_batch_kernel(const MinView* __restrict__ v, const int4* __restrict__ gblk) {
  const int4 gb = gblk[blockIdx.x];
  const MinView& d = v[gb.w];
  dominance_block(d.G, d.n, d.ldg, d.W, d.masks, gb, d.lstart, d.kb, d.p_idx, d.p_pk, d.p_sig, d.p_l1, d.keep,
                  blockIdx.y, blockIdx.z);
}

// prefix: compaction blocks; phase 0 counts, 1 writes
__global__ void min_compact_batch_kernel(const MinView* __restrict__ v, const int64_t* __restrict__ prefix, int count,
                                         int phase) {
  const int i = find_inst(prefix, count, blockIdx.x);
  const MinView& d = v[i];
  const int64_t b = blockIdx.x - prefix[i];
  if (phase == 0) count_kept_block(d.keep, d.K, d.bcount, b);
  else write_kept_block(d.G, d.K, d.ldg, d.keep, d.bstart, d.out, b);
}

int64_t min_gblocks_cap(int64_t K, int n) {
  const int kb = n < kKeyCoords ? n : kKeyCoords;
  int nlists = 1;
  for (int b = 0; b < kb; ++b) nlists *= 3;
  return mape_detail::ceil_div(K, kTile) + nlists;
}

}  // namespace

extern "C" size_t mape_minimal_filter_batch_workspace_bytes(const mape_minimal_item* items, int32_t count) {
  if (!items || count <= 0) return 0;
  int64_t gb = 0;
  for (int i = 0; i < count; ++i) gb += items[i].K > 0 && items[i].n > 0 ? min_gblocks_cap(items[i].K, items[i].n) : 0;
  mape_detail::Sizer s;
  s.take<MinView>((size_t)count);
  s.take<int64_t>((size_t)6 * (count + 1));  // prefix tables
  s.take<int64_t>((size_t)count);            // valid rows per instance
  s.take<int4>((size_t)(gb > 0 ? gb : 1));   // g-blocks of all instances
  return s.bytes();
}

extern "C" int mape_minimal_filter_batch(mape_minimal_item* items, int32_t count, void* workspace,
                                         size_t workspace_bytes, void* stream) {
  using namespace mape_detail;
  if (!items || count <= 0) return MAPE_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const mape_minimal_item& it = items[i];
    if (it.K < 0 || it.n <= 0 || it.ldg < it.n || it.ldg % 16 != 0 || (it.K > 0 && (!it.G || !it.keep || !it.out)))
      return MAPE_ERR_INVALID_ARG;
    if (it.n > 4096 || it.K >= ((int64_t)1 << 31)) return MAPE_ERR_SHAPE;
  }
  int64_t gb_cap = 0;
  for (int i = 0; i < count; ++i) gb_cap += items[i].K > 0 ? min_gblocks_cap(items[i].K, items[i].n) : 0;
  Carver bc(workspace, workspace_bytes);
  MinView* d_views = bc.take<MinView>((size_t)count);
  int64_t* d_px = bc.take<int64_t>((size_t)6 * (count + 1));
  int64_t* d_nvalid = bc.take<int64_t>((size_t)count);
  int4* d_gblk = bc.take<int4>((size_t)(gb_cap > 0 ? gb_cap : 1));
  if (!bc.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  const int n1 = count + 1;
  std::vector<int64_t> px((size_t)6 * n1, 0);
  auto prefix = [&](int t, auto units) -> int64_t {
    int64_t* p = px.data() + (size_t)t * n1;
    p[0] = 0;
    for (int i = 0; i < count; ++i) p[i + 1] = p[i] + units(i);
    return p[count];
  };
  auto dpx = [&](int t) -> const int64_t* { return d_px + (size_t)t * n1; };
  std::vector<MinView> v((size_t)count);
  int max_n = 1;
  for (int i = 0; i < count; ++i) {
    mape_minimal_item& it = items[i];
    it.K_out = 0;
    MinView& d = v[(size_t)i];
    d = MinView{};
    d.G = it.G; d.K = it.K; d.n = it.n; d.ldg = it.ldg; d.valid = it.valid; d.keep = it.keep; d.out = it.out;
    if (it.K == 0) continue;
    const int64_t K = it.K;
    const int n = it.n;
    d.W = (n + 63) / 64;
    d.nb = l1_bins(n);
    d.nblk = ceil_div(K, kCompact);
    const int64_t nblk_part_max = ceil_div(K, kPartBlock);
    d.kb = n < kKeyCoords ? n : kKeyCoords;
    d.nlists = 1;
    for (int b = 0; b < d.kb; ++b) d.nlists *= 3;
    d.K_sample = K < kDensitySample ? K : kDensitySample;
    max_n = std::max(max_n, n);
    // the same carve as mape_minimal_filter
    Carver cv(it.workspace, it.workspace_bytes);
    d.l1 = cv.take<int32_t>((size_t)K);
    d.masks = cv.take<uint64_t>((size_t)K * 2 * d.W);
    d.hist = cv.take<uint32_t>((size_t)d.nb);
    d.start = cv.take<uint32_t>((size_t)d.nb);
    d.cursor = cv.take<uint32_t>((size_t)d.nb);
    d.s_idx = cv.take<uint32_t>((size_t)K);
    d.s_pk = cv.take<uint64_t>((size_t)K);
    d.s_sig = cv.take<ulonglong2>((size_t)K);
    d.s_l1 = cv.take<int32_t>((size_t)K);
    d.s_list = cv.take<uint16_t>((size_t)K);
    d.p_idx = cv.take<uint32_t>((size_t)K);
    d.p_pk = cv.take<uint64_t>((size_t)K);
    d.p_sig = cv.take<ulonglong2>((size_t)K);
    d.p_l1 = cv.take<int32_t>((size_t)K);
    d.cnt = cv.take<uint32_t>((size_t)n);
    d.keys = cv.take<int32_t>((size_t)kKeyCoords);
    d.bc = cv.take<uint32_t>((size_t)kLists * nblk_part_max);
    d.boff = cv.take<uint32_t>((size_t)kLists * nblk_part_max + 1);
    d.lstart = cv.take<uint32_t>((size_t)kLists + 1);
    d.gblk = cv.take<int4>((size_t)ceil_div(K, kTile) + kLists);
    d.bcount = cv.take<uint32_t>((size_t)d.nblk + 1);
    d.bstart = cv.take<uint32_t>((size_t)d.nblk + 1);
    if (!cv.ok) return MAPE_ERR_CAPACITY;
    MAPE_CUDA_TRY(cudaMemsetAsync(d.hist, 0, sizeof(uint32_t) * d.nb, st));
    MAPE_CUDA_TRY(cudaMemsetAsync(d.bcount, 0, sizeof(uint32_t) * (d.nblk + 1), st));
    MAPE_CUDA_TRY(cudaMemsetAsync(d.cnt, 0, sizeof(uint32_t) * n, st));
  }
  enum { kRows, kCoord, kValid, kPart, kLs, kCmp };
  const int64_t rows = prefix(kRows, [&](int i) { return v[(size_t)i].K; });
  if (rows == 0) return MAPE_OK;
  const int64_t cblocks = prefix(kCoord, [&](int i) { return ceil_div(v[(size_t)i].K_sample, 64); });
  const int64_t cmp = prefix(kCmp, [&](int i) { return v[(size_t)i].K > 0 ? v[(size_t)i].nblk : 0; });
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_views, v.data(), sizeof(MinView) * count, cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_px, px.data(), sizeof(int64_t) * px.size(), cudaMemcpyHostToDevice, st));
  const unsigned gr = (unsigned)ceil_div(rows, kTile);
  const MinView* cv_ = d_views;
  // l1 norms and masks, the l1 order, cleared flags, the key coordinates
  launch(min_rows_batch_kernel, gr, kTile, 0, st, cv_, dpx(kRows), (int)count, 0);
  launch(min_scan_batch_kernel, (unsigned)count, 1024, 0, st, cv_, 0);
  launch(min_rows_batch_kernel, gr, kTile, 0, st, cv_, dpx(kRows), (int)count, 1);
  launch(min_rows_batch_kernel, gr, kTile, 0, st, cv_, dpx(kRows), (int)count, 2);
  launch(min_coord_batch_kernel, (unsigned)cblocks, 256, sizeof(uint32_t) * max_n, st, cv_, dpx(kCoord), (int)count);
  launch(min_keys_batch_kernel, (unsigned)count, 1024, 0, st, cv_, d_nvalid);
  MAPE_LAUNCH_CHECK();
  std::vector<int64_t> nvalid((size_t)count, 0);
  MAPE_CUDA_TRY(cudaMemcpyAsync(nvalid.data(), d_nvalid, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i) {
    v[(size_t)i].nvalid = nvalid[(size_t)i];
    v[(size_t)i].nblk_part = (int)ceil_div(nvalid[(size_t)i], kPartBlock);
  }
  const int64_t valid_rows = prefix(kValid, [&](int i) { return v[(size_t)i].nvalid; });
  if (valid_rows > 0) {
    // pattern lists, each in l1 order
    const int64_t pblocks = prefix(kPart, [&](int i) { return (int64_t)v[(size_t)i].nblk_part; });
    const int64_t ls = prefix(kLs, [&](int i) { return v[(size_t)i].nvalid > 0 ? v[(size_t)i].nlists + 1 : 0; });
    MAPE_CUDA_TRY(cudaMemcpyAsync(d_views, v.data(), sizeof(MinView) * count, cudaMemcpyHostToDevice, st));
    MAPE_CUDA_TRY(cudaMemcpyAsync(d_px + (size_t)kValid * n1, px.data() + (size_t)kValid * n1,
                                  sizeof(int64_t) * 3 * n1, cudaMemcpyHostToDevice, st));
    launch(min_key_rows_batch_kernel, (unsigned)ceil_div(valid_rows, kTile), kTile, 0, st, cv_, dpx(kValid),
           (int)count);
    launch(min_part_batch_kernel, (unsigned)pblocks, kPartBlock, 0, st, cv_, dpx(kPart), (int)count, 0);
    launch(min_scan_batch_kernel, (unsigned)count, 1024, 0, st, cv_, 1);
    launch(min_part_batch_kernel, (unsigned)pblocks, 32, 0, st, cv_, dpx(kPart), (int)count, 1);
    launch(min_list_start_batch_kernel, (unsigned)ceil_div(ls, 256), 256, 0, st, cv_, dpx(kLs), (int)count);
    MAPE_LAUNCH_CHECK();
    std::vector<std::vector<uint32_t>> lst((size_t)count);
    for (int i = 0; i < count; ++i) {
      if (v[(size_t)i].nvalid == 0) continue;
      lst[(size_t)i].resize((size_t)v[(size_t)i].nlists + 1);
      MAPE_CUDA_TRY(cudaMemcpyAsync(lst[(size_t)i].data(), v[(size_t)i].lstart, sizeof(uint32_t) * lst[(size_t)i].size(),
                                    cudaMemcpyDeviceToHost, st));
    }
    MAPE_CUDA_TRY(cudaStreamSynchronize(st));
    // g-blocks of every instance: runs of at most kTile rows of one list
    std::vector<int4> gb;
    uint32_t max_list = 0;
    int max_kb = 0;
    for (int i = 0; i < count; ++i) {
      if (v[(size_t)i].nvalid == 0) continue;
      max_kb = std::max(max_kb, v[(size_t)i].kb);
      const std::vector<uint32_t>& l = lst[(size_t)i];
      for (int L = 0; L < v[(size_t)i].nlists; ++L) {
        const uint32_t a = l[(size_t)L], b = l[(size_t)L + 1];
        max_list = std::max(max_list, b - a);
        for (uint32_t o = a; o < b; o += kTile)
          gb.push_back(make_int4((int)o, (int)std::min<uint32_t>(kTile, b - o), L, i));
      }
    }
    if (!gb.empty()) {
      if ((int64_t)gb.size() > gb_cap) return MAPE_ERR_CAPACITY;
      MAPE_CUDA_TRY(cudaMemcpyAsync(d_gblk, gb.data(), sizeof(int4) * gb.size(), cudaMemcpyHostToDevice, st));
      const dim3 grid((unsigned)gb.size(), 2u << max_kb, (unsigned)ceil_div(max_list, kChunk));
      launch(min_dominance_batch_kernel, grid, kTile, 0, st, cv_, (const int4*)d_gblk);
    }
  }
  // keep flags, then the kept rows in input order
  launch(min_rows_batch_kernel, gr, kTile, 0, st, cv_, dpx(kRows), (int)count, 3);
  launch(min_compact_batch_kernel, (unsigned)cmp, kCompact, 0, st, cv_, dpx(kCmp), (int)count, 0);
  launch(min_scan_batch_kernel, (unsigned)count, 1024, 0, st, cv_, 2);
  launch(min_compact_batch_kernel, (unsigned)cmp, kCompact, 0, st, cv_, dpx(kCmp), (int)count, 1);
  MAPE_LAUNCH_CHECK();
  std::vector<uint32_t> tot((size_t)count, 0);
  for (int i = 0; i < count; ++i)
    if (v[(size_t)i].K > 0)
      MAPE_CUDA_TRY(cudaMemcpyAsync(&tot[(size_t)i], v[(size_t)i].bstart + v[(size_t)i].nblk, 4,
                                    cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i) items[i].K_out = (int64_t)tot[(size_t)i];
  return MAPE_OK;
}
