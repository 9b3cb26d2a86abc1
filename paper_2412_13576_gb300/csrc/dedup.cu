// a10: the set union of Algorithm 2 (§3.2).
//
// 1. every candidate row gets a 64-bit hash (16-byte vector loads);
// 2. rows are inserted into an open-addressing table of row indices with
//    linear probing.  Rows are fully written before the insert kernel runs,
//    so an insert only ever compares against complete rows: a lock-free CAS
//    on an empty slot makes a row the representative of its value, and a
//    match (hash, then bytes) marks it a duplicate.  The table holds at least
//    twice as many slots as rows, so every probe sequence meets an empty slot
//    and the loop is bounded by the table size;
// 3. representatives are compacted (order not fixed by the hardware) and
//    then sorted lexicographically, which fixes the output order
//    independently of the atomics.  The key of a row is its first 8 bytes as
//    one unsigned number (first byte most significant, sign bits flipped).
//    A bitonic network sorts (key, row index) pairs, one 64-bit compare on
//    data in shared memory each; then every run of equal keys (rows that
//    share their first 8 bytes) is sorted by the rows' remaining bytes, one
//    block per run.  Should a run be longer than a block sorts, the whole
//    array is sorted again with the comparison that reads the rows.
#include "common.cuh"

#include <algorithm>
#include <mutex>
#include <vector>

namespace {

constexpr uint32_t kEmpty = 0xffffffffu;

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 31;
  x *= 0x7fb5d329728ea185ull;
  x ^= x >> 27;
  x *= 0x81dadef4bc2dd44dull;
  x ^= x >> 33;
  return x;
}

__device__ __forceinline__ void hash_row(const int8_t* __restrict__ rows, int64_t r, int ldc,
                                         uint64_t* __restrict__ h) {
  const uint4* p = reinterpret_cast<const uint4*>(rows + r * ldc);
  uint64_t acc = 0x243f6a8885a308d3ull ^ (uint64_t)ldc;
  for (int c = 0; c < ldc / 16; ++c) {
    uint4 v = p[c];
    acc = mix64(acc ^ (((uint64_t)v.y << 32) | v.x));
    acc = mix64(acc + (((uint64_t)v.w << 32) | v.z));
  }
  h[r] = acc;
}

__global__ void hash_rows_kernel(const int8_t* __restrict__ rows, int64_t count, int ldc,
                                 uint64_t* __restrict__ h) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= count) return;
  hash_row(rows, r, ldc, h);
}

__device__ __forceinline__ bool rows_equal(const int8_t* a, const int8_t* b, int ldc) {
  const uint4* pa = reinterpret_cast<const uint4*>(a);
  const uint4* pb = reinterpret_cast<const uint4*>(b);
  for (int c = 0; c < ldc / 16; ++c) {
    uint4 x = pa[c], y = pb[c];
    if (x.x != y.x || x.y != y.y || x.z != y.z || x.w != y.w) return false;
  }
  return true;
}

__device__ __forceinline__ void insert_row(const int8_t* __restrict__ rows, const uint64_t* __restrict__ h,
                                           int64_t r, int ldc, uint32_t* __restrict__ table, uint64_t mask,
                                           uint8_t* __restrict__ is_rep) {
  uint64_t hr = h[r];
  uint64_t slot = hr & mask;
  uint8_t rep = 0;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    uint32_t cur = table[slot];
    if (cur == kEmpty) {
      uint32_t old = atomicCAS(&table[slot], kEmpty, (uint32_t)r);
      if (old == kEmpty) { rep = 1; break; }
      cur = old;
    }
    if (h[cur] == hr && rows_equal(rows + (int64_t)cur * ldc, rows + r * ldc, ldc)) break;
    slot = (slot + 1) & mask;
  }
  is_rep[r] = rep;
}

__global__ void insert_kernel(const int8_t* __restrict__ rows, const uint64_t* __restrict__ h, int64_t count,
                              int ldc, uint32_t* __restrict__ table, uint64_t mask,
                              uint8_t* __restrict__ is_rep) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= count) return;
  insert_row(rows, h, r, ldc, table, mask, is_rep);
}

__device__ __forceinline__ void compact_row(const uint8_t* __restrict__ is_rep, int64_t r,
                                            uint32_t* __restrict__ idx, unsigned long long* __restrict__ K) {
  if (!is_rep[r]) return;
  unsigned long long at = atomicAdd(K, 1ull);
  idx[at] = (uint32_t)r;
}

__global__ void compact_reps_kernel(const uint8_t* __restrict__ is_rep, int64_t count,
                                    uint32_t* __restrict__ idx, unsigned long long* __restrict__ K) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= count) return;
  compact_row(is_rep, r, idx, K);
}

__global__ void pad_idx_kernel(uint32_t* idx, int64_t from, int64_t to) {
  int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < to) idx[i] = kEmpty;
}

// The first 8 bytes of a row, first byte most significant, sign bits flipped:
// unsigned order of keys = lexicographic order of the signed bytes
__device__ __forceinline__ uint64_t row_key(const int8_t* row) {
  const uint2 w = *reinterpret_cast<const uint2*>(row);
  const uint32_t hi = __byte_perm(w.x, 0, 0x0123) ^ 0x80808080u;
  const uint32_t lo = __byte_perm(w.y, 0, 0x0123) ^ 0x80808080u;
  return ((uint64_t)hi << 32) | lo;
}

// Lexicographic order on signed bytes of (key, row) pairs; kEmpty sorts last.
// Rows with equal keys are compared from byte 8 on, 16 bytes at a time.
__device__ __forceinline__ int cmp_keyed(const int8_t* rows, int ldc, uint64_t ka, uint32_t a, uint64_t kb,
                                         uint32_t b) {
  if (a == b) return 0;
  if (a == kEmpty) return 1;
  if (b == kEmpty) return -1;
  if (ka != kb) return ka < kb ? -1 : 1;
  const uint32_t* pa = reinterpret_cast<const uint32_t*>(rows + (int64_t)a * ldc);
  const uint32_t* pb = reinterpret_cast<const uint32_t*>(rows + (int64_t)b * ldc);
  for (int c = 2; c < ldc / 4; ++c) {
    const uint32_t x = __byte_perm(pa[c], 0, 0x0123) ^ 0x80808080u;
    const uint32_t y = __byte_perm(pb[c], 0, 0x0123) ^ 0x80808080u;
    if (x != y) return x < y ? -1 : 1;
  }
  return 0;
}

__global__ void key_rows_kernel(const int8_t* __restrict__ rows, int ldc, const uint32_t* __restrict__ idx,
                                int64_t npad, uint64_t* __restrict__ key) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npad) return;
  const uint32_t a = idx[i];
  key[i] = a == kEmpty ? ~0ull : row_key(rows + (int64_t)a * ldc);
}

// (key, index) order, or the rows' lexicographic order (kFull)
template <bool kFull>
__device__ __forceinline__ int cmp_pair(const int8_t* rows, int ldc, uint64_t ka, uint32_t a, uint64_t kb, uint32_t b) {
  if (kFull) return cmp_keyed(rows, ldc, ka, a, kb, b);
  if (ka != kb) return ka < kb ? -1 : 1;
  return a == b ? 0 : (a < b ? -1 : 1);
}

template <bool kFull>
__device__ __forceinline__ void bitonic_step_one(const int8_t* __restrict__ rows, int ldc, uint64_t* __restrict__ key,
                                                 uint32_t* __restrict__ idx, int64_t i, int64_t j, int64_t k) {
  int64_t l = i ^ j;
  if (l <= i) return;
  const uint32_t a = idx[i], b = idx[l];
  const uint64_t ka = key[i], kb = key[l];
  bool ascending = (i & k) == 0;
  int c = cmp_pair<kFull>(rows, ldc, ka, a, kb, b);
  if ((ascending && c > 0) || (!ascending && c < 0)) {
    idx[i] = b;
    idx[l] = a;
    key[i] = kb;
    key[l] = ka;
  }
}

template <bool kFull>
__global__ void bitonic_step_kernel(const int8_t* __restrict__ rows, int ldc, uint64_t* __restrict__ key,
                                    uint32_t* __restrict__ idx, int64_t npad, int64_t j, int64_t k) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npad) return;
  bitonic_step_one<kFull>(rows, ldc, key, idx, i, j, k);
}

constexpr int kSeg = 2048;

// Bitonic stages k = kfirst .. klast (doubling), distances j < seg, on the
// segment of seg pairs owned by this block (seg <= kSeg, a power of two).
template <bool kFull>
__device__ __forceinline__ void bitonic_local_seg(const int8_t* __restrict__ rows, int ldc,
                                                  uint64_t* __restrict__ key, uint32_t* __restrict__ idx,
                                                  int64_t seg, int64_t kfirst, int64_t klast, int64_t sgi) {
  __shared__ uint64_t sk[kSeg];
  __shared__ uint32_t s[kSeg];
  const int64_t base = sgi * seg;
  for (int t = threadIdx.x; t < seg; t += blockDim.x) {
    s[t] = idx[base + t];
    sk[t] = key[base + t];
  }
  __syncthreads();
  for (int64_t k = kfirst; k <= klast; k <<= 1) {
    for (int64_t j = ((k >> 1) < (seg >> 1) ? (k >> 1) : (seg >> 1)); j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < seg / 2; t += blockDim.x) {
        const int64_t i = (t / j) * 2 * j + (t % j);  // lower element of the pair
        const int64_t l = i + j;
        const bool ascending = ((base + i) & k) == 0;
        const uint32_t a = s[i], b = s[l];
        const uint64_t ka = sk[i], kb = sk[l];
        const int c = cmp_pair<kFull>(rows, ldc, ka, a, kb, b);
        if ((ascending && c > 0) || (!ascending && c < 0)) {
          s[i] = b;
          s[l] = a;
          sk[i] = kb;
          sk[l] = ka;
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < seg; t += blockDim.x) {
    idx[base + t] = s[t];
    key[base + t] = sk[t];
  }
}

template <bool kFull>
__global__ void bitonic_local_kernel(const int8_t* __restrict__ rows, int ldc, uint64_t* __restrict__ key,
                                     uint32_t* __restrict__ idx, int64_t seg, int64_t kfirst, int64_t klast) {
  bitonic_local_seg<kFull>(rows, ldc, key, idx, seg, kfirst, klast, blockIdx.x);
}

constexpr int kRunWarpRows = 32;      // runs up to this length are sorted by one warp ...
constexpr int kRunWarpBytes = 8192;   // ... when their rows fit in its share of shared memory
constexpr int kRunWarps = 4;          // warps (runs) per block of the warp kernel (32 KB)

// runs of equal keys among the first K sorted pairs: (start, length) of
// every run of two or more (short ones, that one warp sorts, from the front
// of `runs`, the others from the back), their counts and the longest length
__device__ __forceinline__ void key_run_at(const uint64_t* __restrict__ key, int64_t K, int ldc,
                                           int2* __restrict__ runs, int64_t runs_cap,
                                           unsigned int* __restrict__ nshort, unsigned int* __restrict__ nlong,
                                           unsigned int* __restrict__ maxlen, int64_t i) {
  if (i > 0 && key[i] == key[i - 1]) return;      // not the start of a run
  if (i + 1 >= K || key[i + 1] != key[i]) return;  // a run of one
  int64_t j = i + 2;
  while (j < K && key[j] == key[i]) ++j;
  const unsigned int len = (unsigned int)(j - i);
  atomicMax(maxlen, len);
  if (len <= (unsigned)kRunWarpRows && (int64_t)len * ldc <= kRunWarpBytes) {
    const unsigned int at = atomicAdd(nshort, 1u);
    runs[at] = make_int2((int)i, (int)len);
  } else {
    const unsigned int at = atomicAdd(nlong, 1u);
    runs[runs_cap - 1 - at] = make_int2((int)i, (int)len);
  }
}

__global__ void key_runs_kernel(const uint64_t* __restrict__ key, int64_t K, int ldc, int2* __restrict__ runs,
                                int64_t runs_cap, unsigned int* __restrict__ nshort, unsigned int* __restrict__ nlong,
                                unsigned int* __restrict__ maxlen) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= K) return;
  key_run_at(key, K, ldc, runs, runs_cap, nshort, nlong, maxlen, i);
}

constexpr int kRunStageBytes = 32 * 1024;  // rows of a run staged in shared memory up to this size
constexpr int kRunStageRows = 256;

// lexicographic order of two staged rows (positions a, b; kEmpty last), bytes 8 on
__device__ __forceinline__ int cmp_staged(const int8_t* srow, int ldc, uint32_t a, uint32_t b) {
  if (a == b) return 0;
  if (a == kEmpty) return 1;
  if (b == kEmpty) return -1;
  const uint32_t* pa = reinterpret_cast<const uint32_t*>(srow + (size_t)a * ldc);
  const uint32_t* pb = reinterpret_cast<const uint32_t*>(srow + (size_t)b * ldc);
  for (int c = 2; c < ldc / 4; ++c) {
    const uint32_t x = __byte_perm(pa[c], 0, 0x0123) ^ 0x80808080u;
    const uint32_t y = __byte_perm(pb[c], 0, 0x0123) ^ 0x80808080u;
    if (x != y) return x < y ? -1 : 1;
  }
  return 0;
}

// one warp per short run: the run's rows are copied into the warp's share of
// shared memory, and a bitonic network over the lanes (one position each,
// partners by shuffle) orders them from byte 8 on
__device__ __forceinline__ void run_sort_warp(const int8_t* __restrict__ rows, int ldc, int2 rr,
                                              uint32_t* __restrict__ idx) {
  extern __shared__ __align__(16) int8_t sm_runs[];  // kRunWarps x kRunWarpBytes
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int len = rr.y;
  int8_t* srow = sm_runs + w * kRunWarpBytes;
  const uint32_t orig = lane < len ? idx[rr.x + lane] : kEmpty;
  const int q = ldc / 16, tot = len * q;
  for (int base = 0; base < tot; base += 32) {  // the same trip count in every lane
    const int e = base + lane;
    const uint32_t src = __shfl_sync(0xffffffffu, orig, (e < tot ? e : tot - 1) / q);
    if (e < tot) reinterpret_cast<uint4*>(srow)[e] = reinterpret_cast<const uint4*>(rows + (int64_t)src * ldc)[e % q];
  }
  __syncwarp();
  int np = 2;
  while (np < len) np <<= 1;
  uint32_t pos = lane < len ? (uint32_t)lane : kEmpty;
  for (int k = 2; k <= np; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint32_t other = __shfl_xor_sync(0xffffffffu, pos, j);
      const bool lower = (lane & j) == 0, ascending = (lane & k) == 0;
      const int c = cmp_staged(srow, ldc, lower ? pos : other, lower ? other : pos);  // lower vs upper element
      const bool swap = ascending ? c > 0 : c < 0;
      if (swap) pos = other;
    }
  }
  const uint32_t out = __shfl_sync(0xffffffffu, orig, (int)(pos == kEmpty ? 0 : pos));
  if (lane < len) idx[rr.x + lane] = out;
}

__global__ void run_sort_warp_kernel(const int8_t* __restrict__ rows, int ldc, const int2* __restrict__ runs,
                                     unsigned int nruns, uint32_t* __restrict__ idx) {
  const unsigned int run = blockIdx.x * kRunWarps + (threadIdx.x >> 5);
  if (run >= nruns) return;  // warp-uniform
  run_sort_warp(rows, ldc, runs[run], idx);
}

constexpr int kRunMax = 2048;  // longest run one block sorts

// one block per (long) run: bitonic on the run (padded with the sentinel to a power
// of two) comparing the rows from byte 8 on; a run whose rows fit is first
// copied into shared memory, and the network then sorts positions in it
__device__ __forceinline__ void run_sort_block(const int8_t* __restrict__ rows, int ldc, int2 rr,
                                               uint32_t* __restrict__ idx) {
  __shared__ uint32_t s[kRunMax];
  __shared__ uint32_t s_orig[kRunStageRows];
  extern __shared__ __align__(16) int8_t srow[];  // kRunStageBytes
  int np = 2;
  while (np < rr.y) np <<= 1;
  const bool staged = rr.y <= kRunStageRows && (int64_t)rr.y * ldc <= kRunStageBytes;
  if (staged) {
    for (int t = threadIdx.x; t < rr.y; t += blockDim.x) s_orig[t] = idx[rr.x + t];
    __syncthreads();
    const int w = ldc / 16;
    for (int e = threadIdx.x; e < rr.y * w; e += blockDim.x)
      reinterpret_cast<uint4*>(srow)[e] = reinterpret_cast<const uint4*>(rows + (int64_t)s_orig[e / w] * ldc)[e % w];
  }
  for (int t = threadIdx.x; t < np; t += blockDim.x)
    s[t] = t < rr.y ? (staged ? (uint32_t)t : idx[rr.x + t]) : kEmpty;
  __syncthreads();
  for (int k = 2; k <= np; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < np / 2; t += blockDim.x) {
        const int i = (t / j) * 2 * j + (t % j), l = i + j;
        const bool ascending = (i & k) == 0;
        const uint32_t a = s[i], b = s[l];
        const int c = staged ? cmp_staged(srow, ldc, a, b) : cmp_keyed(rows, ldc, 0, a, 0, b);  // equal keys: bytes 8 on
        if ((ascending && c > 0) || (!ascending && c < 0)) {
          s[i] = b;
          s[l] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < rr.y; t += blockDim.x) idx[rr.x + t] = staged ? s_orig[s[t]] : s[t];
}

__global__ void run_sort_kernel(const int8_t* __restrict__ rows, int ldc, const int2* __restrict__ runs,
                                uint32_t* __restrict__ idx) {
  run_sort_block(rows, ldc, runs[blockIdx.x], idx);
}

__global__ void gather_rows_kernel(const int8_t* __restrict__ rows, int ldc, const uint32_t* __restrict__ idx,
                                   int64_t K, int8_t* __restrict__ out) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int chunks = ldc / 16;
  int64_t r = t / chunks;
  int c = (int)(t % chunks);
  if (r >= K) return;
  reinterpret_cast<uint4*>(out + r * ldc)[c] = reinterpret_cast<const uint4*>(rows + (int64_t)idx[r] * ldc)[c];
}

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace

namespace mape_detail {

// Sorts rows[idx[0..K)] lexicographically in place of idx (npad >= K, power of 2,
// idx[K..npad) set to the sentinel by this call; key: npad words of scratch).
// The network is the plain bitonic one; all stages with distance j < seg run
// inside one launch on shared-memory segments of seg = min(npad, 2048) pairs
// (the compare direction still comes from the global index).
template <bool kFull>
void bitonic_sort(const int8_t* rows, int ldc, uint32_t* idx, uint64_t* key, int64_t npad, cudaStream_t st) {
  const int64_t seg = npad < kSeg ? npad : kSeg;
  const unsigned nseg = (unsigned)(npad / seg);
  mape_detail::launch(bitonic_local_kernel<kFull>, nseg, kSeg / 2, 0, st, rows, ldc, key, idx, seg, (int64_t)2, seg);
  for (int64_t k = 2 * seg; k <= npad; k <<= 1) {
    for (int64_t j = k >> 1; j >= seg; j >>= 1)
      mape_detail::launch(bitonic_step_kernel<kFull>, (unsigned)ceil_div(npad, 256), 256, 0, st, rows, ldc, key, idx,
                          npad, j, k);
    mape_detail::launch(bitonic_local_kernel<kFull>, nseg, kSeg / 2, 0, st, rows, ldc, key, idx, seg, k, k);
  }
}

int sort_row_indices(const int8_t* rows, int ldc, uint32_t* idx, uint64_t* key, int2* runs, unsigned int* counters,
                     int64_t K, int64_t npad, cudaStream_t st) {
  if (npad > K) mape_detail::launch(pad_idx_kernel, (unsigned)ceil_div(npad - K, 256), 256, 0, st, idx, K, npad);
  if (npad < 2) return MAPE_OK;
  mape_detail::launch(key_rows_kernel, (unsigned)ceil_div(npad, 256), 256, 0, st, rows, ldc, idx, npad, key);
  bitonic_sort<false>(rows, ldc, idx, key, npad, st);
  const int64_t runs_cap = K / 2 + 1;
  MAPE_CUDA_TRY(cudaMemsetAsync(counters, 0, 3 * sizeof(unsigned int), st));
  mape_detail::launch(key_runs_kernel, (unsigned)ceil_div(K, 256), 256, 0, st, key, K, ldc, runs, runs_cap, counters,
                      counters + 1, counters + 2);
  MAPE_LAUNCH_CHECK();
  unsigned int hc[3] = {0, 0, 0};  // short runs, long runs, longest
  MAPE_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  if (hc[2] > (unsigned)kRunMax) {
    bitonic_sort<true>(rows, ldc, idx, key, npad, st);  // the rows decide every comparison
  } else {
    if (hc[0] > 0)
      mape_detail::launch(run_sort_warp_kernel, (unsigned)ceil_div(hc[0], kRunWarps), 32 * kRunWarps,
                          (size_t)kRunWarps * kRunWarpBytes, st, rows, ldc, runs, hc[0], idx);
    if (hc[1] > 0)
      mape_detail::launch(run_sort_kernel, hc[1], 128, kRunStageBytes, st, rows, ldc, runs + (runs_cap - hc[1]), idx);
  }
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}

uint64_t dedup_table_slots(int64_t count) { return next_pow2((uint64_t)(count > 0 ? count : 1) * 2); }

}  // namespace mape_detail

extern "C" size_t mape_dedup_workspace_bytes(int64_t count, int32_t ldc) {
  (void)ldc;
  if (count < 0) return 0;
  mape_detail::Sizer s;
  s.take<uint64_t>((size_t)count);                               // hashes
  s.take<uint32_t>((size_t)mape_detail::dedup_table_slots(count)); // table
  s.take<uint8_t>((size_t)count);                                 // representative flags
  s.take<uint32_t>((size_t)next_pow2((uint64_t)(count > 0 ? count : 1)));  // sorted indices
  s.take<uint64_t>((size_t)next_pow2((uint64_t)(count > 0 ? count : 1)));  // their sort keys
  s.take<int2>((size_t)(count > 0 ? count : 1) / 2 + 1);          // runs of equal keys
  s.take<unsigned int>(3);                                        // short and long run counts, longest run
  s.take<unsigned long long>(1);                                  // counter
  return s.bytes();
}

extern "C" int mape_dedup(const int8_t* cand, int64_t count, int32_t n, int32_t ldc, int8_t* uniq,
                          int64_t uniq_cap, int64_t* K_out, void* workspace, size_t workspace_bytes,
                          void* stream) {
  using namespace mape_detail;
  if (!K_out || count < 0 || n <= 0 || ldc < n || ldc % 16 != 0 || uniq_cap < 0) return MAPE_ERR_INVALID_ARG;
  if (count > 0 && !cand) return MAPE_ERR_INVALID_ARG;
  if (count >= (int64_t)kEmpty) return MAPE_ERR_SHAPE;
  *K_out = 0;
  if (count == 0) return MAPE_OK;
  Carver cv(workspace, workspace_bytes);
  uint64_t* h = cv.take<uint64_t>((size_t)count);
  uint64_t slots = dedup_table_slots(count);
  uint32_t* table = cv.take<uint32_t>((size_t)slots);
  uint8_t* is_rep = cv.take<uint8_t>((size_t)count);
  uint64_t npad_cap = next_pow2((uint64_t)count);
  uint32_t* idx = cv.take<uint32_t>((size_t)npad_cap);
  uint64_t* keys = cv.take<uint64_t>((size_t)npad_cap);
  int2* runs = cv.take<int2>((size_t)count / 2 + 1);
  unsigned int* run_counters = cv.take<unsigned int>(3);
  unsigned long long* dK = cv.take<unsigned long long>(1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  unsigned g = (unsigned)ceil_div(count, 256);
  MAPE_CUDA_TRY(cudaMemsetAsync(table, 0xff, slots * sizeof(uint32_t), st));
  MAPE_CUDA_TRY(cudaMemsetAsync(dK, 0, sizeof(unsigned long long), st));
  mape_detail::launch(hash_rows_kernel, g, 256, 0, st, cand, count, ldc, h);
  mape_detail::launch(insert_kernel, g, 256, 0, st, cand, h, count, ldc, table, slots - 1, is_rep);
  mape_detail::launch(compact_reps_kernel, g, 256, 0, st, is_rep, count, idx, dK);
  MAPE_LAUNCH_CHECK();
  unsigned long long K = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&K, dK, sizeof(K), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  *K_out = (int64_t)K;
  if ((int64_t)K > uniq_cap) return MAPE_ERR_CAPACITY;
  if (!uniq) return MAPE_ERR_INVALID_ARG;
  int rc = sort_row_indices(cand, ldc, idx, keys, runs, run_counters, (int64_t)K, (int64_t)next_pow2(K), st);
  if (rc != MAPE_OK) return rc;
  int64_t chunks = (int64_t)K * (ldc / 16);
  mape_detail::launch(gather_rows_kernel, (unsigned)ceil_div(chunks, 256), 256, 0, st, cand, ldc, idx, (int64_t)K, uniq);
  MAPE_LAUNCH_CHECK();
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  return MAPE_OK;
}

// ---- the same stage without any device allocation ----------------------------
//
// For callers that cannot allocate device memory at the point where they
// dedup: hosts that reserve all device memory up front and forbid allocations
// later (fixed-memory long-running loops), or plugins whose host owns the
// device allocator.  The call stays synchronous (it reads the distinct count
// back and synchronises the stream), so it cannot run inside a stream capture.
// The scratch lives in a file-scope device array that every GPU loading this
// library holds until the process exits.  Host code cannot pass that array's
// name to a kernel (in host code it is only a host-side stand-in), so its
// device address is looked up once per device, with that device current, by
// cudaGetSymbolAddress, and cached; a CUDA error forgets the cached address
// (a cudaDeviceReset invalidates it), so the next call looks it up again.

namespace {

constexpr int64_t kStaticDedupRows = (int64_t)1 << 18;       // candidate rows per call
constexpr size_t kStaticDedupBytes = (size_t)10 << 20;        // >= mape_dedup_workspace_bytes(2^18, any ldc)
static __device__ __align__(256) unsigned char g_dedup_scratch[kStaticDedupBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_dedup_scratch on the current device (looked up once).
int static_dedup_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    mape_detail::record_cuda_error(e, "cudaGetDevice", __FILE__, __LINE__);
    return MAPE_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    mape_detail::record_message("mape_dedup_static: device index beyond the 64 devices it supports");
    return MAPE_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dedup_scratch);
    if (e != cudaSuccess || p == nullptr) {
      mape_detail::record_cuda_error(e, "cudaGetSymbolAddress(g_dedup_scratch)", __FILE__, __LINE__);
      return MAPE_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MAPE_OK;
}

// Drops the cached address of the current device (after a CUDA error, which
// may come from a reset context): the next call looks it up again.
void forget_static_dedup_scratch() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  g_scratch_ptr[dev] = nullptr;
}

}  // namespace

extern "C" int64_t mape_dedup_static_max_rows(void) { return kStaticDedupRows; }

extern "C" int mape_dedup_static(const int8_t* cand, int64_t count, int32_t n, int32_t ldc, int8_t* uniq,
                                 int64_t uniq_cap, int64_t* K_out, void* stream) {
  if (!K_out || count < 0 || n <= 0 || ldc < n || ldc % 16 != 0 || uniq_cap < 0) return MAPE_ERR_INVALID_ARG;
  *K_out = 0;
  if (count > kStaticDedupRows) return MAPE_ERR_CAPACITY;  // more rows than the static scratch holds
  if (mape_dedup_workspace_bytes(count, ldc) > kStaticDedupBytes) return MAPE_ERR_CAPACITY;
  if (count == 0) return MAPE_OK;
  void* scratch = nullptr;
  int rc = static_dedup_scratch(&scratch);
  if (rc != MAPE_OK) return rc;
  // the table and the counter are cleared by the stage itself on every call
  rc = mape_dedup(cand, count, n, ldc, uniq, uniq_cap, K_out, scratch, kStaticDedupBytes, stream);
  if (rc == MAPE_ERR_CUDA) forget_static_dedup_scratch();
  return rc;
}

// ---- many candidate sets at once -------------------------------------------
//
// mape_dedup for `count` independent sets in one sequence of launches: every
// kernel of the stage runs once over the rows (or sort positions, runs,
// output pieces) of all sets, each thread, warp or block finding its set by
// binary search over the launch's prefix table.  Each set keeps its own hash
// table, sort arrays and output, carved from its own workspace exactly as
// mape_dedup carves it, so its output is the same.  The bitonic stages run
// for the largest set; a set whose sort is already complete at a stage sits
// it out.

namespace {

struct DedupView {
  const int8_t* rows;
  int64_t count;
  int ldc;
  uint64_t* h;
  uint32_t* table;
  uint64_t mask;
  uint8_t* is_rep;
  uint32_t* idx;
  uint64_t* key;
  int2* runs;
  int64_t runs_cap;
  int8_t* uniq;
  int64_t K, npad, seg;  // distinct rows, sort size, segment of the local stages (0: no sort)
  int64_t nshort, nlong;  // runs of equal keys for the warp and block sorts
};

__device__ __forceinline__ int find_set(const int64_t* __restrict__ prefix, int count, int64_t x) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// prefix: rows (count + 1 entries)
__global__ void hash_insert_batch_kernel(const DedupView* __restrict__ v, const int64_t* __restrict__ prefix, int count,
                                         int phase, unsigned long long* __restrict__ K) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= prefix[count]) return;
  const int i = find_set(prefix, count, t);
  const DedupView& d = v[i];
  const int64_t r = t - prefix[i];
  if (phase == 0) hash_row(d.rows, r, d.ldc, d.h);
  else if (phase == 1) insert_row(d.rows, d.h, r, d.ldc, d.table, d.mask, d.is_rep);
  else compact_row(d.is_rep, r, d.idx, K + i);
}

// prefix: sort positions (npad); the padding sentinel and the keys
__global__ void key_batch_kernel(const DedupView* __restrict__ v, const int64_t* __restrict__ prefix, int count) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= prefix[count]) return;
  const int i = find_set(prefix, count, t);
  const DedupView& d = v[i];
  const int64_t p = t - prefix[i];
  if (p >= d.K) d.idx[p] = kEmpty;
  const uint32_t a = d.idx[p];
  d.key[p] = a == kEmpty ? ~0ull : row_key(d.rows + (int64_t)a * d.ldc);
}

// prefix: segments (npad / seg); k = 0: the first stages (2 .. seg), else
// stage k alone (sets with fewer than k positions sit it out)
__global__ void bitonic_local_batch_kernel(const DedupView* __restrict__ v, const int64_t* __restrict__ prefix,
                                           int count, int64_t k) {
  const int i = find_set(prefix, count, blockIdx.x);
  const DedupView& d = v[i];
  if (k > d.npad) return;
  const int64_t kf = k == 0 ? 2 : k, kl = k == 0 ? d.seg : k;
  bitonic_local_seg<false>(d.rows, d.ldc, d.key, d.idx, d.seg, kf, kl, blockIdx.x - prefix[i]);
}

// prefix: sort positions; distance j of stage k
__global__ void bitonic_step_batch_kernel(const DedupView* __restrict__ v, const int64_t* __restrict__ prefix,
                                          int count, int64_t j, int64_t k) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= prefix[count]) return;
  const int i = find_set(prefix, count, t);
  const DedupView& d = v[i];
  if (k > d.npad) return;
  bitonic_step_one<false>(d.rows, d.ldc, d.key, d.idx, t - prefix[i], j, k);
}

// prefix: distinct rows; counters: 3 per set
__global__ void key_runs_batch_kernel(const DedupView* __restrict__ v, const int64_t* __restrict__ prefix, int count,
                                      unsigned int* __restrict__ counters) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= prefix[count]) return;
  const int i = find_set(prefix, count, t);
  const DedupView& d = v[i];
  unsigned int* c = counters + 3 * i;
  key_run_at(d.key, d.K, d.ldc, d.runs, d.runs_cap, c, c + 1, c + 2, t - prefix[i]);
}

// prefix: short runs; one warp per run
__global__ void run_sort_warp_batch_kernel(const DedupView* __restrict__ v, const int64_t* __restrict__ prefix,
                                           int count) {
  const int64_t g = (int64_t)blockIdx.x * kRunWarps + (threadIdx.x >> 5);
  if (g >= prefix[count]) return;  // warp-uniform
  const int i = find_set(prefix, count, g);
  const DedupView& d = v[i];
  run_sort_warp(d.rows, d.ldc, d.runs[g - prefix[i]], d.idx);
}

// prefix: long runs; one block per run
__global__ void run_sort_batch_kernel(const DedupView* __restrict__ v, const int64_t* __restrict__ prefix, int count) {
  const int i = find_set(prefix, count, blockIdx.x);
  const DedupView& d = v[i];
  const int64_t b = blockIdx.x - prefix[i];
  run_sort_block(d.rows, d.ldc, d.runs[d.runs_cap - d.nlong + b], d.idx);
}

// prefix: 16-byte pieces of the distinct rows
__global__ void gather_batch_kernel(const DedupView* __restrict__ v, const int64_t* __restrict__ prefix, int count) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= prefix[count]) return;
  const int i = find_set(prefix, count, t);
  const DedupView& d = v[i];
  const int64_t e = t - prefix[i];
  const int chunks = d.ldc / 16;
  const int64_t r = e / chunks;
  const int c = (int)(e % chunks);
  reinterpret_cast<uint4*>(d.uniq + r * d.ldc)[c] = reinterpret_cast<const uint4*>(d.rows + (int64_t)d.idx[r] * d.ldc)[c];
}

}  // namespace

// prefix tables of the batch launches, `count` + 1 entries each
enum { kPxRows, kPxPos, kPxSegs, kPxKeyed, kPxPieces, kPxShort, kPxLong, kPxTables };

extern "C" size_t mape_dedup_batch_workspace_bytes(int32_t count) {
  if (count <= 0) return 0;
  mape_detail::Sizer s;
  s.take<DedupView>((size_t)count);
  s.take<int64_t>((size_t)kPxTables * (count + 1));  // prefix tables
  s.take<unsigned long long>((size_t)count);         // distinct-row counters
  s.take<unsigned int>((size_t)3 * count);           // run counters
  return s.bytes();
}

extern "C" int mape_dedup_batch(mape_dedup_item* items, int32_t count, void* workspace, size_t workspace_bytes,
                                void* stream) {
  using namespace mape_detail;
  if (!items || count <= 0) return MAPE_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const mape_dedup_item& it = items[i];
    if (it.count < 0 || it.n <= 0 || it.ldc < it.n || it.ldc % 16 != 0 || it.uniq_cap < 0) return MAPE_ERR_INVALID_ARG;
    if (it.count > 0 && !it.cand) return MAPE_ERR_INVALID_ARG;
    if (it.count >= (int64_t)kEmpty) return MAPE_ERR_SHAPE;
  }
  Carver bc(workspace, workspace_bytes);
  DedupView* d_views = bc.take<DedupView>((size_t)count);
  int64_t* d_px = bc.take<int64_t>((size_t)kPxTables * (count + 1));
  unsigned long long* d_K = bc.take<unsigned long long>((size_t)count);
  unsigned int* d_runc = bc.take<unsigned int>((size_t)3 * count);
  if (!bc.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  const int n1 = count + 1;
  std::vector<int64_t> px((size_t)kPxTables * n1, 0);
  // prefix table `t` over units(i), returning its total
  auto prefix = [&](int t, auto units) -> int64_t {
    int64_t* p = px.data() + (size_t)t * n1;
    p[0] = 0;
    for (int i = 0; i < count; ++i) p[i + 1] = p[i] + units(i);
    return p[count];
  };
  auto dpx = [&](int t) -> const int64_t* { return d_px + (size_t)t * n1; };
  std::vector<DedupView> v((size_t)count);
  for (int i = 0; i < count; ++i) {
    mape_dedup_item& it = items[i];
    it.K = 0;
    it.status = MAPE_OK;
    DedupView& d = v[(size_t)i];
    d = DedupView{};
    d.rows = it.cand;
    d.count = it.count;
    d.ldc = it.ldc;
    d.uniq = it.uniq;
    if (it.count == 0) continue;
    // the same carve as mape_dedup
    Carver cv(it.workspace, it.workspace_bytes);
    d.h = cv.take<uint64_t>((size_t)it.count);
    const uint64_t slots = dedup_table_slots(it.count);
    d.table = cv.take<uint32_t>((size_t)slots);
    d.mask = slots - 1;
    d.is_rep = cv.take<uint8_t>((size_t)it.count);
    const uint64_t npad_cap = next_pow2((uint64_t)it.count);
    d.idx = cv.take<uint32_t>((size_t)npad_cap);
    d.key = cv.take<uint64_t>((size_t)npad_cap);
    d.runs = cv.take<int2>((size_t)it.count / 2 + 1);
    cv.take<unsigned int>(3);
    cv.take<unsigned long long>(1);
    if (!cv.ok) {
      it.status = MAPE_ERR_CAPACITY;
      return MAPE_ERR_CAPACITY;
    }
    MAPE_CUDA_TRY(cudaMemsetAsync(d.table, 0xff, slots * sizeof(uint32_t), st));
  }
  // 1. hash, insert, compact over the rows of every set
  const int64_t rows = prefix(kPxRows, [&](int i) { return v[(size_t)i].count; });
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_views, v.data(), sizeof(DedupView) * count, cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_px, px.data(), sizeof(int64_t) * n1, cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(d_K, 0, sizeof(unsigned long long) * count, st));
  if (rows > 0) {
    const unsigned g = (unsigned)ceil_div(rows, 256);
    for (int phase = 0; phase < 3; ++phase)
      launch(hash_insert_batch_kernel, g, 256, 0, st, (const DedupView*)d_views, dpx(kPxRows), (int)count, phase, d_K);
    MAPE_LAUNCH_CHECK();
  }
  std::vector<unsigned long long> hK((size_t)count, 0);
  MAPE_CUDA_TRY(cudaMemcpyAsync(hK.data(), d_K, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  int first_err = MAPE_OK;
  int64_t max_npad = 0;
  for (int i = 0; i < count; ++i) {
    mape_dedup_item& it = items[i];
    DedupView& d = v[(size_t)i];
    it.K = (int64_t)hK[(size_t)i];
    d.K = it.K;
    if (it.K > it.uniq_cap || (it.K > 0 && !it.uniq)) {  // as mape_dedup: the count only
      it.status = it.K > it.uniq_cap ? MAPE_ERR_CAPACITY : MAPE_ERR_INVALID_ARG;
      if (first_err == MAPE_OK) first_err = it.status;
      d.K = 0;
    }
    d.npad = d.K > 0 ? (int64_t)next_pow2((uint64_t)d.K) : 0;
    d.seg = d.npad >= 2 ? (d.npad < kSeg ? d.npad : kSeg) : 0;
    d.runs_cap = d.K / 2 + 1;
    if (d.seg) max_npad = std::max(max_npad, d.npad);
  }
  // 2. keys and the bitonic network on them, for the largest set
  const int64_t pos = prefix(kPxPos, [&](int i) { return v[(size_t)i].npad; });
  const int64_t segs = prefix(kPxSegs, [&](int i) { return v[(size_t)i].seg ? v[(size_t)i].npad / v[(size_t)i].seg : 0; });
  const int64_t keyed = prefix(kPxKeyed, [&](int i) { return v[(size_t)i].seg ? v[(size_t)i].K : 0; });
  const int64_t pieces = prefix(kPxPieces, [&](int i) { return v[(size_t)i].K * (v[(size_t)i].ldc / 16); });
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_views, v.data(), sizeof(DedupView) * count, cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_px, px.data(), sizeof(int64_t) * kPxShort * n1, cudaMemcpyHostToDevice, st));
  if (pos > 0)
    launch(key_batch_kernel, (unsigned)ceil_div(pos, 256), 256, 0, st, (const DedupView*)d_views, dpx(kPxPos),
           (int)count);
  if (max_npad >= 2) {
    launch(bitonic_local_batch_kernel, (unsigned)segs, kSeg / 2, 0, st, (const DedupView*)d_views, dpx(kPxSegs),
           (int)count, (int64_t)0);
    for (int64_t k = 2 * kSeg; k <= max_npad; k <<= 1) {
      for (int64_t j = k >> 1; j >= kSeg; j >>= 1)
        launch(bitonic_step_batch_kernel, (unsigned)ceil_div(pos, 256), 256, 0, st, (const DedupView*)d_views,
               dpx(kPxPos), (int)count, j, k);
      launch(bitonic_local_batch_kernel, (unsigned)segs, kSeg / 2, 0, st, (const DedupView*)d_views, dpx(kPxSegs),
             (int)count, k);
    }
    MAPE_LAUNCH_CHECK();
    // 3. runs of equal keys, sorted by the rows' remaining bytes
    MAPE_CUDA_TRY(cudaMemsetAsync(d_runc, 0, sizeof(unsigned int) * 3 * count, st));
    launch(key_runs_batch_kernel, (unsigned)ceil_div(keyed, 256), 256, 0, st, (const DedupView*)d_views,
           dpx(kPxKeyed), (int)count, d_runc);
    MAPE_LAUNCH_CHECK();
    std::vector<unsigned int> hc((size_t)3 * count, 0);
    MAPE_CUDA_TRY(cudaMemcpyAsync(hc.data(), d_runc, sizeof(unsigned int) * 3 * count, cudaMemcpyDeviceToHost, st));
    MAPE_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < count; ++i) {
      DedupView& d = v[(size_t)i];
      if (!d.seg) continue;
      if (hc[(size_t)3 * i + 2] > (unsigned)kRunMax) {  // a run too long for one block: the rows decide every comparison
        bitonic_sort<true>(d.rows, d.ldc, d.idx, d.key, d.npad, st);
      } else {
        d.nshort = hc[(size_t)3 * i];
        d.nlong = hc[(size_t)3 * i + 1];
      }
    }
    const int64_t nshort = prefix(kPxShort, [&](int i) { return v[(size_t)i].nshort; });
    const int64_t nlong = prefix(kPxLong, [&](int i) { return v[(size_t)i].nlong; });
    MAPE_CUDA_TRY(cudaMemcpyAsync(d_views, v.data(), sizeof(DedupView) * count, cudaMemcpyHostToDevice, st));
    MAPE_CUDA_TRY(cudaMemcpyAsync(d_px + (size_t)kPxShort * n1, px.data() + (size_t)kPxShort * n1,
                                  sizeof(int64_t) * 2 * n1, cudaMemcpyHostToDevice, st));
    if (nshort > 0)
      launch(run_sort_warp_batch_kernel, (unsigned)ceil_div(nshort, kRunWarps), 32 * kRunWarps,
             (size_t)kRunWarps * kRunWarpBytes, st, (const DedupView*)d_views, dpx(kPxShort), (int)count);
    if (nlong > 0)
      launch(run_sort_batch_kernel, (unsigned)nlong, 128, kRunStageBytes, st, (const DedupView*)d_views, dpx(kPxLong),
             (int)count);
    MAPE_LAUNCH_CHECK();
  }
  // 4. the distinct rows in order
  if (pieces > 0)
    launch(gather_batch_kernel, (unsigned)ceil_div(pieces, 256), 256, 0, st, (const DedupView*)d_views,
           dpx(kPxPieces), (int)count);
  MAPE_LAUNCH_CHECK();
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  return first_err;
}
