// a12-a14: Algorithm 1 (§2) with the direction set as test set, for S starts
// at once, in exact int64 arithmetic.
//
// For f(x) = x^T Q x + c^T x + sum_i w_i x_i^4 and a move x -> x + lambda e g
// (e = +-1, lambda >= 1):
//   Delta f = lambda^2 a_g + lambda e g^T r + sum_i w_i ((x_i + lambda e g_i)^4 - x_i^4)
// with a_g = g^T Q g and r = 2 Q x + c; the quartic part expands to
//   4 e lambda sum w x^3 g + 6 lambda^2 sum w x^2 g^2 + 4 e lambda^3 sum w x g^3
//   + lambda^4 sum w g^4.
// The largest feasible lambda is lambda_max = min over e g_i > 0 of
// floor((u_i - x_i)/(e g_i)) and over e g_i < 0 of floor((x_i - l_i)/(-e g_i)).
// Without the quartic term the best lambda in [1, lambda_max] is the integer
// next to the vertex -e b/(2a) (a > 0) or an end point (a <= 0); with it,
// every lambda in [1, lambda_max] is evaluated.  Candidates are ordered by
// (Delta f, k, e = +1 first, lambda); the order is total, so the argmin does
// not depend on the reduction order, nor on how the directions are spread
// over threads and blocks.
//
// The scoring pass reads every direction once per iteration.  L lanes share a
// direction (L = 1 .. 32, a power of two): lane j takes the row's 16-byte
// pieces j, j + L, ..., and the group combines its partial sums (exact int64)
// and lambda bounds by shuffles; L is autotuned per shape (a few timed score
// passes on the call's own data, which the pass does not modify) unless the
// caller fixes it.  A block visits directions in a grid-stride loop, so that
// at most kMaxScoreBlocks partial minima per start go to the apply pass.
//
// Many instances at once (mape_augment_run_batch): one score and one apply
// launch per iteration cover the starts of every instance, each block finding
// its instance by binary search over the launch's prefix table; an iteration
// counter on the device lets a chunk of iterations be captured once as a CUDA
// graph and replayed until every start of every instance has stopped.
#include "common.cuh"

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace {

using namespace mape_detail;

struct Best {
  long long df;
  long long key;  // k * 512 + (e < 0) * 256 + lambda
};

__device__ __forceinline__ bool better(const Best& a, const Best& b) {
  return a.df < b.df || (a.df == b.df && a.key < b.key);
}

constexpr long long kNoMove = 0x7fffffffffffffffll;

__device__ __forceinline__ Best warp_min(Best v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Best o;
    o.df = __shfl_xor_sync(0xffffffffu, v.df, off);
    o.key = __shfl_xor_sync(0xffffffffu, v.key, off);
    if (better(o, v)) v = o;
  }
  return v;
}

// One warp per group of directions: the lanes take the entries of Q
// (coalesced) and of w, the directions' rows are staged in shared memory, a
// warp reduction sums (integer arithmetic, exact in any order).
constexpr int kCoefWarps = 8;
constexpr int kCoefMaxRow = 4096;  // ldg <= 4096 bytes (n <= 4096)

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// directions k0 .. k0 + cnt - 1 (cnt <= kCoefRows) by the calling warp (g:
// its kCoefRows shared-memory rows, ldg bytes apart): each entry of Q and w
// is loaded once for all of them, and their sums are independent chains
constexpr int kCoefRows = 4;

__device__ __forceinline__ void coeffs_rows(const int32_t* __restrict__ qr, const int32_t* __restrict__ qc,
                                            const int32_t* __restrict__ qv, int nnz, const int32_t* __restrict__ w,
                                            int n, const int8_t* __restrict__ G, int64_t k0, int cnt, int ldg,
                                            int vec, int8_t* g, int64_t* __restrict__ a, int64_t* __restrict__ q4) {
  const int lane = threadIdx.x & 31;
  for (int q = 0; q < cnt; ++q) {
    if (vec) {  // rows 16-byte aligned (ldg a multiple of 16, G aligned)
      const uint4* src = reinterpret_cast<const uint4*>(G + (k0 + q) * ldg);
      for (int c = lane; c < ldg / 16; c += 32) reinterpret_cast<uint4*>(g + q * ldg)[c] = src[c];
    } else {
      for (int c = lane; c < n; c += 32) g[q * ldg + c] = G[(k0 + q) * ldg + c];
    }
  }
  __syncwarp();
  // products of int8 entries in 32 bits (|g_i g_j| <= 2^14, twice that off
  // the diagonal; g^4 <= 2^28), then one 32 x 32 -> 64-bit product each
  long long acc[kCoefRows] = {0, 0, 0, 0};
  for (int e = lane; e < nnz; e += 32) {
    const int i = qr[e], j = qc[e];
    const int f = (i == j) ? 1 : 2;
    const long long v = qv[e];
#pragma unroll
    for (int q = 0; q < kCoefRows; ++q)
      acc[q] += v * (f * (int)g[q * ldg + i] * (int)g[q * ldg + j]);  // rows past cnt: unused
  }
  long long s4[kCoefRows] = {0, 0, 0, 0};
  if (w)
    for (int i = lane; i < n; i += 32) {
      const long long wi = w[i];
#pragma unroll
      for (int q = 0; q < kCoefRows; ++q) {
        const int gi = g[q * ldg + i];
        const int g2 = gi * gi;
        s4[q] += wi * (g2 * g2);
      }
    }
#pragma unroll
  for (int q = 0; q < kCoefRows; ++q) {
    const long long sa = warp_sum_ll(acc[q]), sq = warp_sum_ll(s4[q]);
    if (lane == 0 && q < cnt) {
      a[k0 + q] = sa;
      q4[k0 + q] = sq;
    }
  }
}

// dynamic shared memory: kCoefWarps x kCoefRows rows of ldg bytes
__global__ void coeffs_kernel(const int32_t* __restrict__ qr, const int32_t* __restrict__ qc,
                              const int32_t* __restrict__ qv, int nnz, const int32_t* __restrict__ w, int n,
                              const int8_t* __restrict__ G, int64_t K, int ldg, int vec, int64_t* __restrict__ a,
                              int64_t* __restrict__ q4) {
  extern __shared__ __align__(16) int8_t s_rows[];
  const int wid = threadIdx.x >> 5;
  const int64_t k0 = ((int64_t)blockIdx.x * kCoefWarps + wid) * kCoefRows;
  if (k0 >= K) return;  // warp-uniform
  coeffs_rows(qr, qc, qv, nnz, w, n, G, k0, (int)(K - k0 < kCoefRows ? K - k0 : kCoefRows), ldg, vec,
              s_rows + (size_t)wid * kCoefRows * ldg, a, q4);
}

// many instances: a warp per group of kCoefRows directions of any instance,
// the instance found by binary search over the groups' prefix table; dynamic
// shared memory kCoefWarps x kCoefRows rows of max_ldg bytes
__global__ void coeffs_batch_kernel(const mape_coeffs_item* __restrict__ items, const int64_t* __restrict__ prefix,
                                    const int32_t* __restrict__ vec, int count, int max_ldg) {
  extern __shared__ __align__(16) int8_t s_rows[];
  const int wid = threadIdx.x >> 5;
  const int64_t g = (int64_t)blockIdx.x * kCoefWarps + wid;
  if (g >= prefix[count]) return;  // warp-uniform
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const mape_coeffs_item& it = items[lo];
  const int64_t k0 = (g - prefix[lo]) * kCoefRows;
  coeffs_rows(it.q_row, it.q_col, it.q_val, it.nnz, it.w, it.n, it.G, k0,
              (int)(it.K - k0 < kCoefRows ? it.K - k0 : kCoefRows), it.ldg, vec[lo],
              s_rows + (size_t)wid * kCoefRows * max_ldg, it.a, it.q4);
}

// One instance's arguments and its workspace, as the kernels see them.
struct AugView {
  const int8_t* G;
  int64_t K;
  int ldg, n, S, nb;  // nb: score blocks per start
  const int64_t* a;
  const int64_t* q4;
  const int32_t *qr, *qc, *qv;
  int nnz, moves_cap;
  const int32_t *c, *w, *l, *u;
  int32_t* X;
  int64_t* fval;
  int64_t* moves;
  int32_t* nmoves;
  long long* R;
  uint8_t* active;
  Best* partial;
  int32_t* iters;
  unsigned int* n_active;
  int32_t* bad;
  int64_t max_iters;
};

constexpr int kScoreThreads = 256;
constexpr int kMaxScoreBlocks = 1024;  // per start

// r = 2 Q x + c and f(x) of start s; checks l <= x <= u.
__device__ __forceinline__ void init_body(const AugView& v, int s) {
  const int n = v.n;
  const int32_t* x = v.X + (int64_t)s * n;
  long long* r = v.R + (int64_t)s * n;
  __shared__ long long s_f[32];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    r[i] = v.c[i];
    if (x[i] < v.l[i] || x[i] > v.u[i]) atomicOr(v.bad, 1);
  }
  __syncthreads();
  long long f = 0;
  for (int e = threadIdx.x; e < v.nnz; e += blockDim.x) {
    int i = v.qr[e], j = v.qc[e];
    long long q = v.qv[e];
    atomicAdd((unsigned long long*)&r[i], (unsigned long long)(2 * q * x[j]));
    if (i != j) atomicAdd((unsigned long long*)&r[j], (unsigned long long)(2 * q * x[i]));
    f += (i == j ? 1 : 2) * q * x[i] * x[j];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    long long xi = x[i];
    f += (long long)v.c[i] * xi;
    if (v.w) f += (long long)v.w[i] * xi * xi * xi * xi;
  }
  for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
  if ((threadIdx.x & 31) == 0) s_f[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_f[i];
    v.fval[s] = t;
    v.active[s] = 1;
  }
}

__device__ __forceinline__ long long floor_div(long long a, long long b) {  // b > 0
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

// The per-start tables the score pass reads for every direction, by
// coordinate i: rw[2 i] = (r_i, w x_i^3), rw[2 i + 1] = (w x_i^2, w x_i) with
// r = 2 Q x + c (the w terms 0 without the quartic term), ud[i] = (u - x,
// x - l), so that an entry takes one 16-byte load (two with the quartic term)
// and one 8-byte load.
struct ScoreSmem {
  longlong2* rw;
  int2* ud;
  const uint32_t* rcp;  // rcp[b] = ceil(2^20 / b), b = 1 .. 128
};

// floor(a / b) for 0 <= a < 2048 and 1 <= b <= 128 as (a ceil(2^20 / b)) >> 20:
// with ceil(2^20 / b) = (2^20 + e) / b, 0 <= e < b, the product is
// 2^20 (a / b) + a e / b and a e < 2^20, so the shift drops only the fraction
// (division by an invariant integer by multiplication, Granlund and
// Montgomery, PLDI 1994).  Other operands take the division instruction.
// The steps' spans u - x, x - l lie in [0, 127] and |g_i| <= 128 (int8).
constexpr int kRcpShift = 20;
__device__ __forceinline__ int div_small(int a, int b, const uint32_t* rcp) {
  if ((unsigned)a < 2048u && b <= 128) return (int)(((uint32_t)a * rcp[b]) >> kRcpShift);
  return a / b;
}

__device__ __forceinline__ ScoreSmem stage_start(const AugView& v, int s) {
  extern __shared__ __align__(16) long long smem[];
  const int n = v.n;
  ScoreSmem t;
  t.rw = reinterpret_cast<longlong2*>(smem);                 // 32 n bytes
  t.ud = reinterpret_cast<int2*>(smem + 4 * (int64_t)n);    // 8 n bytes
  __shared__ uint32_t s_rcp[129];
  for (int b = threadIdx.x; b <= 128; b += blockDim.x)
    s_rcp[b] = b ? ((1u << kRcpShift) + (uint32_t)b - 1u) / (uint32_t)b : 0u;
  t.rcp = s_rcp;
  const int32_t* x = v.X + (int64_t)s * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const long long xi = x[i];
    const long long wi = v.w ? v.w[i] : 0;
    t.rw[2 * i] = make_longlong2(v.R[(int64_t)s * n + i], wi * xi * xi * xi);
    t.rw[2 * i + 1] = make_longlong2(wi * xi * xi, wi * xi);
    t.ud[i] = make_int2(v.u[i] - x[i], x[i] - v.l[i]);
  }
  return t;
}

// Partial sums of one direction over the entries a lane visits.
struct DirSums {
  long long b = 0, c1 = 0, c2 = 0, c3 = 0;
  int lam_p = 0x7fffffff, lam_m = 0x7fffffff;  // lambda_max for +g and -g
};

__device__ __forceinline__ void add_entry(DirSums& d, const ScoreSmem& t, bool quartic, int i, int gi) {
  const longlong2 rw = t.rw[2 * i];
  d.b += (long long)gi * rw.x;
  if (quartic) {  // g^2 <= 2^14 and |g^3| <= 2^21: one 64 x 32-bit product each
    const longlong2 ww = t.rw[2 * i + 1];
    const int g2 = gi * gi;
    d.c1 += rw.y * gi;
    d.c2 += ww.x * g2;
    d.c3 += ww.y * (g2 * gi);
  }
  const int2 ud = t.ud[i];
  const int ag = abs(gi);
  const int up = div_small(ud.x, ag, t.rcp), dn = div_small(ud.y, ag, t.rcp);  // both nonnegative
  if (gi > 0) { d.lam_p = min(d.lam_p, up); d.lam_m = min(d.lam_m, dn); }
  else        { d.lam_p = min(d.lam_p, dn); d.lam_m = min(d.lam_m, up); }
}

// The best move along +-g_k given the direction's sums.
__device__ __forceinline__ void best_move(const AugView& v, int64_t k, const DirSums& d, Best& best) {
  long long ak = v.a[k];
  long long c4 = v.q4[k];
  for (int e = 1; e >= -1; e -= 2) {
    int L = (e > 0) ? d.lam_p : d.lam_m;
    // L <= max(u - l) <= 127 for a nonzero row; a zero row has no move
    if (L < 1 || L > 255) continue;
    long long eb = e * d.b;
    if (!v.w) {
      long long cand[2];
      if (ak > 0) {
        // vertex at -eb / (2 a); the integer minimiser is floor or ceil of it
        long long fl = floor_div(-eb, 2 * ak);
        cand[0] = fl;
        cand[1] = fl + 1;
      } else {
        cand[0] = 1;
        cand[1] = L;
      }
      for (int q = 0; q < 2; ++q) {
        long long lam = cand[q] < 1 ? 1 : (cand[q] > L ? L : cand[q]);
        long long df = lam * lam * ak + lam * eb;
        Best cb{df, k * 512 + (e < 0 ? 256 : 0) + lam};
        if (better(cb, best)) best = cb;
      }
    } else {
      for (int lam = 1; lam <= L; ++lam) {
        long long lm = lam;
        long long df = lm * lm * ak + lm * eb + 4 * e * lm * d.c1 + 6 * lm * lm * d.c2 +
                       4 * e * lm * lm * lm * d.c3 + lm * lm * lm * lm * c4;
        Best cb{df, k * 512 + (e < 0 ? 256 : 0) + lm};
        if (better(cb, best)) best = cb;
      }
    }
  }
}

// Score block bx of start s.  kL lanes per direction; kVec: the rows are read
// as 16-byte pieces (ldg a multiple of 16, G 16-byte aligned), else byte by
// byte (kL = 1).
template <int kL, bool kVec>
__device__ __forceinline__ void score_body(const AugView& v, int s, int bx) {
  if (!v.active[s]) return;  // block-uniform
  const ScoreSmem t = stage_start(v, s);
  __syncthreads();
  const int n = v.n;
  const bool quartic = v.w != nullptr;
  const int sub = threadIdx.x % kL;
  const int per_block = blockDim.x / kL;  // directions per block and round
  Best best{kNoMove, kNoMove};
  for (int64_t k0 = (int64_t)bx * per_block; k0 < v.K; k0 += (int64_t)v.nb * per_block) {  // block-uniform
    const int64_t k = k0 + threadIdx.x / kL;
    DirSums d;
    if (k < v.K) {
      const int8_t* g = v.G + k * v.ldg;
      if (kVec) {
        for (int p = sub; p * 16 < n; p += kL) {
          const int4 q = *reinterpret_cast<const int4*>(g + p * 16);
          const uint32_t w4[4] = {(uint32_t)q.x, (uint32_t)q.y, (uint32_t)q.z, (uint32_t)q.w};
#pragma unroll
          for (int b = 0; b < 16; ++b) {
            const int i = p * 16 + b;
            const int gi = (int)(int8_t)(w4[b >> 2] >> (8 * (b & 3)));
            if (gi != 0 && i < n) add_entry(d, t, quartic, i, gi);
          }
        }
      } else {
        for (int i = 0; i < n; ++i) {
          const int gi = g[i];
          if (gi != 0) add_entry(d, t, quartic, i, gi);
        }
      }
    }
    if (kL > 1) {  // the group's lanes are consecutive within one warp
#pragma unroll
      for (int o = kL / 2; o > 0; o >>= 1) {
        d.b += __shfl_xor_sync(0xffffffffu, d.b, o);
        d.c1 += __shfl_xor_sync(0xffffffffu, d.c1, o);
        d.c2 += __shfl_xor_sync(0xffffffffu, d.c2, o);
        d.c3 += __shfl_xor_sync(0xffffffffu, d.c3, o);
        d.lam_p = min(d.lam_p, __shfl_xor_sync(0xffffffffu, d.lam_p, o));
        d.lam_m = min(d.lam_m, __shfl_xor_sync(0xffffffffu, d.lam_m, o));
      }
    }
    if (k < v.K && sub == 0) best_move(v, k, d, best);
  }
  // block argmin
  __shared__ Best s_best[32];
  best = warp_min(best);
  if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    Best b = threadIdx.x < (blockDim.x >> 5) ? s_best[threadIdx.x] : Best{kNoMove, kNoMove};
    b = warp_min(b);
    if (threadIdx.x == 0) v.partial[(int64_t)s * v.nb + bx] = b;
  }
}

// Final argmin of start s over its score blocks; move or stop.
__device__ __forceinline__ void apply_body(const AugView& v, int s) {
  if (!v.active[s]) return;
  __shared__ Best s_best[32];
  Best best{kNoMove, kNoMove};
  for (int b = threadIdx.x; b < v.nb; b += blockDim.x) {
    Best p = v.partial[(int64_t)s * v.nb + b];
    if (better(p, best)) best = p;
  }
  best = warp_min(best);
  if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    Best p = threadIdx.x < (blockDim.x >> 5) ? s_best[threadIdx.x] : Best{kNoMove, kNoMove};
    p = warp_min(p);
    if (threadIdx.x == 0) s_best[0] = p;
  }
  __syncthreads();
  best = s_best[0];
  if (threadIdx.x == 0) v.iters[s] += 1;
  if (best.df >= 0) {  // no improving move: this start is done
    if (threadIdx.x == 0) {
      v.active[s] = 0;
      atomicSub(v.n_active, 1u);
    }
    return;
  }
  const int n = v.n;
  long long k = best.key >> 9;
  int e = (best.key & 256) ? -1 : 1;
  long long lam = best.key & 255;
  long long step = e * lam;
  const int8_t* g = v.G + k * v.ldg;
  int32_t* x = v.X + (int64_t)s * n;
  long long* r = v.R + (int64_t)s * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] += (int32_t)(step * g[i]);
  for (int q = threadIdx.x; q < v.nnz; q += blockDim.x) {
    int i = v.qr[q], j = v.qc[q];
    long long val = v.qv[q];
    atomicAdd((unsigned long long*)&r[i], (unsigned long long)(2 * step * val * g[j]));
    if (i != j) atomicAdd((unsigned long long*)&r[j], (unsigned long long)(2 * step * val * g[i]));
  }
  if (threadIdx.x == 0) {
    long long fnew = v.fval[s] + best.df;
    v.fval[s] = fnew;
    int m = v.nmoves ? v.nmoves[s] : 0;
    if (v.moves && m < v.moves_cap) {
      int64_t* mv = v.moves + ((int64_t)s * v.moves_cap + m) * 4;
      mv[0] = k;
      mv[1] = e;
      mv[2] = lam;
      mv[3] = fnew;
    }
    if (v.nmoves) v.nmoves[s] = m + 1;
  }
}

__global__ void init_kernel(AugView v) { init_body(v, blockIdx.x); }

template <int kL, bool kVec>
__global__ void score_kernel(AugView v) { score_body<kL, kVec>(v, blockIdx.y, blockIdx.x); }

__global__ void apply_kernel(AugView v) { apply_body(v, blockIdx.x); }

// ---- many instances: block b of a launch belongs to the instance i with
// prefix[i] <= b < prefix[i + 1] (prefix of `count` + 1 entries)
__device__ __forceinline__ int find_item(const int64_t* __restrict__ prefix, int count, int64_t b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void init_batch_kernel(const AugView* __restrict__ items, const int64_t* __restrict__ st_prefix,
                                  int count) {
  const int i = find_item(st_prefix, count, blockIdx.x);
  const AugView v = items[i];
  init_body(v, (int)(blockIdx.x - st_prefix[i]));
}

// iteration *iter: instances past their max_iters (or without directions) sit out
template <int kL, bool kVec>
__global__ void score_batch_kernel(const AugView* __restrict__ items, const int64_t* __restrict__ blk_prefix,
                                   int count, const int64_t* __restrict__ iter) {
  const int i = find_item(blk_prefix, count, blockIdx.x);
  const AugView v = items[i];
  if (*iter >= v.max_iters || v.K == 0) return;
  const int64_t b = blockIdx.x - blk_prefix[i];
  score_body<kL, kVec>(v, (int)(b / v.nb), (int)(b % v.nb));
}

__global__ void apply_batch_kernel(const AugView* __restrict__ items, const int64_t* __restrict__ st_prefix,
                                   int count, const int64_t* __restrict__ iter) {
  const int i = find_item(st_prefix, count, blockIdx.x);
  const AugView v = items[i];
  if (*iter >= v.max_iters || v.K == 0) return;
  apply_body(v, (int)(blockIdx.x - st_prefix[i]));
}

__global__ void tick_kernel(int64_t* iter) { *iter += 1; }

// per instance: the largest iteration count over its starts
__global__ void iters_max_kernel(const AugView* __restrict__ items, int count, int64_t* __restrict__ out) {
  const int i = blockIdx.x;
  if (i >= count) return;
  const AugView v = items[i];
  int m = 0;
  for (int s = threadIdx.x; s < v.S; s += blockDim.x) m = max(m, v.iters[s]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ int s_m[32];
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = max(t, s_m[w]);
    out[i] = t;
  }
}

// ---- the variants of the score pass: kL lanes per direction, 16-byte pieces
// or bytes
using ScoreFn = void (*)(AugView);
using ScoreBatchFn = void (*)(const AugView*, const int64_t*, int, const int64_t*);

constexpr int kLaneChoices[] = {1, 2, 4, 8, 16, 32};

ScoreFn score_fn(int lanes, bool vec) {
  if (!vec) return score_kernel<1, false>;
  switch (lanes) {
    case 1: return score_kernel<1, true>;
    case 2: return score_kernel<2, true>;
    case 4: return score_kernel<4, true>;
    case 8: return score_kernel<8, true>;
    case 16: return score_kernel<16, true>;
    default: return score_kernel<32, true>;
  }
}

ScoreBatchFn score_batch_fn(int lanes, bool vec) {
  if (!vec) return score_batch_kernel<1, false>;
  switch (lanes) {
    case 1: return score_batch_kernel<1, true>;
    case 2: return score_batch_kernel<2, true>;
    case 4: return score_batch_kernel<4, true>;
    case 8: return score_batch_kernel<8, true>;
    case 16: return score_batch_kernel<16, true>;
    default: return score_batch_kernel<32, true>;
  }
}

bool valid_lanes(int lanes) {
  for (int c : kLaneChoices)
    if (c == lanes) return true;
  return false;
}

int score_blocks(int64_t K, int lanes) {
  const int64_t per_block = kScoreThreads / lanes;
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(K, per_block), kMaxScoreBlocks));
}

size_t score_smem(int n) { return (size_t)n * (4 * sizeof(long long) + 2 * sizeof(int32_t)); }

// the shared-memory limit of every variant that may take more than 48 KB
int allow_score_smem(size_t smem, bool batch) {
  if (smem <= 48 * 1024) return MAPE_OK;
  for (int lanes : kLaneChoices)
    for (bool vec : {true, false}) {
      if (!vec && lanes != 1) continue;
      size_t lim = 0;
      const void* f = batch ? (const void*)score_batch_fn(lanes, vec) : (const void*)score_fn(lanes, vec);
      const int rc = allow_max_dynamic_smem(f, &lim);
      if (rc != MAPE_OK) return rc;
      if (smem > lim) return MAPE_ERR_SHAPE;
    }
  return MAPE_OK;
}

// ---- autotuned lanes per direction, per shape class
struct AugTuneKey {
  int n;
  int64_t kb;  // K rounded up to a power of two
  int sb;      // S rounded up to a power of two
  int quartic;
  bool operator<(const AugTuneKey& o) const {
    return std::tie(n, kb, sb, quartic) < std::tie(o.n, o.kb, o.sb, o.quartic);
  }
};

std::mutex g_aug_tune_mu;
std::map<AugTuneKey, mape_augment_tune_info> g_aug_tuned;

int64_t pow2_at_least(int64_t x) {
  int64_t b = 1;
  while (b < x && b < ((int64_t)1 << 40)) b <<= 1;
  return b;
}

AugTuneKey tune_key(int n, int64_t K, int S, bool quartic) {
  return AugTuneKey{n, pow2_at_least(K), (int)pow2_at_least(S), quartic ? 1 : 0};
}

AugView make_view(const mape_augment_args* A, long long* R, uint8_t* active, Best* partial, int32_t* iters,
                  unsigned int* n_active, int32_t* bad, int32_t* nmoves, int lanes) {
  AugView v{};
  v.G = A->G; v.K = A->K; v.ldg = A->ldg; v.n = A->n; v.S = A->S; v.nb = score_blocks(A->K, lanes);
  v.a = A->a; v.q4 = A->q4; v.qr = A->q_row; v.qc = A->q_col; v.qv = A->q_val; v.nnz = A->nnz;
  v.moves_cap = A->moves_cap;
  v.c = A->c; v.w = A->w; v.l = A->l; v.u = A->u; v.X = A->X; v.fval = A->fval;
  v.moves = A->moves; v.nmoves = nmoves;
  v.R = R; v.active = active; v.partial = partial; v.iters = iters; v.n_active = n_active; v.bad = bad;
  v.max_iters = A->max_iters;
  return v;
}

// Times one score pass of every lane count on the start's state (the pass
// writes only the partial minima) and returns the fastest.
int tune_lanes(const AugView& base, size_t smem, cudaStream_t st, mape_augment_tune_info* out) {
  cudaEvent_t e0, e1;
  MAPE_CUDA_TRY(cudaEventCreate(&e0));
  MAPE_CUDA_TRY(cudaEventCreate(&e1));
  *out = mape_augment_tune_info{};
  float best = 1e30f;
  int nc = 0;
  for (int lanes : kLaneChoices) {
    AugView v = base;
    v.nb = score_blocks(v.K, lanes);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch loads the kernel
      MAPE_CUDA_TRY(cudaEventRecord(e0, st));
      launch(score_fn(lanes, true), dim3((unsigned)v.nb, (unsigned)v.S), kScoreThreads, smem, st, v);
      MAPE_CUDA_TRY(cudaEventRecord(e1, st));
      MAPE_CUDA_TRY(cudaEventSynchronize(e1));
      MAPE_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    }
    out->cand_lanes[nc] = lanes;
    out->probe_ms[nc] = ms;
    ++nc;
    if (ms < best) {
      best = ms;
      out->lanes = lanes;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  out->candidates = nc;
  return MAPE_OK;
}

// The lane count of a call: the caller's, or the autotuned one for its shape
// (tuned on this call's state if the shape is new).
int pick_lanes(const mape_augment_args* A, const AugView& v, bool vec, size_t smem, cudaStream_t st, int* lanes) {
  if (!vec) {
    *lanes = 1;
    return MAPE_OK;
  }
  if (A->score_lanes != 0) {
    *lanes = A->score_lanes;
    return MAPE_OK;
  }
  const AugTuneKey key = tune_key(A->n, A->K, A->S, A->w != nullptr);
  {
    std::lock_guard<std::mutex> lk(g_aug_tune_mu);
    auto it = g_aug_tuned.find(key);
    if (it != g_aug_tuned.end()) {
      *lanes = it->second.lanes;
      return MAPE_OK;
    }
  }
  mape_augment_tune_info info{};
  const int rc = tune_lanes(v, smem, st, &info);
  if (rc != MAPE_OK) return rc;
  std::lock_guard<std::mutex> lk(g_aug_tune_mu);
  g_aug_tuned[key] = info;
  *lanes = info.lanes;
  return MAPE_OK;
}

bool rows_vectorisable(const mape_augment_args* A) {
  return A->ldg % 16 == 0 && (reinterpret_cast<uintptr_t>(A->G) & 15) == 0;
}

int check_args(const mape_augment_args* A) {
  const int n = A->n, S = A->S;
  const int64_t K = A->K;
  if (n <= 0 || S < 0 || K < 0 || A->ldg < n || A->max_iters < 0) return MAPE_ERR_INVALID_ARG;
  if (S > 0 && (!A->X || !A->fval || !A->c || !A->l || !A->u)) return MAPE_ERR_INVALID_ARG;
  if (K > 0 && (!A->G || !A->a || !A->q4)) return MAPE_ERR_INVALID_ARG;
  if (A->nnz > 0 && (!A->q_row || !A->q_col || !A->q_val)) return MAPE_ERR_INVALID_ARG;
  if (A->moves && A->moves_cap <= 0) return MAPE_ERR_INVALID_ARG;
  if (A->score_lanes != 0 && !valid_lanes(A->score_lanes)) return MAPE_ERR_INVALID_ARG;
  if (K >= ((int64_t)1 << 40)) return MAPE_ERR_SHAPE;
  return MAPE_OK;
}

// The per-instance workspace pieces (the same carve for a single run and a batch).
struct AugCarve {
  long long* R;
  uint8_t* active;
  Best* partial;
  int32_t* iters;
  unsigned int* n_active;
  int32_t* bad;
  int32_t* own_nmoves;
  bool ok;
};

AugCarve carve(const mape_augment_args* A) {
  const int n = A->n, S = A->S;
  Carver cv(A->workspace, A->workspace_bytes);
  AugCarve c{};
  c.R = cv.take<long long>((size_t)S * n);
  c.active = cv.take<uint8_t>((size_t)S);
  c.partial = cv.take<Best>((size_t)S * kMaxScoreBlocks);
  c.iters = cv.take<int32_t>((size_t)S);
  c.n_active = cv.take<unsigned int>(1);
  c.bad = cv.take<int32_t>(1);
  c.own_nmoves = cv.take<int32_t>((size_t)S);
  c.ok = cv.ok;
  return c;
}

}  // namespace

namespace mape_detail {
void augment_tune_clear() {
  std::lock_guard<std::mutex> lk(g_aug_tune_mu);
  g_aug_tuned.clear();
}
}  // namespace mape_detail

extern "C" int mape_augment_tune_lookup(int32_t n, int64_t K, int32_t S, int32_t quartic,
                                        mape_augment_tune_info* out) {
  if (!out) return MAPE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_aug_tune_mu);
  auto it = g_aug_tuned.find(tune_key(n, K, S, quartic != 0));
  if (it == g_aug_tuned.end()) return MAPE_ERR_STATE;
  *out = it->second;
  return MAPE_OK;
}

extern "C" int mape_direction_coeffs(const int32_t* q_row, const int32_t* q_col, const int32_t* q_val,
                                     int32_t nnz, const int32_t* w, int32_t n, const int8_t* G, int64_t K,
                                     int32_t ldg, int64_t* a, int64_t* q4, void* stream) {
  using namespace mape_detail;
  if (nnz < 0 || n <= 0 || ldg < n || K < 0 || (nnz > 0 && (!q_row || !q_col || !q_val)) ||
      (K > 0 && (!G || !a || !q4)))
    return MAPE_ERR_INVALID_ARG;
  if (K == 0) return MAPE_OK;
  if (ldg > kCoefMaxRow) return MAPE_ERR_SHAPE;
  const int vec = (ldg % 16 == 0 && (reinterpret_cast<uintptr_t>(G) & 15) == 0) ? 1 : 0;
  const size_t smem = (size_t)kCoefWarps * kCoefRows * ldg;
  if (smem > 48 * 1024) {
    size_t lim = 0;
    const int rc = allow_max_dynamic_smem((const void*)coeffs_kernel, &lim);
    if (rc != MAPE_OK) return rc;
    if (smem > lim) return MAPE_ERR_SHAPE;
  }
  mape_detail::launch(coeffs_kernel, (unsigned)ceil_div(K, (int64_t)kCoefWarps * kCoefRows), 32 * kCoefWarps, smem,
                      as_stream(stream), q_row, q_col, q_val, nnz, w, n, G, K, ldg, vec, a, q4);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}

extern "C" size_t mape_direction_coeffs_batch_workspace_bytes(int32_t count) {
  if (count <= 0) return 0;
  mape_detail::Sizer s;
  s.take<mape_coeffs_item>((size_t)count);
  s.take<int64_t>((size_t)count + 1);
  s.take<int32_t>((size_t)count);
  return s.bytes();
}

extern "C" int mape_direction_coeffs_batch(const mape_coeffs_item* items, int32_t count, void* workspace,
                                           size_t workspace_bytes, void* stream) {
  using namespace mape_detail;
  if (!items || count <= 0) return MAPE_ERR_INVALID_ARG;
  std::vector<int64_t> prefix((size_t)count + 1, 0);
  std::vector<int32_t> vec((size_t)count, 0);
  int max_ldg = 16;
  for (int i = 0; i < count; ++i) {
    const mape_coeffs_item& it = items[i];
    if (it.nnz < 0 || it.n <= 0 || it.ldg < it.n || it.K < 0 || (it.nnz > 0 && (!it.q_row || !it.q_col || !it.q_val)) ||
        (it.K > 0 && (!it.G || !it.a || !it.q4)))
      return MAPE_ERR_INVALID_ARG;
    if (it.K > 0 && it.ldg > kCoefMaxRow) return MAPE_ERR_SHAPE;
    prefix[(size_t)i + 1] = prefix[(size_t)i] + (it.K + kCoefRows - 1) / kCoefRows;  // groups of directions
    vec[(size_t)i] = (it.ldg % 16 == 0 && (reinterpret_cast<uintptr_t>(it.G) & 15) == 0) ? 1 : 0;
    if (it.K > 0) max_ldg = std::max(max_ldg, (int)it.ldg);
  }
  const int64_t total = prefix[(size_t)count];
  if (total == 0) return MAPE_OK;
  Carver bc(workspace, workspace_bytes);
  mape_coeffs_item* d_items = bc.take<mape_coeffs_item>((size_t)count);
  int64_t* d_prefix = bc.take<int64_t>((size_t)count + 1);
  int32_t* d_vec = bc.take<int32_t>((size_t)count);
  if (!bc.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_items, items, sizeof(mape_coeffs_item) * count, cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_prefix, prefix.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_vec, vec.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, st));
  const size_t smem = (size_t)kCoefWarps * kCoefRows * max_ldg;
  if (smem > 48 * 1024) {
    size_t lim = 0;
    const int rc = allow_max_dynamic_smem((const void*)coeffs_batch_kernel, &lim);
    if (rc != MAPE_OK) return rc;
    if (smem > lim) return MAPE_ERR_SHAPE;
  }
  launch(coeffs_batch_kernel, (unsigned)ceil_div(total, kCoefWarps), 32 * kCoefWarps, smem, st,
         (const mape_coeffs_item*)d_items, (const int64_t*)d_prefix, (const int32_t*)d_vec, (int)count, max_ldg);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}

extern "C" size_t mape_augment_workspace_bytes(int32_t n, int32_t S, int64_t K) {
  using namespace mape_detail;
  if (n <= 0 || S < 0 || K < 0) return 0;
  Sizer s;
  s.take<long long>((size_t)S * n);          // R
  s.take<uint8_t>((size_t)S);                // active
  s.take<Best>((size_t)S * kMaxScoreBlocks); // partial minima
  s.take<int32_t>((size_t)S);                // per-start iteration counts
  s.take<unsigned int>(1);                   // active count
  s.take<int32_t>(1);                        // bad-start flag
  s.take<int32_t>((size_t)S);                // move counts when the caller gives none
  return s.bytes();
}

extern "C" int mape_augment_run(const mape_augment_args* A, int64_t* iters_out, void* stream) {
  using namespace mape_detail;
  if (!A || !iters_out) return MAPE_ERR_INVALID_ARG;
  int rc = check_args(A);
  if (rc != MAPE_OK) return rc;
  const int n = A->n, S = A->S;
  const int64_t K = A->K;
  *iters_out = 0;
  if (S == 0) return MAPE_OK;
  const AugCarve w = carve(A);
  if (!w.ok) return MAPE_ERR_CAPACITY;
  int32_t* nmoves = A->nmoves ? A->nmoves : w.own_nmoves;
  cudaStream_t st = as_stream(stream);
  const bool vec = rows_vectorisable(A);
  AugView v = make_view(A, w.R, w.active, w.partial, w.iters, w.n_active, w.bad, nmoves, 1);
  MAPE_CUDA_TRY(cudaMemsetAsync(w.iters, 0, sizeof(int32_t) * S, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(nmoves, 0, sizeof(int32_t) * S, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(w.bad, 0, sizeof(int32_t), st));
  unsigned int h_active = (unsigned)S;
  MAPE_CUDA_TRY(cudaMemcpyAsync(w.n_active, &h_active, sizeof(unsigned int), cudaMemcpyHostToDevice, st));
  launch(init_kernel, S, 256, 0, st, v);
  MAPE_LAUNCH_CHECK();
  int32_t h_bad = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&h_bad, w.bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_bad) return MAPE_ERR_BOUNDS;
  if (K == 0) {
    *iters_out = 1;
    return MAPE_OK;
  }
  const size_t smem = score_smem(n);
  if ((rc = allow_score_smem(smem, false)) != MAPE_OK) return rc;
  int lanes = 1;
  if ((rc = pick_lanes(A, v, vec, smem, st, &lanes)) != MAPE_OK) return rc;
  v.nb = score_blocks(K, lanes);
  const ScoreFn score = score_fn(lanes, vec);
  int64_t done_iters = 0;
  const int64_t chunk = 8;
  while (done_iters < A->max_iters) {
    int64_t c = std::min<int64_t>(chunk, A->max_iters - done_iters);
    for (int64_t q = 0; q < c; ++q) {
      launch(score, dim3((unsigned)v.nb, (unsigned)S), kScoreThreads, smem, st, v);
      launch(apply_kernel, S, 256, 0, st, v);
    }
    MAPE_LAUNCH_CHECK();
    done_iters += c;
    MAPE_CUDA_TRY(cudaMemcpyAsync(&h_active, w.n_active, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    MAPE_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_active == 0) break;
  }
  std::vector<int32_t> it(S);
  MAPE_CUDA_TRY(cudaMemcpyAsync(it.data(), w.iters, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  *iters_out = *std::max_element(it.begin(), it.end());
  return MAPE_OK;
}

namespace {
constexpr int kBatchChunk = 8;  // iterations per captured graph
}

extern "C" size_t mape_augment_run_batch_workspace_bytes(int32_t count) {
  using namespace mape_detail;
  if (count <= 0) return 0;
  Sizer s;
  s.take<AugView>((size_t)count);       // the instances' views
  s.take<int64_t>((size_t)count + 1);   // start prefix
  s.take<int64_t>((size_t)count + 1);   // score-block prefix
  s.take<unsigned int>((size_t)count);  // active counts
  s.take<int32_t>((size_t)count);       // bad-start flags
  s.take<int64_t>((size_t)count);       // iterations run per instance
  s.take<int64_t>(1);                   // iteration counter
  return s.bytes();
}

extern "C" int mape_augment_run_batch(const mape_augment_args* items, int32_t count, int64_t* iters_out,
                                      void* workspace, size_t workspace_bytes, void* stream,
                                      mape_augment_done_fn done, void* done_ctx) {
  using namespace mape_detail;
  if (!items || count <= 0 || !iters_out) return MAPE_ERR_INVALID_ARG;
  int rc = MAPE_OK;
  for (int i = 0; i < count; ++i)
    if ((rc = check_args(&items[i])) != MAPE_OK) return rc;
  Carver bc(workspace, workspace_bytes);
  AugView* d_views = bc.take<AugView>((size_t)count);
  int64_t* d_st_prefix = bc.take<int64_t>((size_t)count + 1);
  int64_t* d_blk_prefix = bc.take<int64_t>((size_t)count + 1);
  unsigned int* d_active = bc.take<unsigned int>((size_t)count);
  int32_t* d_bad = bc.take<int32_t>((size_t)count);
  int64_t* d_iters = bc.take<int64_t>((size_t)count);
  int64_t* d_iter = bc.take<int64_t>(1);
  if (!bc.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  for (int i = 0; i < count; ++i) iters_out[i] = 0;

  // the lane count: the caller's when every instance gives the same one,
  // else the autotuned one of the instance with the most row entries
  bool vec = true;
  int lanes = items[0].score_lanes, big = 0;
  size_t smem = 0;
  for (int i = 0; i < count; ++i) {
    const mape_augment_args* A = &items[i];
    if (A->S == 0) continue;
    if (A->K > 0 && !rows_vectorisable(A)) vec = false;
    if (A->score_lanes != lanes) lanes = 0;
    if (A->K * A->n > items[big].K * items[big].n) big = i;
    smem = std::max(smem, score_smem(A->n));
  }
  std::vector<AugView> views((size_t)count);
  std::vector<AugCarve> carves((size_t)count);
  std::vector<int64_t> st_prefix((size_t)count + 1, 0), blk_prefix((size_t)count + 1, 0);
  for (int i = 0; i < count; ++i) {
    const mape_augment_args* A = &items[i];
    carves[i] = carve(A);
    if (A->S > 0 && !carves[i].ok) return MAPE_ERR_CAPACITY;
  }
  // instances with starts: their state is set up (the timed probes of the
  // autotuner read the biggest one's)
  for (int i = 0; i < count; ++i) {
    const mape_augment_args* A = &items[i];
    const AugCarve& w = carves[i];
    int32_t* nmoves = A->nmoves ? A->nmoves : w.own_nmoves;
    views[i] = make_view(A, w.R, w.active, w.partial, w.iters, d_active + i, d_bad + i, nmoves, 1);
    if (A->S == 0) continue;
    MAPE_CUDA_TRY(cudaMemsetAsync(w.iters, 0, sizeof(int32_t) * A->S, st));
    MAPE_CUDA_TRY(cudaMemsetAsync(nmoves, 0, sizeof(int32_t) * A->S, st));
  }
  for (int i = 0; i < count; ++i) st_prefix[i + 1] = st_prefix[i] + items[i].S;
  const int64_t total_starts = st_prefix[count];
  if (total_starts == 0) {
    if (done)
      for (int i = 0; i < count; ++i) done(i, 0, done_ctx);
    return MAPE_OK;
  }
  std::vector<unsigned int> h_active((size_t)count);
  for (int i = 0; i < count; ++i) h_active[i] = (unsigned)items[i].S;
  MAPE_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int32_t) * count, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_active, h_active.data(), sizeof(unsigned int) * count, cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_views, views.data(), sizeof(AugView) * count, cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_st_prefix, st_prefix.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice,
                                st));
  launch(init_batch_kernel, (unsigned)total_starts, 256, 0, st, d_views, d_st_prefix, count);
  MAPE_LAUNCH_CHECK();
  std::vector<int32_t> h_bad((size_t)count, 0);
  MAPE_CUDA_TRY(cudaMemcpyAsync(h_bad.data(), d_bad, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i)
    if (h_bad[i]) return MAPE_ERR_BOUNDS;
  int64_t max_iters = 0;
  for (int i = 0; i < count; ++i) {
    if (items[i].S == 0) continue;
    if (items[i].K == 0) iters_out[i] = 1;  // as mape_augment_run: the initial pass only
    else max_iters = std::max(max_iters, items[i].max_iters);
  }
  if (max_iters == 0) {  // no instance has an iteration to run
    if (done)
      for (int i = 0; i < count; ++i) done(i, iters_out[i], done_ctx);
    return MAPE_OK;
  }
  if ((rc = allow_score_smem(smem, true)) != MAPE_OK) return rc;
  if (!vec) {
    lanes = 1;
  } else if (lanes == 0) {
    AugView vb = views[big];
    if ((rc = pick_lanes(&items[big], vb, true, smem, st, &lanes)) != MAPE_OK) return rc;
  }
  for (int i = 0; i < count; ++i) {
    views[i].nb = score_blocks(items[i].K, lanes);
    const int64_t blocks = (items[i].S > 0 && items[i].K > 0) ? (int64_t)views[i].nb * items[i].S : 0;
    blk_prefix[i + 1] = blk_prefix[i] + blocks;
  }
  const int64_t total_blocks = blk_prefix[count];
  if (total_blocks > INT32_MAX) return MAPE_ERR_SHAPE;
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_views, views.data(), sizeof(AugView) * count, cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(d_blk_prefix, blk_prefix.data(), sizeof(int64_t) * (count + 1),
                                cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(d_iter, 0, sizeof(int64_t), st));
  const ScoreBatchFn score = score_batch_fn(lanes, vec);
  auto enqueue_chunk = [&]() -> int {
    for (int q = 0; q < kBatchChunk; ++q) {
      launch(score, (unsigned)total_blocks, kScoreThreads, smem, st, (const AugView*)d_views,
             (const int64_t*)d_blk_prefix, (int)count, (const int64_t*)d_iter);
      launch(apply_batch_kernel, (unsigned)total_starts, 256, 0, st, (const AugView*)d_views,
             (const int64_t*)d_st_prefix, (int)count, (const int64_t*)d_iter);
      launch(tick_kernel, 1, 1, 0, st, d_iter);
    }
    MAPE_LAUNCH_CHECK();
    return MAPE_OK;
  };
  // a chunk of iterations as one CUDA graph, captured once and replayed (the
  // legacy default stream cannot be captured: there the chunk is launched
  // directly)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto destroy_graph = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  };
  if (st != nullptr) {
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      record_cuda_error(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
      return MAPE_ERR_CUDA;
    }
    rc = enqueue_chunk();
    e = cudaStreamEndCapture(st, &graph);
    if (rc == MAPE_OK && e != cudaSuccess) {
      record_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
      rc = MAPE_ERR_CUDA;
    }
    if (rc == MAPE_OK && (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
      record_cuda_error(e, "cudaGraphInstantiate", __FILE__, __LINE__);
      rc = MAPE_ERR_CUDA;
    }
    if (rc != MAPE_OK) {
      destroy_graph();
      return rc;
    }
  }
  // items that have finished are reported (done) as soon as a chunk shows it:
  // every start stopped, or its own iteration limit reached, or nothing to run
  std::vector<char> told((size_t)count, 0);
  std::vector<int64_t> it_now((size_t)count, 0);
  auto running = [&](int i, int64_t iters_done) {
    return items[i].S > 0 && items[i].K > 0 && h_active[(size_t)i] > 0 && iters_done < items[i].max_iters;
  };
  auto tell = [&](int64_t iters_done, bool all) -> int {
    bool fresh = false;
    for (int i = 0; i < count; ++i) fresh |= !told[(size_t)i] && (all || !running(i, iters_done));
    if (!fresh || !done) return MAPE_OK;
    launch(iters_max_kernel, (unsigned)count, 256, 0, st, (const AugView*)d_views, (int)count, d_iters);
    MAPE_LAUNCH_CHECK();
    MAPE_CUDA_TRY(cudaMemcpyAsync(it_now.data(), d_iters, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, st));
    MAPE_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < count; ++i) {
      if (told[(size_t)i] || !(all || !running(i, iters_done))) continue;
      told[(size_t)i] = 1;
      const int64_t its = items[i].S == 0 ? 0 : (items[i].K == 0 ? 1 : it_now[(size_t)i]);
      done(i, its, done_ctx);
    }
    return MAPE_OK;
  };
  if ((rc = tell(0, false)) != MAPE_OK) {
    destroy_graph();
    return rc;
  }
  int64_t done_iters = 0;
  while (done_iters < max_iters) {
    if (exec) {
      const cudaError_t e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) {
        record_cuda_error(e, "cudaGraphLaunch", __FILE__, __LINE__);
        destroy_graph();
        return MAPE_ERR_CUDA;
      }
    } else if ((rc = enqueue_chunk()) != MAPE_OK) {
      return rc;
    }
    done_iters += kBatchChunk;
    if (cudaMemcpyAsync(h_active.data(), d_active, sizeof(unsigned int) * count, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      record_cuda_error(cudaGetLastError(), "augment batch", __FILE__, __LINE__);
      destroy_graph();
      return MAPE_ERR_CUDA;
    }
    // an instance still running needs starts left and iterations left
    bool any = false;
    for (int i = 0; i < count; ++i) any |= running(i, done_iters);
    if (!any) break;
    if ((rc = tell(done_iters, false)) != MAPE_OK) {
      destroy_graph();
      return rc;
    }
  }
  destroy_graph();
  launch(iters_max_kernel, (unsigned)count, 256, 0, st, (const AugView*)d_views, (int)count, d_iters);
  MAPE_LAUNCH_CHECK();
  std::vector<int64_t> it((size_t)count);
  MAPE_CUDA_TRY(cudaMemcpyAsync(it.data(), d_iters, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i)
    if (items[i].S > 0 && items[i].K > 0) iters_out[i] = it[i];
  if (done)
    for (int i = 0; i < count; ++i)
      if (!told[(size_t)i]) done(i, iters_out[i], done_ctx);
  return MAPE_OK;
}
