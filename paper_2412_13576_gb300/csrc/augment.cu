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
// not depend on the reduction order.
#include "common.cuh"

#include <algorithm>
#include <vector>

namespace {

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

// One warp per direction: the lanes take the entries of Q (coalesced) and of
// w, the direction's row is staged in shared memory, a warp reduction sums
// (integer arithmetic, exact in any order).
constexpr int kCoefWarps = 8;
constexpr int kCoefMaxRow = 4096;  // ldg <= 4096 bytes (n <= 4096)

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void coeffs_kernel(const int32_t* __restrict__ qr, const int32_t* __restrict__ qc,
                              const int32_t* __restrict__ qv, int nnz, const int32_t* __restrict__ w, int n,
                              const int8_t* __restrict__ G, int64_t K, int ldg, int64_t* __restrict__ a,
                              int64_t* __restrict__ q4) {
  __shared__ __align__(16) int8_t s_row[kCoefWarps][kCoefMaxRow];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * kCoefWarps + wid;
  if (k >= K) return;  // warp-uniform
  int8_t* g = s_row[wid];
  const uint4* src = reinterpret_cast<const uint4*>(G + k * ldg);
  for (int c = lane; c < ldg / 16; c += 32) reinterpret_cast<uint4*>(g)[c] = src[c];
  __syncwarp();
  long long acc = 0;
  for (int e = lane; e < nnz; e += 32) {
    const int i = qr[e], j = qc[e];
    const long long t = (long long)qv[e] * g[i] * g[j];
    acc += (i == j) ? t : 2 * t;
  }
  acc = warp_sum_ll(acc);
  long long s4 = 0;
  if (w)
    for (int i = lane; i < n; i += 32) {
      const long long gi = g[i];
      s4 += (long long)w[i] * gi * gi * gi * gi;
    }
  s4 = warp_sum_ll(s4);
  if (lane == 0) {
    a[k] = acc;
    q4[k] = s4;
  }
}

// r = 2 Q x + c and f(x), one block per start; checks l <= x <= u.
__global__ void init_kernel(const int32_t* __restrict__ qr, const int32_t* __restrict__ qc,
                            const int32_t* __restrict__ qv, int nnz, const int32_t* __restrict__ c,
                            const int32_t* __restrict__ w, const int32_t* __restrict__ l,
                            const int32_t* __restrict__ u, const int32_t* __restrict__ X, int n,
                            long long* __restrict__ R, int64_t* __restrict__ fval,
                            uint8_t* __restrict__ active, int32_t* __restrict__ bad) {
  int s = blockIdx.x;
  const int32_t* x = X + (int64_t)s * n;
  long long* r = R + (int64_t)s * n;
  __shared__ long long s_f[32];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    r[i] = c[i];
    if (x[i] < l[i] || x[i] > u[i]) atomicOr(bad, 1);
  }
  __syncthreads();
  long long f = 0;
  for (int e = threadIdx.x; e < nnz; e += blockDim.x) {
    int i = qr[e], j = qc[e];
    long long q = qv[e];
    atomicAdd((unsigned long long*)&r[i], (unsigned long long)(2 * q * x[j]));
    if (i != j) atomicAdd((unsigned long long*)&r[j], (unsigned long long)(2 * q * x[i]));
    f += (i == j ? 1 : 2) * q * x[i] * x[j];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    long long xi = x[i];
    f += (long long)c[i] * xi;
    if (w) f += (long long)w[i] * xi * xi * xi * xi;
  }
  for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
  if ((threadIdx.x & 31) == 0) s_f[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_f[i];
    fval[s] = t;
    active[s] = 1;
  }
}

__device__ __forceinline__ long long floor_div(long long a, long long b) {  // b > 0
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

// One thread per direction k, blockIdx.y = start.
__global__ void score_kernel(const int8_t* __restrict__ G, int64_t K, int ldg, int n,
                             const int64_t* __restrict__ a, const int64_t* __restrict__ q4,
                             const int32_t* __restrict__ w, const int32_t* __restrict__ l,
                             const int32_t* __restrict__ u, const int32_t* __restrict__ X,
                             const long long* __restrict__ R, const uint8_t* __restrict__ active,
                             Best* __restrict__ partial, int nblocks) {
  extern __shared__ long long smem[];
  int s = blockIdx.y;
  if (!active[s]) return;
  long long* s_r = smem;                  // n
  long long* s_w3 = s_r + n;              // n: w x^3 (quartic only)
  long long* s_w2 = s_w3 + n;             // n: w x^2
  long long* s_w1 = s_w2 + n;             // n: w x
  int32_t* s_up = reinterpret_cast<int32_t*>(s_w1 + n);  // n: u - x
  int32_t* s_dn = s_up + n;                              // n: x - l
  const int32_t* x = X + (int64_t)s * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    long long xi = x[i];
    s_r[i] = R[(int64_t)s * n + i];
    s_up[i] = u[i] - x[i];
    s_dn[i] = x[i] - l[i];
    if (w) {
      long long wi = w[i];
      s_w3[i] = wi * xi * xi * xi;
      s_w2[i] = wi * xi * xi;
      s_w1[i] = wi * xi;
    }
  }
  __syncthreads();
  Best best{kNoMove, kNoMove};
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < K) {
    const int8_t* g = G + k * ldg;
    long long b = 0, c1 = 0, c2 = 0, c3 = 0;
    int lam_p = 0x7fffffff, lam_m = 0x7fffffff;  // lambda_max for +g and -g
    for (int i = 0; i < n; ++i) {
      int gi = g[i];
      if (gi == 0) continue;
      b += (long long)gi * s_r[i];
      if (w) {
        long long g1 = gi;
        c1 += s_w3[i] * g1;
        c2 += s_w2[i] * g1 * g1;
        c3 += s_w1[i] * g1 * g1 * g1;
      }
      int ag = abs(gi);
      int up = s_up[i] / ag, dn = s_dn[i] / ag;  // both nonnegative
      if (gi > 0) { lam_p = min(lam_p, up); lam_m = min(lam_m, dn); }
      else        { lam_p = min(lam_p, dn); lam_m = min(lam_m, up); }
    }
    long long ak = a[k];
    long long c4 = q4[k];
    for (int e = 1; e >= -1; e -= 2) {
      int L = (e > 0) ? lam_p : lam_m;
      // L <= max(u - l) <= 127 for a nonzero row; a zero row has no move
      if (L < 1 || L > 255) continue;
      long long eb = e * b;
      if (!w) {
        long long cand[2];
        int nc;
        if (ak > 0) {
          // vertex at -eb / (2 a); the integer minimiser is floor or ceil of it
          long long fl = floor_div(-eb, 2 * ak);
          cand[0] = fl;
          cand[1] = fl + 1;
          nc = 2;
        } else {
          cand[0] = 1;
          cand[1] = L;
          nc = 2;
        }
        for (int q = 0; q < nc; ++q) {
          long long lam = cand[q] < 1 ? 1 : (cand[q] > L ? L : cand[q]);
          long long df = lam * lam * ak + lam * eb;
          Best cb{df, k * 512 + (e < 0 ? 256 : 0) + lam};
          if (better(cb, best)) best = cb;
        }
      } else {
        for (int lam = 1; lam <= L; ++lam) {
          long long lm = lam;
          long long df = lm * lm * ak + lm * eb + 4 * e * lm * c1 + 6 * lm * lm * c2 +
                         4 * e * lm * lm * lm * c3 + lm * lm * lm * lm * c4;
          Best cb{df, k * 512 + (e < 0 ? 256 : 0) + lm};
          if (better(cb, best)) best = cb;
        }
      }
    }
  }
  // block argmin
  __shared__ Best s_best[32];
  best = warp_min(best);
  if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    Best v = threadIdx.x < (blockDim.x >> 5) ? s_best[threadIdx.x] : Best{kNoMove, kNoMove};
    v = warp_min(v);
    if (threadIdx.x == 0) partial[(int64_t)s * nblocks + blockIdx.x] = v;
  }
}

// One block per start: final argmin; move or stop.
__global__ void apply_kernel(const int8_t* __restrict__ G, int ldg, int n, const int32_t* __restrict__ qr,
                             const int32_t* __restrict__ qc, const int32_t* __restrict__ qv, int nnz,
                             int32_t* __restrict__ X, long long* __restrict__ R, int64_t* __restrict__ fval,
                             uint8_t* __restrict__ active, const Best* __restrict__ partial, int nblocks,
                             int64_t* __restrict__ moves, int32_t* __restrict__ nmoves, int moves_cap,
                             int32_t* __restrict__ iters, unsigned int* __restrict__ n_active) {
  int s = blockIdx.x;
  if (!active[s]) return;
  __shared__ Best s_best[32];
  Best best{kNoMove, kNoMove};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    Best v = partial[(int64_t)s * nblocks + b];
    if (better(v, best)) best = v;
  }
  best = warp_min(best);
  if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    Best v = threadIdx.x < (blockDim.x >> 5) ? s_best[threadIdx.x] : Best{kNoMove, kNoMove};
    v = warp_min(v);
    if (threadIdx.x == 0) s_best[0] = v;
  }
  __syncthreads();
  best = s_best[0];
  if (threadIdx.x == 0) iters[s] += 1;
  if (best.df >= 0) {  // no improving move: this start is done
    if (threadIdx.x == 0) {
      active[s] = 0;
      atomicSub(n_active, 1u);
    }
    return;
  }
  long long k = best.key >> 9;
  int e = (best.key & 256) ? -1 : 1;
  long long lam = best.key & 255;
  long long step = e * lam;
  const int8_t* g = G + k * ldg;
  int32_t* x = X + (int64_t)s * n;
  long long* r = R + (int64_t)s * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] += (int32_t)(step * g[i]);
  for (int q = threadIdx.x; q < nnz; q += blockDim.x) {
    int i = qr[q], j = qc[q];
    long long v = qv[q];
    atomicAdd((unsigned long long*)&r[i], (unsigned long long)(2 * step * v * g[j]));
    if (i != j) atomicAdd((unsigned long long*)&r[j], (unsigned long long)(2 * step * v * g[i]));
  }
  if (threadIdx.x == 0) {
    long long fnew = fval[s] + best.df;
    fval[s] = fnew;
    int m = nmoves ? nmoves[s] : 0;
    if (moves && m < moves_cap) {
      int64_t* mv = moves + ((int64_t)s * moves_cap + m) * 4;
      mv[0] = k;
      mv[1] = e;
      mv[2] = lam;
      mv[3] = fnew;
    }
    if (nmoves) nmoves[s] = m + 1;
  }
}

}  // namespace

extern "C" int mape_direction_coeffs(const int32_t* q_row, const int32_t* q_col, const int32_t* q_val,
                                     int32_t nnz, const int32_t* w, int32_t n, const int8_t* G, int64_t K,
                                     int32_t ldg, int64_t* a, int64_t* q4, void* stream) {
  using namespace mape_detail;
  if (nnz < 0 || n <= 0 || ldg < n || K < 0 || (nnz > 0 && (!q_row || !q_col || !q_val)) ||
      (K > 0 && (!G || !a || !q4)))
    return MAPE_ERR_INVALID_ARG;
  if (K == 0) return MAPE_OK;
  if (ldg > kCoefMaxRow) return MAPE_ERR_SHAPE;
  mape_detail::launch(coeffs_kernel, (unsigned)ceil_div(K, kCoefWarps), 32 * kCoefWarps, 0, as_stream(stream), q_row,
                      q_col, q_val, nnz, w, n, G, K, ldg, a, q4);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}

namespace {
constexpr int kScoreThreads = 256;
}

extern "C" size_t mape_augment_workspace_bytes(int32_t n, int32_t S, int64_t K) {
  using namespace mape_detail;
  if (n <= 0 || S < 0 || K < 0) return 0;
  int64_t nb = std::max<int64_t>(1, ceil_div(K, kScoreThreads));
  Sizer s;
  s.take<long long>((size_t)S * n);   // R
  s.take<uint8_t>((size_t)S);         // active
  s.take<Best>((size_t)S * nb);       // partial bests
  s.take<int32_t>((size_t)S);         // per-start iteration counts
  s.take<unsigned int>(1);            // active count
  s.take<int32_t>(1);                 // bad-start flag
  s.take<int32_t>((size_t)S);         // move counts when the caller gives none
  return s.bytes();
}

extern "C" int mape_augment_run(const mape_augment_args* A, int64_t* iters_out, void* stream) {
  using namespace mape_detail;
  if (!A || !iters_out) return MAPE_ERR_INVALID_ARG;
  const int n = A->n, S = A->S;
  const int64_t K = A->K;
  if (n <= 0 || S < 0 || K < 0 || A->ldg < n || A->max_iters < 0) return MAPE_ERR_INVALID_ARG;
  if (S > 0 && (!A->X || !A->fval || !A->c || !A->l || !A->u)) return MAPE_ERR_INVALID_ARG;
  if (K > 0 && (!A->G || !A->a || !A->q4)) return MAPE_ERR_INVALID_ARG;
  if (A->nnz > 0 && (!A->q_row || !A->q_col || !A->q_val)) return MAPE_ERR_INVALID_ARG;
  if (A->moves && A->moves_cap <= 0) return MAPE_ERR_INVALID_ARG;
  if (K >= ((int64_t)1 << 40)) return MAPE_ERR_SHAPE;
  *iters_out = 0;
  if (S == 0) return MAPE_OK;
  int nb = (int)std::max<int64_t>(1, ceil_div(K, kScoreThreads));
  Carver cv(A->workspace, A->workspace_bytes);
  long long* R = cv.take<long long>((size_t)S * n);
  uint8_t* active = cv.take<uint8_t>((size_t)S);
  Best* partial = cv.take<Best>((size_t)S * nb);
  int32_t* iters = cv.take<int32_t>((size_t)S);
  unsigned int* n_active = cv.take<unsigned int>(1);
  int32_t* bad = cv.take<int32_t>(1);
  int32_t* own_nmoves = cv.take<int32_t>((size_t)S);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  int32_t* nmoves = A->nmoves ? A->nmoves : own_nmoves;
  cudaStream_t st = as_stream(stream);
  MAPE_CUDA_TRY(cudaMemsetAsync(iters, 0, sizeof(int32_t) * S, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(nmoves, 0, sizeof(int32_t) * S, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
  unsigned int h_active = (unsigned)S;
  MAPE_CUDA_TRY(cudaMemcpyAsync(n_active, &h_active, sizeof(unsigned int), cudaMemcpyHostToDevice, st));
  mape_detail::launch(init_kernel, S, 256, 0, st, A->q_row, A->q_col, A->q_val, A->nnz, A->c, A->w, A->l, A->u, A->X, n, R,
                                 A->fval, active, bad);
  MAPE_LAUNCH_CHECK();
  int32_t h_bad = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&h_bad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_bad) return MAPE_ERR_BOUNDS;
  if (K == 0) {
    *iters_out = 1;
    return MAPE_OK;
  }
  size_t smem = (size_t)n * (4 * sizeof(long long) + 2 * sizeof(int32_t));
  if (smem > 48 * 1024) {
    size_t lim = 0;
    const int rc = allow_max_dynamic_smem((const void*)score_kernel, &lim);
    if (rc != MAPE_OK) return rc;
    if (smem > lim) return MAPE_ERR_SHAPE;
  }
  int64_t done_iters = 0;
  const int64_t chunk = 8;
  while (done_iters < A->max_iters) {
    int64_t c = std::min<int64_t>(chunk, A->max_iters - done_iters);
    for (int64_t q = 0; q < c; ++q) {
      mape_detail::launch(score_kernel, dim3((unsigned)nb, (unsigned)S), kScoreThreads, smem, st, 
          A->G, K, A->ldg, n, A->a, A->q4, A->w, A->l, A->u, A->X, R, active, partial, nb);
      mape_detail::launch(apply_kernel, S, 256, 0, st, A->G, A->ldg, n, A->q_row, A->q_col, A->q_val, A->nnz, A->X, R, A->fval,
                                      active, partial, nb, A->moves, nmoves, A->moves_cap, iters, n_active);
    }
    MAPE_LAUNCH_CHECK();
    done_iters += c;
    MAPE_CUDA_TRY(cudaMemcpyAsync(&h_active, n_active, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    MAPE_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_active == 0) break;
  }
  std::vector<int32_t> it(S);
  MAPE_CUDA_TRY(cudaMemcpyAsync(it.data(), iters, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  *iters_out = *std::max_element(it.begin(), it.end());
  return MAPE_OK;
}
