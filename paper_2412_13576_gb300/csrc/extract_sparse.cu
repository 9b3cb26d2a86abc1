// Algorithm 2 (§3.2) for an identity-topped basis B = [I_d ; B'] whose B' is
// sparse (A = [C | I] with C at a few percent density): the sparse path.
//
// One block per start, persistent over the T steps, with the start's FP32
// z, m, v in shared memory for the whole call: every step costs on-chip work
// only.  B' is read from compressed sparse rows (for B' z and B' round(z)) and
// compressed sparse columns (for B'^T sign(B' z)), both small enough to stay in
// L1/L2.  Per step:
//   y = B' z (one thread per row of B'), S = sign(y); on collection steps
//   also g' = B' round(z) exactly in int32, its bound test (C4);
//   the previous rounding's candidate is appended (canonical sign from the
//   identity rows, whose entries are round(z) itself);
//   per coordinate j: grad = sign(z_j) + (B'^T S)_j + lambda1 (ceil z + floor z
//   - 2 z) + inverse-norm term, Adam, and the trackers of the next
//   collection (rounding changed / beyond 256, identity rows out of the box,
//   first nonzero entry) and of ||z||_inf with its first index (block-wide
//   atomics on shared words).
// FP32 CUDA-core arithmetic, the same per-coordinate update as the other
// paths; the products are sums over the nonzeros of a row or column in
// storage order.
#include "common.cuh"
#include "extract_internal.cuh"

#include <cmath>
#include <vector>

namespace {

constexpr int kThreads = 256;
constexpr int kNoNz = 0x7fffffff;
constexpr uint32_t kChanged = 1, kUnexact = 2, kOutId = 4, kOutB = 8;

struct SpParams {
  int n, d, mr, P, t0, T, period;
  const int32_t* rp;   // CSR of B': row pointers [mr + 1]
  const int32_t* ci;   // column indices
  const float* rv;     // values
  const int32_t* cp;   // CSC of B': column pointers [d + 1]
  const int32_t* ri;   // row indices
  const float* cv;     // values
  const int32_t* span;
  float* Z;
  float* M;
  float* V;
  const float2* bias;  // (lr / (1 - beta1^t), 1 / sqrt(1 - beta2^t)) per step
  float lambda1, lambda2, eps, beta1, beta2, omb1, omb2;
  int8_t* cand;
  int ldc;
  int64_t cap;
  unsigned long long* count;
  int32_t* flags;
  float* dbg_phi;
  float* dbg_grad;
};

__device__ __forceinline__ unsigned long long zkey(float a, int j) {
  return ((unsigned long long)__float_as_uint(a) << 32) | (0xffffffffu - (uint32_t)j);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__global__ void __launch_bounds__(kThreads) sparse_extract_kernel(SpParams p) {
  extern __shared__ __align__(16) float sm[];
  const int d = p.d, mr = p.mr;
  float* z = sm;
  float* mm = z + d;
  float* vv = mm + d;
  float* sg = vv + d;                                        // sign(B' z), mr entries
  int32_t* gb = reinterpret_cast<int32_t*>(sg + mr);         // B' round(z), mr entries
  __shared__ unsigned long long s_key, s_key_next;
  __shared__ uint32_t s_fl;       // changed | unexact since the last collection; out-of-box bits of the current rounding
  __shared__ int32_t s_first, s_first_next;
  __shared__ long long s_slot;
  __shared__ float s_red[kThreads / 32];
  const int tid = threadIdx.x;
  const int64_t pg = blockIdx.x;
  float* Zg = p.Z + pg * d;
  float* Mg = p.M + pg * d;
  float* Vg = p.V + pg * d;
  if (tid == 0) {
    s_key = 0ull;
    s_key_next = 0ull;
    s_fl = kChanged;  // the first collection of a call always counts
    s_first = kNoNz;
    s_first_next = kNoNz;
  }
  __syncthreads();
  unsigned long long kloc = 0ull;
  for (int j = tid; j < d; j += kThreads) {
    z[j] = Zg[j];
    mm[j] = Mg[j];
    vv[j] = Vg[j];
    const unsigned long long k = zkey(fabsf(z[j]), j);
    kloc = k > kloc ? k : kloc;
  }
  kloc = warp_max_u64(kloc);
  if ((tid & 31) == 0 && kloc) atomicMax(&s_key, kloc);
  __syncthreads();

  // appends the candidate of the current z if due (all threads)
  auto collect = [&]() {
    // g' = B' round(z) and its bound test
    bool out = false;
    for (int i = tid; i < mr; i += kThreads) {
      int acc = 0;
      for (int k = p.rp[i]; k < p.rp[i + 1]; ++k) acc += (int)p.rv[k] * (int)rintf(z[p.ci[k]]);
      gb[i] = acc;
      const int sp = p.span[d + i];
      if (acc > sp || -acc > sp) out = true;
    }
    if (__any_sync(0xffffffffu, out) && (tid & 31) == 0) atomicOr(&s_fl, kOutB);
    __syncthreads();
    if (tid == 0) {
      long long slot = -1;
      const uint32_t f = s_fl;
      if ((f & kChanged) && !(f & (kOutB | kOutId)) && s_first != kNoNz) {
        if (f & kUnexact) {
          atomicOr(p.flags, 2);
        } else {
          const unsigned long long at = atomicAdd(p.count, 1ull);
          if ((int64_t)at < p.cap) slot = (long long)at;
          else atomicOr(p.flags, 1);
        }
      }
      s_slot = slot;
      s_fl = f & ~(kChanged | kUnexact | kOutB);
    }
    __syncthreads();
    const long long slot = s_slot;
    if (slot >= 0) {
      const int sgn = (s_first & 1) ? -1 : 1;
      int8_t* row = p.cand + slot * p.ldc;
      for (int j = tid; j < p.ldc; j += kThreads) {
        int v = 0;
        if (j < d) v = (int)rintf(z[j]);
        else if (j < p.n) v = gb[j - d];
        row[j] = (int8_t)(sgn * v);
      }
    }
  };

  for (int s = 0; s < p.T; ++s) {
    const int t = p.t0 + s + 1;
    const bool collect_prev = s >= 1 && ((t - 1) % p.period == 0);
    const bool dbg = s == 0 && (p.dbg_phi || p.dbg_grad);
    float l1 = 0.f;
    for (int i = tid; i < mr; i += kThreads) {
      float acc = 0.f;
      for (int k = p.rp[i]; k < p.rp[i + 1]; ++k) acc = fmaf(p.rv[k], z[p.ci[k]], acc);
      sg[i] = (float)mape_sign_f(acc);
      if (dbg) l1 += fabsf(acc);
    }
    if (collect_prev) collect();  // its barriers also order sg for the gradient
    __syncthreads();
    const unsigned long long key = s_key;
    const float zinf = __uint_as_float((uint32_t)(key >> 32));
    const int kmax = key ? (int)(0xffffffffu - (uint32_t)key) : -1;
    float inv_term = 0.f;
    if (zinf < 1.f && zinf > 0.f) inv_term = -p.lambda2 / (zinf * zinf);
    const float2 ad = p.bias[s];
    unsigned long long knew = 0ull;
    uint32_t fb = 0u;
    int first_id = kNoNz;
    float frac = 0.f;
    for (int j = tid; j < d; j += kThreads) {
      const float x = z[j];
      float g = 0.f;
      for (int k = p.cp[j]; k < p.cp[j + 1]; ++k) g = fmaf(p.cv[k], sg[p.ri[k]], g);
      const float fl = floorf(x);
      const float sx = (float)mape_sign_f(x);
      float grad = g + p.lambda1 * (2.f * fl + (x != fl ? 1.f : 0.f) - 2.f * x);
      if (j == kmax) grad += inv_term * sx;
      grad += sx;  // identity row j: sign((Bz)_j) = sign(z_j)
      if (dbg) {
        frac += (x - fl) * (ceilf(x) - x);
        l1 += fabsf(x);
        if (p.dbg_grad) p.dbg_grad[pg * d + j] = grad;
      }
      const float m1 = p.beta1 * mm[j] + p.omb1 * grad;
      const float v1 = p.beta2 * vv[j] + p.omb2 * grad * grad;
      const float den = (v1 > 0.f ? v1 * rsqrtf(v1) : 0.f) * ad.y + p.eps;
      const float xn = x - ad.x * __fdividef(m1, den);
      z[j] = xn;
      mm[j] = m1;
      vv[j] = v1;
      const float rn = rintf(xn);
      if (rn != rintf(x)) fb |= kChanged;
      if (fabsf(rn) > 256.f) fb |= kUnexact;
      if (fabsf(rn) > (float)p.span[j]) fb |= kOutId;
      if (first_id == kNoNz && rn != 0.f) first_id = (j << 1) | (rn < 0.f ? 1 : 0);
      const unsigned long long k = zkey(fabsf(xn), j);
      knew = k > knew ? k : knew;
    }
    if (dbg && p.dbg_phi) {
      float v = l1 + p.lambda1 * frac;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0) s_red[tid >> 5] = v;
    }
    // reductions of the new state: out-of-box of the identity rows is a
    // property of the current rounding (replaced), the others accumulate
    if (tid == 0) {
      s_fl &= ~kOutId;
      s_key_next = 0ull;
      s_first_next = kNoNz;
    }
    __syncthreads();
    // one shared atomic per warp and word
    fb = __reduce_or_sync(0xffffffffu, fb);
    knew = warp_max_u64(knew);
    first_id = __reduce_min_sync(0xffffffffu, first_id);
    if ((tid & 31) == 0) {
      if (fb) atomicOr(&s_fl, fb);
      if (knew) atomicMax(&s_key_next, knew);
      if (first_id != kNoNz) atomicMin(&s_first_next, first_id);
    }
    __syncthreads();
    if (tid == 0) {
      if (dbg && p.dbg_phi) {
        float tot = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) tot += s_red[w];
        const float inv = zinf > 0.f ? fmaxf(1.f / zinf - 1.f, 0.f) : INFINITY;
        p.dbg_phi[pg] = tot + p.lambda2 * inv;
      }
      s_key = s_key_next;
      s_first = s_first_next;
    }
    __syncthreads();
  }
  if (p.T > 0 && (p.t0 + p.T) % p.period == 0) collect();  // the candidate of the last step
  __syncthreads();
  for (int j = tid; j < d; j += kThreads) {
    Zg[j] = z[j];
    Mg[j] = mm[j];
    Vg[j] = vv[j];
  }
}

// identity-top test, CSR counts of B' (rows d .. n-1) and CSC counts
__global__ void sparse_scan_kernel(const int32_t* __restrict__ B, int n, int d, int32_t* __restrict__ notid,
                                   int32_t* __restrict__ rcount, int32_t* __restrict__ ccount,
                                   int32_t* __restrict__ bad) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * d) return;
  const int i = (int)(e / d), j = (int)(e % d);
  const int v = B[e];
  if (i < d) {
    if (v != (i == j ? 1 : 0)) atomicOr(notid, 1);
    return;
  }
  if (v == 0) return;
  if (v > (1 << 23) || v < -(1 << 23)) atomicOr(bad, 1);  // exact in FP32
  atomicAdd(&rcount[i - d], 1);
  atomicAdd(&ccount[j], 1);
}

// fills CSR (one thread per row, column order) and CSC (one thread per column, row order)
__global__ void sparse_fill_rows_kernel(const int32_t* __restrict__ B, int n, int d, const int32_t* __restrict__ rp,
                                        int32_t* __restrict__ ci, float* __restrict__ rv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - d) return;
  int k = rp[i];
  for (int j = 0; j < d; ++j) {
    const int v = B[(int64_t)(d + i) * d + j];
    if (v != 0) {
      ci[k] = j;
      rv[k] = (float)v;
      ++k;
    }
  }
}

__global__ void sparse_fill_cols_kernel(const int32_t* __restrict__ B, int n, int d, const int32_t* __restrict__ cp,
                                        int32_t* __restrict__ ri, float* __restrict__ cv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  int k = cp[j];
  for (int i = 0; i < n - d; ++i) {
    const int v = B[(int64_t)(d + i) * d + j];
    if (v != 0) {
      ri[k] = i;
      cv[k] = (float)v;
      ++k;
    }
  }
}

size_t sparse_smem(int d, int mr) { return (size_t)3 * d * sizeof(float) + (size_t)mr * (sizeof(float) + sizeof(int32_t)); }

}  // namespace

namespace mape_detail {

constexpr size_t kSparseSmemLimit = 220 * 1024;

bool extract_sparse_supported(int32_t n, int32_t d) {
  return n > d && sparse_smem(d, n - d) <= kSparseSmemLimit;
}

size_t extract_sparse_workspace(int32_t n, int32_t d, int32_t P) {
  (void)P;
  if (!extract_sparse_supported(n, d)) return 0;
  const size_t mr = (size_t)(n - d), nnz = mr * d;  // bound: dense B'
  Sizer s;
  s.take<int32_t>(mr + 1);
  s.take<int32_t>(nnz);
  s.take<float>(nnz);
  s.take<int32_t>((size_t)d + 1);
  s.take<int32_t>(nnz);
  s.take<float>(nnz);
  s.take<int32_t>(4);  // identity flag, inexact flag, spare
  s.take<float2>((size_t)1 << 20);
  return s.bytes();
}

int extract_sparse(const mape_extract_args* a, cudaStream_t st) {
  const int n = a->n, d = a->d, P = a->P, mr = n - d;
  if (a->T > (1 << 20) || !extract_sparse_supported(n, d)) return MAPE_ERR_SHAPE;
  const size_t nnz_max = (size_t)mr * d;
  Carver cv(a->workspace, a->workspace_bytes);
  int32_t* rp = cv.take<int32_t>((size_t)mr + 1);
  int32_t* ci = cv.take<int32_t>(nnz_max);
  float* rv = cv.take<float>(nnz_max);
  int32_t* cp = cv.take<int32_t>((size_t)d + 1);
  int32_t* ri = cv.take<int32_t>(nnz_max);
  float* cvv = cv.take<float>(nnz_max);
  int32_t* fl = cv.take<int32_t>(4);
  float2* bias = cv.take<float2>((size_t)1 << 20);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  // counts into the pointer arrays (shifted by one), then prefix sums on the host
  MAPE_CUDA_TRY(cudaMemsetAsync(rp, 0, sizeof(int32_t) * (mr + 1), st));
  MAPE_CUDA_TRY(cudaMemsetAsync(cp, 0, sizeof(int32_t) * (d + 1), st));
  MAPE_CUDA_TRY(cudaMemsetAsync(fl, 0, sizeof(int32_t) * 4, st));
  launch(sparse_scan_kernel, (unsigned)ceil_div((int64_t)n * d, 256), 256, 0, st, a->B, n, d, fl, rp + 1, cp + 1,
         fl + 1);
  MAPE_LAUNCH_CHECK();
  std::vector<int32_t> hr((size_t)mr + 1), hc((size_t)d + 1), hf(4);
  MAPE_CUDA_TRY(cudaMemcpyAsync(hr.data(), rp, sizeof(int32_t) * (mr + 1), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(hc.data(), cp, sizeof(int32_t) * (d + 1), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(hf.data(), fl, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  if (hf[0]) return MAPE_ERR_SHAPE;  // the sparse path takes identity-topped bases only
  if (hf[1]) return MAPE_ERR_NUMERIC;
  for (int i = 0; i < mr; ++i) hr[i + 1] += hr[i];
  for (int j = 0; j < d; ++j) hc[j + 1] += hc[j];
  MAPE_CUDA_TRY(cudaMemcpyAsync(rp, hr.data(), sizeof(int32_t) * (mr + 1), cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(cp, hc.data(), sizeof(int32_t) * (d + 1), cudaMemcpyHostToDevice, st));
  launch(sparse_fill_rows_kernel, (unsigned)ceil_div(mr, 128), 128, 0, st, a->B, n, d, rp, ci, rv);
  launch(sparse_fill_cols_kernel, (unsigned)ceil_div(d, 128), 128, 0, st, a->B, n, d, cp, ri, cvv);
  std::vector<float2> bc((size_t)a->T);
  for (int s = 0; s < a->T; ++s) {
    const double t = (double)a->t0 + s + 1;
    const double bc1 = 1.0 - std::pow(a->beta1, t), bc2 = 1.0 - std::pow(a->beta2, t);
    bc[s] = make_float2((float)((double)a->lr / bc1), (float)(1.0 / std::sqrt(bc2)));
  }
  MAPE_CUDA_TRY(cudaMemcpyAsync(bias, bc.data(), sizeof(float2) * bc.size(), cudaMemcpyHostToDevice, st));
  SpParams p{};
  p.n = n; p.d = d; p.mr = mr; p.P = P; p.t0 = a->t0; p.T = a->T; p.period = a->period;
  p.rp = rp; p.ci = ci; p.rv = rv; p.cp = cp; p.ri = ri; p.cv = cvv; p.span = a->span;
  p.Z = a->Z; p.M = a->M; p.V = a->V; p.bias = bias;
  p.lambda1 = a->lambda1; p.lambda2 = a->lambda2; p.eps = a->eps;
  p.beta1 = (float)a->beta1; p.beta2 = (float)a->beta2;
  p.omb1 = (float)(1.0 - a->beta1); p.omb2 = (float)(1.0 - a->beta2);
  p.cand = a->cand; p.ldc = a->ldc; p.cap = a->cand_cap; p.count = a->cand_count; p.flags = a->flags;
  p.dbg_phi = a->dbg_phi; p.dbg_grad = a->dbg_grad;
  const size_t smem = sparse_smem(d, mr);
  {
    size_t lim = 0;
    const int rc = allow_max_dynamic_smem((const void*)sparse_extract_kernel, &lim);
    if (rc != MAPE_OK) return rc;
    if ((size_t)smem > lim) return MAPE_ERR_SHAPE;
  }
  launch(sparse_extract_kernel, (unsigned)P, kThreads, smem, st, p);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}

}  // namespace mape_detail
