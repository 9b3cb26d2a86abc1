// Algorithm 2 (§3.2) in FP32: the plain single-instance per-step path, the
// baseline the tensor-core paths are measured against.  It is what a direct
// PyTorch version of the method does on a GPU: per Adam step, the products
// are FP32 GEMMs from cuBLAS (strict FP32, no TF32) and everything else is a
// separate elementwise kernel:
//   Y = B Z (GEMM), S = sign(Y), G = B^T S (GEMM), ||z||_inf and its first
//   index per start, the gradient terms of Eq. (3) and the Adam update (marks
//   starts whose rounding changed); on collection steps R = round(Z),
//   B R (GEMM, exact: every |partial sum| stays below 2^24, else the start
//   is flagged), the bound test (C4), the first nonzero entry and the
//   append in canonical sign.
// State is coordinate-major ([d][P]): elementwise kernels read and write it
// coalesced, and it is the column-major P x d operand of the GEMMs.
#include "common.cuh"
#include "extract_internal.cuh"

#include <cublas_v2.h>

#include <cmath>
#include <map>
#include <mutex>
#include <vector>

namespace {

__global__ void to_float_kernel(const int32_t* __restrict__ B, float* __restrict__ Bf, int64_t count) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < count) Bf[i] = (float)B[i];
}

// [rows x cols] -> [cols x rows]
__global__ void transpose_kernel(const float* __restrict__ in, float* __restrict__ out, int rows, int cols) {
  __shared__ float tile[32][33];
  int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = in[(int64_t)r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(int64_t)c * rows + r] = tile[threadIdx.x][k];
  }
}

// S = sign(Y), elementwise over [n][P]
__global__ void sign_kernel(const float* __restrict__ Y, float* __restrict__ S, int64_t count) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < count) S[e] = (float)mape_sign_f(Y[e]);
}

// per start: ||z||_inf and its first index; with dbg, Phi at z (||Bz||_1 from Y)
__global__ void zinf_kernel(const float* __restrict__ Zt, const float* __restrict__ Y, int n, int d, int P,
                            float* __restrict__ zinf, int32_t* __restrict__ kmax, float lambda1, float lambda2,
                            float* __restrict__ dbg_phi) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float zi = 0.f, frac = 0.f;
  int k = 0;
  for (int j = 0; j < d; ++j) {
    const float zj = Zt[(int64_t)j * P + p];
    const float a = fabsf(zj);
    if (a > zi) { zi = a; k = j; }
    if (dbg_phi) frac += (zj - floorf(zj)) * (ceilf(zj) - zj);
  }
  zinf[p] = zi;
  kmax[p] = k;
  if (dbg_phi) {
    float l1 = 0.f;
    for (int i = 0; i < n; ++i) l1 += fabsf(Y[(int64_t)i * P + p]);
    const float inv = zi > 0.f ? fmaxf(1.f / zi - 1.f, 0.f) : INFINITY;
    dbg_phi[p] = l1 + lambda1 * frac + lambda2 * inv;
  }
}

struct StepParams {
  float lambda1, lambda2, lr, beta1, beta2, omb1, omb2, eps, bc1, bc2;
};

// the rest of the gradient and the Adam update, elementwise over [d][P]
__global__ void adam_kernel(const float* __restrict__ G, float* __restrict__ Zt, float* __restrict__ Mt,
                            float* __restrict__ Vt, const float* __restrict__ zinf, const int32_t* __restrict__ kmax,
                            uint8_t* __restrict__ changed, StepParams sp, int d, int P,
                            float* __restrict__ dbg_grad) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)d * P) return;
  const int j = (int)(e / P), p = (int)(e % P);
  const float z = Zt[e];
  float grad = G[e] + sp.lambda1 * (ceilf(z) + floorf(z) - 2.f * z);
  const float zi = zinf[p];
  if (j == kmax[p] && zi < 1.f && zi > 0.f) grad += -sp.lambda2 * (float)mape_sign_f(z) / (zi * zi);
  if (dbg_grad) dbg_grad[(int64_t)p * d + j] = grad;
  const float m = sp.beta1 * Mt[e] + sp.omb1 * grad;
  const float v = sp.beta2 * Vt[e] + sp.omb2 * grad * grad;
  const float mhat = m / sp.bc1;
  const float vhat = v / sp.bc2;
  const float zn = z - sp.lr * mhat / (sqrtf(vhat) + sp.eps);
  Mt[e] = m;
  Vt[e] = v;
  Zt[e] = zn;
  if (rintf(zn) != rintf(z)) changed[p] = 1;
}

// R = round(Z) for the exact map; a start with |round z| above rlim (so that
// B round(z) could leave the exact FP32 range) is flagged and mapped as 0
__global__ void round_kernel(const float* __restrict__ Zt, float* __restrict__ R, int d, int P, float rlim,
                             const uint8_t* __restrict__ changed, uint32_t* __restrict__ bad) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)d * P) return;
  const int p = (int)(e % P);
  float r = rintf(Zt[e]);
  if (fabsf(r) > rlim) {
    if (changed[p]) atomicOr(&bad[p], 4u);
    r = 0.f;
  }
  R[e] = r;
}

// max_i sum_j |B_ij|
__global__ void row_norm_kernel(const int32_t* __restrict__ B, int n, int d, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t s = 0;
  for (int j = 0; j < d; ++j) s += abs(B[(int64_t)i * d + j]);
  atomicMax(out, (int32_t)(s < 0x7fffffff ? s : 0x7fffffff));
}

// The collection of Algorithm 2 after the GEMM B round(Z): map (one thread
// per start whose rounding changed) tests C4, finds the first nonzero entry
// and stages the row as int8 [n x P]; append (one warp per such start) takes
// a slot for a valid row and writes it in canonical sign.
constexpr int kNoFirst = 0x7f7f7f7f;  // a byte pattern, so that cudaMemset can write it

__global__ void map_kernel(const float* __restrict__ Gm, const int32_t* __restrict__ span,
                           const uint8_t* __restrict__ changed, int n, int P, int8_t* __restrict__ S8,
                           uint32_t* __restrict__ bad, int32_t* __restrict__ first) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P || !changed[p]) return;
  uint32_t fl = 0u;
  int fz = kNoFirst;
  for (int i = 0; i < n; ++i) {
    const int g = (int)Gm[(int64_t)i * P + p];
    if (g > span[i] || -g > span[i]) fl |= 1u;
    if (g != 0 && fz == kNoFirst) fz = (i << 1) | (g < 0 ? 1 : 0);
    S8[(int64_t)i * P + p] = (int8_t)g;
  }
  if (fl) atomicOr(&bad[p], fl);
  first[p] = fz;
}

__global__ void append_kernel(uint8_t* __restrict__ changed, uint32_t* __restrict__ bad, int32_t* __restrict__ first,
                              const int8_t* __restrict__ S8, int n, int P, int8_t* __restrict__ cand, int ldc,
                              int64_t cap, unsigned long long* __restrict__ count, int32_t* __restrict__ flags) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= P || !changed[p]) return;
  long long slot = -1;
  int neg = 0;
  if (lane == 0) {
    const uint32_t b = bad[p];
    const int f = first[p];
    changed[p] = 0;
    bad[p] = 0u;
    first[p] = kNoFirst;
    if (b & 4u) {
      atomicOr(flags, 4);
    } else if (!(b & 1u) && f != kNoFirst) {
      const unsigned long long at = atomicAdd(count, 1ull);
      if ((int64_t)at < cap) slot = (long long)at;
      else atomicOr(flags, 1);
    }
    neg = f & 1;
  }
  slot = __shfl_sync(0xffffffffu, slot, 0);
  neg = __shfl_sync(0xffffffffu, neg, 0);
  if (slot < 0) return;
  int8_t* row = cand + slot * ldc;
  for (int i = lane; i < ldc; i += 32) {
    const int v = i < n ? (int)S8[(int64_t)i * P + p] : 0;
    row[i] = (int8_t)(neg ? -v : v);
  }
}

__global__ void fill_u8_kernel(uint8_t* p, uint8_t v, int64_t count) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < count) p[i] = v;
}

// Eq. (3) and its gradient, one block per start (parity tool, mape_phi_grad).
__global__ void phi_grad_kernel(const int32_t* __restrict__ B, const float* __restrict__ Z,
                                int n, int d, float lambda1, float lambda2,
                                float* __restrict__ phi, float* __restrict__ grad) {
  extern __shared__ int8_t s_sign[];
  __shared__ float red[32];
  __shared__ int redk[32];
  int p = blockIdx.x;
  const float* z = Z + (int64_t)p * d;
  float l1 = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float y = 0.f;
    for (int j = 0; j < d; ++j) y = fmaf((float)B[(int64_t)i * d + j], z[j], y);
    s_sign[i] = (int8_t)mape_sign_f(y);
    l1 += fabsf(y);
  }
  // block reductions: l1, frac, (zinf, first argmax)
  float frac = 0.f, zinf = 0.f;
  int kmax = 1 << 30;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    float zj = z[j];
    frac += (zj - floorf(zj)) * (ceilf(zj) - zj);
    float a = fabsf(zj);
    if (a > zinf || (a == zinf && j < kmax)) { zinf = a; kmax = j; }
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    l1 += __shfl_xor_sync(0xffffffffu, l1, off);
    frac += __shfl_xor_sync(0xffffffffu, frac, off);
    float oz = __shfl_xor_sync(0xffffffffu, zinf, off);
    int ok = __shfl_xor_sync(0xffffffffu, kmax, off);
    if (oz > zinf || (oz == zinf && ok < kmax)) { zinf = oz; kmax = ok; }
  }
  __shared__ float rl1[32], rfr[32];
  if (lane == 0) { rl1[wid] = l1; rfr[wid] = frac; red[wid] = zinf; redk[wid] = kmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float L = 0.f, F = 0.f, Zi = 0.f;
    int K = 1 << 30;
    for (int w = 0; w < nw; ++w) {
      L += rl1[w]; F += rfr[w];
      if (red[w] > Zi || (red[w] == Zi && redk[w] < K)) { Zi = red[w]; K = redk[w]; }
    }
    float inv = Zi > 0.f ? fmaxf(1.f / Zi - 1.f, 0.f) : INFINITY;
    phi[p] = L + lambda1 * F + lambda2 * inv;
    red[0] = Zi;
    redk[0] = K;
  }
  __syncthreads();
  zinf = red[0];
  kmax = redk[0];
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    float g = 0.f;
    for (int i = 0; i < n; ++i) g += (float)(B[(int64_t)i * d + j] * s_sign[i]);
    float zj = z[j];
    g += lambda1 * (ceilf(zj) + floorf(zj) - 2.f * zj);
    if (j == kmax && zinf < 1.f && zinf > 0.f) g += -lambda2 * (float)mape_sign_f(zj) / (zinf * zinf);
    grad[(int64_t)p * d + j] = g;
  }
}

template <typename Carve>
void carve_fp32(Carve& cv, int32_t n, int32_t d, int32_t P) {
  cv.template take<float>((size_t)n * d);                           // Bf
  for (int k = 0; k < 3; ++k) cv.template take<float>((size_t)d * P);  // Zt, Mt, Vt
  cv.template take<float>((size_t)n * P);                           // Y, then B round(Z)
  cv.template take<float>((size_t)n * P);                           // S
  cv.template take<float>((size_t)d * P);                           // G, then round(Z)
  cv.template take<float>((size_t)P);                               // ||z||_inf
  cv.template take<int32_t>((size_t)P);                             // its first index
  cv.template take<uint8_t>((size_t)P);                             // changed
  cv.template take<int8_t>((size_t)n * P);                          // staged candidate rows
  cv.template take<uint32_t>((size_t)P);                            // bound / range flags
  cv.template take<int32_t>((size_t)P);                             // first nonzero entry
  cv.template take<int32_t>(1);                                     // max row sum of |B|
}

// One cuBLAS handle per device for the process, created on first use; a
// call holds its mutex while it sets the handle's stream and enqueues (a
// cuBLAS handle must not be used by two threads at once).
struct BlasHandles {
  std::mutex mu;
  std::map<int, cublasHandle_t> by_dev;
};
BlasHandles& blas_handles() {
  static BlasHandles* h = new BlasHandles();  // never destroyed: lives until the process exits
  return *h;
}

}  // namespace

namespace mape_detail {

void adam_bias_table(const mape_extract_args* a, std::vector<float2>& out) {
  out.resize(a->T > 0 ? a->T : 0);
  for (int s = 0; s < a->T; ++s) {
    double t = (double)a->t0 + s + 1;
    out[s] = make_float2((float)(1.0 - std::pow((double)a->beta1, t)),
                         (float)(1.0 - std::pow((double)a->beta2, t)));
  }
}

size_t extract_fp32_workspace(int32_t n, int32_t d, int32_t P) {
  Sizer s;
  carve_fp32(s, n, d, P);
  return s.bytes();
}

#define MAPE_BLAS_TRY(expr)                                                               \
  do {                                                                                    \
    if ((expr) != CUBLAS_STATUS_SUCCESS) {                                                \
      mape_detail::record_cuda_error(cudaErrorUnknown, #expr " (cuBLAS)", __FILE__, __LINE__); \
      return MAPE_ERR_CUDA;                                                               \
    }                                                                                     \
  } while (0)

int extract_fp32(const mape_extract_args* a, cudaStream_t st) {
  const int n = a->n, d = a->d, P = a->P;
  Carver cv(a->workspace, a->workspace_bytes);
  float* Bf = cv.take<float>((size_t)n * d);
  float* Zt = cv.take<float>((size_t)d * P);
  float* Mt = cv.take<float>((size_t)d * P);
  float* Vt = cv.take<float>((size_t)d * P);
  float* Y = cv.take<float>((size_t)n * P);
  float* S = cv.take<float>((size_t)n * P);
  float* G = cv.take<float>((size_t)d * P);
  float* zinf = cv.take<float>((size_t)P);
  int32_t* kmax = cv.take<int32_t>((size_t)P);
  uint8_t* changed = cv.take<uint8_t>((size_t)P);
  int8_t* S8 = cv.take<int8_t>((size_t)n * P);
  uint32_t* badw = cv.take<uint32_t>((size_t)P);
  int32_t* firstw = cv.take<int32_t>((size_t)P);
  int32_t* bnorm = cv.take<int32_t>(1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  int dev = 0;
  MAPE_CUDA_TRY(cudaGetDevice(&dev));
  BlasHandles& H = blas_handles();
  std::lock_guard<std::mutex> blas_lock(H.mu);
  cublasHandle_t& hb = H.by_dev[dev];
  if (!hb) {
    MAPE_BLAS_TRY(cublasCreate(&hb));
    MAPE_BLAS_TRY(cublasSetMathMode(hb, CUBLAS_PEDANTIC_MATH));  // strict FP32
  }
  MAPE_BLAS_TRY(cublasSetStream(hb, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(badw, 0, sizeof(uint32_t) * P, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(firstw, 0x7f, sizeof(int32_t) * P, st));
  MAPE_CUDA_TRY(cudaMemsetAsync(bnorm, 0, sizeof(int32_t), st));

  std::vector<float2> bc;
  adam_bias_table(a, bc);

  launch(to_float_kernel, (unsigned)ceil_div((int64_t)n * d, 256), 256, 0, st, a->B, Bf, (int64_t)n * d);
  launch(row_norm_kernel, (unsigned)ceil_div(n, 128), 128, 0, st, a->B, n, d, bnorm);
  dim3 tb(32, 8);
  launch(transpose_kernel, dim3((unsigned)ceil_div(d, 32), (unsigned)ceil_div(P, 32)), tb, 0, st, a->Z, Zt, P, d);
  launch(transpose_kernel, dim3((unsigned)ceil_div(d, 32), (unsigned)ceil_div(P, 32)), tb, 0, st, a->M, Mt, P, d);
  launch(transpose_kernel, dim3((unsigned)ceil_div(d, 32), (unsigned)ceil_div(P, 32)), tb, 0, st, a->V, Vt, P, d);
  launch(fill_u8_kernel, (unsigned)ceil_div(P, 256), 256, 0, st, changed, 1, P);
  MAPE_LAUNCH_CHECK();
  int32_t h_bnorm = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&h_bnorm, bnorm, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  // |round z_j| <= rlim keeps every partial sum of B round(z) below 2^24
  const float rlim = h_bnorm > 0 ? std::floor(16777215.f / (float)h_bnorm) : 16777215.f;

  const float one = 1.f, zero = 0.f;
  const int64_t nP = (int64_t)n * P, dP = (int64_t)d * P;
  const unsigned g_n = (unsigned)ceil_div(nP, 256), g_d = (unsigned)ceil_div(dP, 256);
  const unsigned g_p = (unsigned)ceil_div(P, 128), g_pw = (unsigned)ceil_div((int64_t)P * 32, 256);
  for (int s = 0; s < a->T; ++s) {
    const bool dbg = s == 0;
    StepParams sp{a->lambda1, a->lambda2, a->lr, (float)a->beta1, (float)a->beta2, (float)(1.0 - a->beta1),
                  (float)(1.0 - a->beta2), a->eps, bc[s].x, bc[s].y};
    // column-major views: Zt is P x d (ld P), Bf is d x n (ld d), Y and S are P x n, G is P x d
    MAPE_BLAS_TRY(cublasSgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, P, n, d, &one, Zt, P, Bf, d, &zero, Y, P));
    launch(sign_kernel, g_n, 256, 0, st, Y, S, nP);
    MAPE_BLAS_TRY(cublasSgemm(hb, CUBLAS_OP_N, CUBLAS_OP_T, P, d, n, &one, S, P, Bf, d, &zero, G, P));
    launch(zinf_kernel, g_p, 128, 0, st, Zt, Y, n, d, P, zinf, kmax, a->lambda1, a->lambda2,
           dbg ? a->dbg_phi : nullptr);
    launch(adam_kernel, g_d, 256, 0, st, G, Zt, Mt, Vt, zinf, kmax, changed, sp, d, P, dbg ? a->dbg_grad : nullptr);
    const int t = a->t0 + s + 1;
    if (t % a->period == 0) {
      launch(round_kernel, g_d, 256, 0, st, Zt, G, d, P, rlim, changed, badw);
      MAPE_BLAS_TRY(cublasSgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, P, n, d, &one, G, P, Bf, d, &zero, Y, P));
      launch(map_kernel, g_p, 128, 0, st, Y, a->span, changed, n, P, S8, badw, firstw);
      launch(append_kernel, g_pw, 256, 0, st, changed, badw, firstw, S8, n, P, a->cand, a->ldc, a->cand_cap,
             a->cand_count, a->flags);
    }
    MAPE_LAUNCH_CHECK();
  }
  launch(transpose_kernel, dim3((unsigned)ceil_div(P, 32), (unsigned)ceil_div(d, 32)), tb, 0, st, Zt, a->Z, d, P);
  launch(transpose_kernel, dim3((unsigned)ceil_div(P, 32), (unsigned)ceil_div(d, 32)), tb, 0, st, Mt, a->M, d, P);
  launch(transpose_kernel, dim3((unsigned)ceil_div(P, 32), (unsigned)ceil_div(d, 32)), tb, 0, st, Vt, a->V, d, P);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}

}  // namespace mape_detail

extern "C" int mape_phi_grad(const int32_t* B, int32_t n, int32_t d, const float* Z, int32_t P,
                             float lambda1, float lambda2, float* phi, float* grad, void* stream) {
  if (n <= 0 || d <= 0 || P < 0 || !B || (P > 0 && (!Z || !phi || !grad))) return MAPE_ERR_INVALID_ARG;
  if (n > 48 * 1024) return MAPE_ERR_SHAPE;
  if (P == 0) return MAPE_OK;
  mape_detail::launch(phi_grad_kernel, P, 128, (size_t)n, mape_detail::as_stream(stream), B, Z, n, d, lambda1, lambda2, phi, grad);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}
