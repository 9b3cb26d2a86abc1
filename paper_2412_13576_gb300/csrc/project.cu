// a2: starting points z0 = (B^T B)^{-1} B^T g (§3.2, Algorithm 2).
//
// Per instance: H = B^T B (exact in int64, rounded to FP32), its Cholesky
// factor L (one block, right-looking, d <= 4096), L^{-1} by forward
// substitution (one thread per column), H^{-1} = L^{-T} L^{-1} and
// W = B H^{-1} (n x d).  Per start: z0 = W^T g, i.e. Z0 = G0 W for all starts
// at once with a tiled FP32 GEMM (64 x 64 output tiles, 4 x 4 per thread).
#include "common.cuh"

namespace {

__global__ void gram_kernel(const int32_t* __restrict__ B, int n, int d, float* __restrict__ H) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  if (j >= d || j < k) return;  // lower triangle: row j >= column k
  long long acc = 0;
  for (int i = 0; i < n; ++i) acc += (long long)B[(int64_t)i * d + j] * B[(int64_t)i * d + k];
  H[(int64_t)j * d + k] = (float)acc;
  H[(int64_t)k * d + j] = (float)acc;
}

// In-place Cholesky of the lower triangle of H (row-major, d x d).
__global__ void cholesky_kernel(float* __restrict__ H, int d, int32_t* __restrict__ status) {
  __shared__ float s_pivot;
  for (int k = 0; k < d; ++k) {
    if (threadIdx.x == 0) {
      float p = H[(int64_t)k * d + k];
      if (!(p > 0.f)) { *status = 1; p = 1.f; }
      s_pivot = sqrtf(p);
      H[(int64_t)k * d + k] = s_pivot;
    }
    __syncthreads();
    float piv = s_pivot;
    for (int i = k + 1 + threadIdx.x; i < d; i += blockDim.x) H[(int64_t)i * d + k] /= piv;
    __syncthreads();
    // trailing update of rows i > k, columns k < j <= i
    int64_t m = d - k - 1;
    int64_t pairs = m * (m + 1) / 2;
    for (int64_t q = threadIdx.x; q < pairs; q += blockDim.x) {
      // q -> (ii, jj) with 0 <= jj <= ii < m, row-major over the triangle
      int64_t ii = (int64_t)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
      while (ii * (ii + 1) / 2 > q) --ii;
      while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
      int64_t jj = q - ii * (ii + 1) / 2;
      int64_t i = k + 1 + ii, j = k + 1 + jj;
      H[i * d + j] -= H[i * d + k] * H[j * d + k];
    }
    __syncthreads();
  }
}

// Y = L^{-1}, one thread per column c: L y = e_c (y_i = 0 for i < c)
__global__ void lower_inverse_kernel(const float* __restrict__ L, int d, float* __restrict__ Y) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d) return;
  for (int i = 0; i < d; ++i) {
    float acc = (i == c) ? 1.f : 0.f;
    if (i >= c)
      for (int k = c; k < i; ++k) acc -= L[(int64_t)i * d + k] * Y[(int64_t)k * d + c];
    Y[(int64_t)i * d + c] = i >= c ? acc / L[(int64_t)i * d + i] : 0.f;
  }
}

// Hi = Y^T Y (= H^{-1}); Y lower triangular
__global__ void hinv_kernel(const float* __restrict__ Y, int d, float* __restrict__ Hi) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  if (j >= d) return;
  float acc = 0.f;
  for (int r = max(j, k); r < d; ++r) acc = fmaf(Y[(int64_t)r * d + j], Y[(int64_t)r * d + k], acc);
  Hi[(int64_t)k * d + j] = acc;
}

// W = B Hi (n x d)
__global__ void w_kernel(const int32_t* __restrict__ B, const float* __restrict__ Hi, int n, int d,
                         float* __restrict__ W) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= d) return;
  float acc = 0.f;
  for (int k = 0; k < d; ++k) {
    int b = B[(int64_t)i * d + k];
    if (b) acc = fmaf((float)b, Hi[(int64_t)k * d + j], acc);
  }
  W[(int64_t)i * d + j] = acc;
}

// Z0 [P x d] = G0 [P x n] . W [n x d]
constexpr int kTM = 64, kTN = 64, kTK = 16;

__global__ void __launch_bounds__(256) gemm_kernel(const float* __restrict__ G0, const float* __restrict__ W, int P,
                                                    int n, int d, float* __restrict__ Z) {
  __shared__ float sA[kTK][kTM + 4];
  __shared__ float sB[kTK][kTN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.y * kTM, col0 = blockIdx.x * kTN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += kTK) {
    for (int e = threadIdx.x; e < kTM * kTK; e += 256) {
      int r = e / kTK, k = e % kTK;
      int gr = row0 + r, gk = k0 + k;
      sA[k][r] = (gr < P && gk < n) ? G0[(int64_t)gr * n + gk] : 0.f;
    }
    for (int e = threadIdx.x; e < kTK * kTN; e += 256) {
      int k = e / kTN, c = e % kTN;
      int gk = k0 + k, gc = col0 + c;
      sB[k][c] = (gk < n && gc < d) ? W[(int64_t)gk * d + gc] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTK; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[k][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[k][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = row0 + ty * 4 + i;
    if (r >= P) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = col0 + tx * 4 + j;
      if (c < d) Z[(int64_t)r * d + c] = acc[i][j];
    }
  }
}

}  // namespace

extern "C" size_t mape_project_prepare_workspace_bytes(int32_t n, int32_t d) {
  (void)n;
  if (d <= 0) return 0;
  mape_detail::Sizer s;
  s.take<float>((size_t)d * d);   // H, then its Cholesky factor
  s.take<float>((size_t)d * d);   // L^{-1}
  s.take<float>((size_t)d * d);   // H^{-1}
  s.take<int32_t>(1);
  return s.bytes();
}

extern "C" int mape_project_prepare(const int32_t* B, int32_t n, int32_t d, float* W, void* workspace,
                                    size_t workspace_bytes, void* stream) {
  using namespace mape_detail;
  if (!B || !W || n <= 0 || d <= 0 || d > n) return MAPE_ERR_INVALID_ARG;
  if (d > 4096) return MAPE_ERR_SHAPE;
  Carver cv(workspace, workspace_bytes);
  float* H = cv.take<float>((size_t)d * d);
  float* Y = cv.take<float>((size_t)d * d);
  float* Hi = cv.take<float>((size_t)d * d);
  int32_t* status = cv.take<int32_t>(1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  MAPE_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  const unsigned gd = (unsigned)ceil_div(d, 128);
  mape_detail::launch(gram_kernel, dim3(gd, (unsigned)d), 128, 0, st, B, n, d, H);
  mape_detail::launch(cholesky_kernel, 1, 1024, 0, st, H, d, status);
  mape_detail::launch(lower_inverse_kernel, gd, 128, 0, st, H, d, Y);
  mape_detail::launch(hinv_kernel, dim3(gd, (unsigned)d), 128, 0, st, Y, d, Hi);
  mape_detail::launch(w_kernel, dim3(gd, (unsigned)n), 128, 0, st, B, Hi, n, d, W);
  MAPE_LAUNCH_CHECK();
  int32_t h_status = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&h_status, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  return h_status ? MAPE_ERR_NUMERIC : MAPE_OK;
}

extern "C" int mape_project_apply(const float* W, int32_t n, int32_t d, const float* G0, int32_t P, float* Z0,
                                  void* stream) {
  using namespace mape_detail;
  if (!W || n <= 0 || d <= 0 || d > n || P < 0 || (P > 0 && (!G0 || !Z0))) return MAPE_ERR_INVALID_ARG;
  if (P == 0) return MAPE_OK;
  mape_detail::launch(gemm_kernel, dim3((unsigned)ceil_div(d, kTN), (unsigned)ceil_div(P, kTM)), 256, 0,
                      as_stream(stream), G0, W, P, n, d, Z0);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}

extern "C" size_t mape_project_workspace_bytes(int32_t n, int32_t d) {
  if (d <= 0 || n <= 0) return 0;
  mape_detail::Sizer s;
  s.take<float>((size_t)n * d);                                   // W
  s.take<char>(mape_project_prepare_workspace_bytes(n, d));
  return s.bytes();
}

extern "C" int mape_project_starts(const int32_t* B, int32_t n, int32_t d, const float* G0, int32_t P,
                                   float* Z0, void* workspace, size_t workspace_bytes, void* stream) {
  using namespace mape_detail;
  if (!B || n <= 0 || d <= 0 || d > n || P < 0 || (P > 0 && (!G0 || !Z0))) return MAPE_ERR_INVALID_ARG;
  if (d > 4096) return MAPE_ERR_SHAPE;
  Carver cv(workspace, workspace_bytes);
  float* W = cv.take<float>((size_t)n * d);
  size_t pb = mape_project_prepare_workspace_bytes(n, d);
  char* pw = cv.take<char>(pb);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  int rc = mape_project_prepare(B, n, d, W, pw, pb, stream);
  if (rc != MAPE_OK) return rc;
  return mape_project_apply(W, n, d, G0, P, Z0, stream);
}
