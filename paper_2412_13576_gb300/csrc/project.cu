// a2: starting points z0 = (B^T B)^{-1} B^T g (§3.2, Algorithm 2).
//
// B^T B is formed exactly in int64 and rounded to FP32, factored in place by
// a one-block right-looking Cholesky (d <= 4096), and every start solves
// L L^T z = B^T g in its own output row (one thread per start).
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

__global__ void solve_kernel(const int32_t* __restrict__ B, const float* __restrict__ L, const float* __restrict__ G0,
                             int n, int d, int P, float* __restrict__ Z) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float* z = Z + (int64_t)p * d;
  const float* g = G0 + (int64_t)p * n;
  for (int j = 0; j < d; ++j) {  // rhs = B^T g
    float acc = 0.f;
    for (int i = 0; i < n; ++i) acc = fmaf((float)B[(int64_t)i * d + j], g[i], acc);
    z[j] = acc;
  }
  for (int j = 0; j < d; ++j) {  // L y = rhs
    float acc = z[j];
    for (int k = 0; k < j; ++k) acc -= L[(int64_t)j * d + k] * z[k];
    z[j] = acc / L[(int64_t)j * d + j];
  }
  for (int j = d - 1; j >= 0; --j) {  // L^T z = y
    float acc = z[j];
    for (int k = j + 1; k < d; ++k) acc -= L[(int64_t)k * d + j] * z[k];
    z[j] = acc / L[(int64_t)j * d + j];
  }
}

}  // namespace

extern "C" size_t mape_project_workspace_bytes(int32_t n, int32_t d) {
  (void)n;
  if (d <= 0) return 0;
  mape_detail::Sizer s;
  s.take<float>((size_t)d * d);
  s.take<int32_t>(1);
  return s.bytes();
}

extern "C" int mape_project_starts(const int32_t* B, int32_t n, int32_t d, const float* G0, int32_t P,
                                   float* Z0, void* workspace, size_t workspace_bytes, void* stream) {
  using namespace mape_detail;
  if (!B || n <= 0 || d <= 0 || d > n || P < 0 || (P > 0 && (!G0 || !Z0))) return MAPE_ERR_INVALID_ARG;
  if (d > 4096) return MAPE_ERR_SHAPE;
  Carver cv(workspace, workspace_bytes);
  float* H = cv.take<float>((size_t)d * d);
  int32_t* status = cv.take<int32_t>(1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  MAPE_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  mape_detail::launch(gram_kernel, dim3((unsigned)ceil_div(d, 128), (unsigned)d), 128, 0, st, B, n, d, H);
  mape_detail::launch(cholesky_kernel, 1, 1024, 0, st, H, d, status);
  if (P > 0) mape_detail::launch(solve_kernel, (unsigned)ceil_div(P, 128), 128, 0, st, B, H, G0, n, d, P, Z0);
  MAPE_LAUNCH_CHECK();
  int32_t h_status = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&h_status, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  return h_status ? MAPE_ERR_NUMERIC : MAPE_OK;
}
