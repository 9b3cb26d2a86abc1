// a2: starting points z0 = (B^T B)^{-1} B^T g (§3.2, Algorithm 2).
//
// Per instance: H = B^T B (exact in int64, rounded to FP32), its Cholesky
// factor L (blocked, right-looking, panels of 64 columns, d <= 4096) and
// W = B H^{-1} (n x d) by a forward and a backward triangular solve per row
// of B.  Per start: z0 = W^T g, i.e. Z0 = G0 W for all starts at once with a
// tiled FP32 GEMM (64 x 64 output tiles, 4 x 4 per thread).
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

// Blocked right-looking Cholesky of the lower triangle of H (row-major,
// d x d), panel width kNB: per panel, (1) the diagonal block is factored in
// shared memory by one CTA, (2) the rows below it are solved against it
// (L21 = A21 L11^{-T}, one thread per row), (3) the trailing matrix takes the
// rank-kNB update A22 -= L21 L21^T on 64 x 64 tiles of its lower triangle.
// Only the lower triangle is read and written; the upper one is left as is.
constexpr int kNB = 64;

__global__ void chol_diag_kernel(float* __restrict__ H, int d, int k0, int32_t* __restrict__ status) {
  __shared__ float a[kNB][kNB + 1];
  const int nb = min(kNB, d - k0);
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    a[i][j] = j <= i ? H[(int64_t)(k0 + i) * d + k0 + j] : 0.f;
  }
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (threadIdx.x == 0) {
      float p = a[k][k];
      if (!(p > 0.f)) { *status = 1; p = 1.f; }
      a[k][k] = sqrtf(p);
    }
    __syncthreads();
    const float piv = a[k][k];
    for (int i = k + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][k] /= piv;
    __syncthreads();
    const int m = nb - k - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) a[i][j] -= a[i][k] * a[j][k];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    if (j <= i) H[(int64_t)(k0 + i) * d + k0 + j] = a[i][j];
  }
}

constexpr int kPanelRows = 64;  // keeps the static shared memory under 48 KB

__global__ void __launch_bounds__(kPanelRows) chol_panel_kernel(float* __restrict__ H, int d, int k0) {
  __shared__ float L11[kNB][kNB + 1];
  __shared__ float xs[kPanelRows][kNB + 1];
  const int nb = min(kNB, d - k0);
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    L11[i][j] = j <= i ? H[(int64_t)(k0 + i) * d + k0 + j] : 0.f;
  }
  const int row0 = k0 + nb + blockIdx.x * kPanelRows;
  for (int e = threadIdx.x; e < kPanelRows * nb; e += blockDim.x) {
    const int r = e / nb, t = e % nb;
    xs[r][t] = row0 + r < d ? H[(int64_t)(row0 + r) * d + k0 + t] : 0.f;
  }
  __syncthreads();
  const int i = row0 + threadIdx.x;
  if (i < d) {
    float* x = xs[threadIdx.x];
    for (int j = 0; j < nb; ++j) {
      float acc = x[j];
      for (int t = 0; t < j; ++t) acc -= x[t] * L11[j][t];
      x[j] = acc / L11[j][j];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kPanelRows * nb; e += blockDim.x) {
    const int r = e / nb, t = e % nb;
    if (row0 + r < d) H[(int64_t)(row0 + r) * d + k0 + t] = xs[r][t];
  }
}

__global__ void __launch_bounds__(256) chol_update_kernel(float* __restrict__ H, int d, int k0) {
  const int nb = min(kNB, d - k0), base = k0 + nb;
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (tj > ti) return;  // lower-triangular tiles only
  const int r0 = base + ti * 64, c0 = base + tj * 64;
  __shared__ float sa[kNB][64 + 4];
  __shared__ float sb[kNB][64 + 4];
  for (int e = threadIdx.x; e < 64 * nb; e += 256) {
    const int r = e / nb, t = e % nb;
    sa[t][r] = r0 + r < d ? H[(int64_t)(r0 + r) * d + k0 + t] : 0.f;
    sb[t][r] = c0 + r < d ? H[(int64_t)(c0 + r) * d + k0 + t] : 0.f;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int t = 0; t < nb; ++t) {
    float av[4], bv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { av[q] = sa[t][ty * 4 + q]; bv[q] = sb[t][tx * 4 + q]; }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = r0 + ty * 4 + p;
    if (i >= d) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = c0 + tx * 4 + q;
      if (j < d && j <= i) H[(int64_t)i * d + j] -= acc[p][q];
    }
  }
}

// Lt = L^T (upper triangle; the strict lower part of Lt is zero)
__global__ void transpose_lower_kernel(const float* __restrict__ L, int d, float* __restrict__ Lt) {
  __shared__ float tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int i = by + y, j = bx + threadIdx.x;
    tile[y][threadIdx.x] = (i < d && j < d && j <= i) ? L[(int64_t)i * d + j] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int i = bx + y, j = by + threadIdx.x;  // Lt[i][j] = L[j][i]
    if (i < d && j < d) Lt[(int64_t)i * d + j] = tile[threadIdx.x][y];
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Row r of W = B H^{-1} = H^{-1} B_r^T (H symmetric): forward solve L u = B_r^T,
// backward solve L^T w = u; one warp per row, the vector in shared memory.
constexpr int kSolveWarps = 4;

__global__ void __launch_bounds__(32 * kSolveWarps) w_solve_kernel(const int32_t* __restrict__ B, const float* __restrict__ L,
                                                          const float* __restrict__ Lt, int n, int d,
                                                          float* __restrict__ W) {
  extern __shared__ float s_vec[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * kSolveWarps + warp;
  if (r >= n) return;  // warp-uniform
  float* u = s_vec + (size_t)warp * d;
  for (int i = lane; i < d; i += 32) u[i] = (float)B[(int64_t)r * d + i];
  __syncwarp();
  for (int i = 0; i < d; ++i) {
    const float* Li = L + (int64_t)i * d;
    float part = 0.f;
    for (int k = lane; k < i; k += 32) part = fmaf(Li[k], u[k], part);
    const float tot = warp_sum(part);
    const float ui = (u[i] - tot) / Li[i];
    __syncwarp();
    if (lane == 0) u[i] = ui;
    __syncwarp();
  }
  for (int i = d - 1; i >= 0; --i) {
    const float* Ri = Lt + (int64_t)i * d;
    float part = 0.f;
    for (int k = i + 1 + lane; k < d; k += 32) part = fmaf(Ri[k], u[k], part);
    const float tot = warp_sum(part);
    const float wi = (u[i] - tot) / Ri[i];
    __syncwarp();
    if (lane == 0) u[i] = wi;
    __syncwarp();
  }
  for (int i = lane; i < d; i += 32) W[(int64_t)r * d + i] = u[i];
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
  s.take<float>((size_t)d * d);   // H, then its Cholesky factor L
  s.take<float>((size_t)d * d);   // L^T
  s.take<float>((size_t)d * d);   // (reserved)
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
  float* Lt = cv.take<float>((size_t)d * d);
  cv.take<float>((size_t)d * d);
  int32_t* status = cv.take<int32_t>(1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  MAPE_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  const unsigned gd = (unsigned)ceil_div(d, 128);
  mape_detail::launch(gram_kernel, dim3(gd, (unsigned)d), 128, 0, st, B, n, d, H);
  for (int k0 = 0; k0 < d; k0 += kNB) {
    mape_detail::launch(chol_diag_kernel, 1, 256, 0, st, H, d, k0, status);
    const int rest = d - k0 - kNB;
    if (rest > 0) {
      mape_detail::launch(chol_panel_kernel, (unsigned)ceil_div(rest, kPanelRows), kPanelRows, 0, st, H, d, k0);
      const unsigned T = (unsigned)ceil_div(rest, 64);
      mape_detail::launch(chol_update_kernel, dim3(T, T), 256, 0, st, H, d, k0);
    }
  }
  const unsigned g32 = (unsigned)ceil_div(d, 32);
  mape_detail::launch(transpose_lower_kernel, dim3(g32, g32), dim3(32, 8), 0, st, H, d, Lt);
  const size_t smem = (size_t)kSolveWarps * d * sizeof(float);
  {
    size_t lim = 0;
    const int rc = allow_max_dynamic_smem((const void*)w_solve_kernel, &lim);
    if (rc != MAPE_OK) return rc;
    if ((size_t)smem > lim) return MAPE_ERR_SHAPE;
  }
  mape_detail::launch(w_solve_kernel, (unsigned)ceil_div(n, kSolveWarps), 32 * kSolveWarps, smem, st, B, H, Lt, n,
                      d, W);
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
