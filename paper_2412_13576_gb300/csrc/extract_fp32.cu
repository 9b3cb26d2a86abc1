// Algorithm 2 (§3.2) on CUDA cores in FP32: the plain per-step path.
//
// Per Adam step three unfused kernels run over all P starts:
//   forward_sign   S = sign(B z) (int8, coordinate-major), partial ||Bz||_1
//   backward_adam  grad = B^T S + lambda1 (ceil z + floor z - 2 z) + inverse
//                  norm term (Eq. (3)); Adam update of z, m, v; marks starts
//                  whose rounding changed
//   collect        for marked starts (one warp each): g = B round(z) in int32,
//                  nonzero and C4 tests, canonical sign, append
// State is kept coordinate-major ([d][P]) so that one thread per start reads
// and writes coalesced rows; B is read through L1 as warp-wide broadcasts.
#include "common.cuh"
#include "extract_internal.cuh"

#include <vector>
#include <cmath>

namespace {

constexpr int kThreads = 128;
constexpr int kRowBlock = 16;   // rows of B per forward thread
constexpr int kColBlock = 16;   // coordinates per backward pass

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

__global__ void forward_sign_kernel(const float* __restrict__ Bf, const float* __restrict__ Zt,
                                    int8_t* __restrict__ S, float* __restrict__ l1_part,
                                    int n, int d, int P) {
  int p = blockIdx.x * kThreads + threadIdx.x;
  int i0 = blockIdx.y * kRowBlock;
  if (p >= P) return;
  float acc[kRowBlock];
#pragma unroll
  for (int r = 0; r < kRowBlock; ++r) acc[r] = 0.f;
  int rows = min(kRowBlock, n - i0);
  for (int j = 0; j < d; ++j) {
    float zj = Zt[(int64_t)j * P + p];
#pragma unroll
    for (int r = 0; r < kRowBlock; ++r)
      if (r < rows) acc[r] = fmaf(Bf[(int64_t)(i0 + r) * d + j], zj, acc[r]);
  }
  float l1 = 0.f;
#pragma unroll
  for (int r = 0; r < kRowBlock; ++r) {
    if (r < rows) {
      S[(int64_t)(i0 + r) * P + p] = (int8_t)mape_sign_f(acc[r]);
      l1 += fabsf(acc[r]);
    }
  }
  if (l1_part) l1_part[(int64_t)blockIdx.y * P + p] = l1;
}

struct StepParams {
  float lambda1, lambda2, lr, beta1, beta2, omb1, omb2, eps, bc1, bc2;
};

__global__ void backward_adam_kernel(const float* __restrict__ Bf, const int8_t* __restrict__ S,
                                     float* __restrict__ Zt, float* __restrict__ Mt, float* __restrict__ Vt,
                                     uint8_t* __restrict__ changed, StepParams sp,
                                     int n, int d, int P, const float* __restrict__ l1_part, int nblk,
                                     float* __restrict__ dbg_phi, float* __restrict__ dbg_grad) {
  int p = blockIdx.x * kThreads + threadIdx.x;
  if (p >= P) return;
  // ||z||_inf and its first maximiser (inverse-norm term of Eq. (3))
  float zinf = 0.f;
  int kmax = 0;
  float frac = 0.f;
  for (int j = 0; j < d; ++j) {
    float zj = Zt[(int64_t)j * P + p];
    float a = fabsf(zj);
    if (a > zinf) { zinf = a; kmax = j; }
    if (dbg_phi) frac += (zj - floorf(zj)) * (ceilf(zj) - zj);
  }
  float inv_term = 0.f;  // gradient entry added at kmax
  if (zinf < 1.f && zinf > 0.f) {
    float zk = Zt[(int64_t)kmax * P + p];
    inv_term = -sp.lambda2 * (float)mape_sign_f(zk) / (zinf * zinf);
  }
  if (dbg_phi) {
    float l1 = 0.f;
    for (int b = 0; b < nblk; ++b) l1 += l1_part[(int64_t)b * P + p];
    float inv = zinf > 0.f ? fmaxf(1.f / zinf - 1.f, 0.f) : INFINITY;
    dbg_phi[p] = l1 + sp.lambda1 * frac + sp.lambda2 * inv;
  }
  bool moved = false;
  for (int j0 = 0; j0 < d; j0 += kColBlock) {
    float g[kColBlock];
#pragma unroll
    for (int c = 0; c < kColBlock; ++c) g[c] = 0.f;
    int cols = min(kColBlock, d - j0);
    for (int i = 0; i < n; ++i) {
      int s = S[(int64_t)i * P + p];
      if (s == 0) continue;
      float fs = (float)s;
      const float* brow = Bf + (int64_t)i * d + j0;
#pragma unroll
      for (int c = 0; c < kColBlock; ++c)
        if (c < cols) g[c] = fmaf(brow[c], fs, g[c]);
    }
#pragma unroll
    for (int c = 0; c < kColBlock; ++c) {
      if (c >= cols) continue;
      int j = j0 + c;
      int64_t at = (int64_t)j * P + p;
      float z = Zt[at];
      float grad = g[c] + sp.lambda1 * (ceilf(z) + floorf(z) - 2.f * z);
      if (j == kmax) grad += inv_term;
      if (dbg_grad) dbg_grad[(int64_t)p * d + j] = grad;
      float m = sp.beta1 * Mt[at] + sp.omb1 * grad;
      float v = sp.beta2 * Vt[at] + sp.omb2 * grad * grad;
      float mhat = m / sp.bc1;
      float vhat = v / sp.bc2;
      float zn = z - sp.lr * mhat / (sqrtf(vhat) + sp.eps);
      Mt[at] = m;
      Vt[at] = v;
      Zt[at] = zn;
      moved |= (rintf(zn) != rintf(z));
    }
  }
  if (moved) changed[p] = 1;
}

// One warp per start: g = B round(z) exactly in int32, tests, append.
__global__ void collect_kernel(const int32_t* __restrict__ B, const float* __restrict__ Zt,
                               const int32_t* __restrict__ span, uint8_t* __restrict__ changed,
                               int n, int d, int P, int8_t* __restrict__ cand, int ldc,
                               int64_t cap, unsigned long long* __restrict__ count,
                               int32_t* __restrict__ flags) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= P) return;
  int p = warp;
  if (!changed[p]) return;
  __syncwarp();
  if (lane == 0) changed[p] = 0;
  // per-lane rows i = lane, lane + 32, ...
  bool valid = true, nonzero = false;
  int first_i = 1 << 30, first_sign = 0;
  bool range_bad = false;
  for (int i = lane; i < n; i += 32) {
    int acc = 0;
    for (int j = 0; j < d; ++j) {
      float zr = rintf(Zt[(int64_t)j * P + p]);
      if (fabsf(zr) > 1048576.f) { range_bad = true; zr = 0.f; }
      acc += B[(int64_t)i * d + j] * (int)zr;
    }
    if (acc != 0) {
      nonzero = true;
      if (i < first_i) { first_i = i; first_sign = acc > 0 ? 1 : -1; }
    }
    if (abs(acc) > span[i]) valid = false;
  }
  valid = __all_sync(0xffffffffu, valid);
  nonzero = __any_sync(0xffffffffu, nonzero);
  range_bad = __any_sync(0xffffffffu, range_bad);
  if (range_bad) {
    if (lane == 0) atomicOr(flags, 4);
    return;
  }
  // canonical sign: sign of the first nonzero entry
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    int oi = __shfl_xor_sync(0xffffffffu, first_i, off);
    int os = __shfl_xor_sync(0xffffffffu, first_sign, off);
    if (oi < first_i) { first_i = oi; first_sign = os; }
  }
  if (!valid || !nonzero) return;
  unsigned long long slot = 0;
  if (lane == 0) slot = atomicAdd(count, 1ull);
  slot = __shfl_sync(0xffffffffu, slot, 0);
  if ((int64_t)slot >= cap) {
    if (lane == 0) atomicOr(flags, 1);
    return;
  }
  int8_t* row = cand + (int64_t)slot * ldc;
  for (int i = lane; i < ldc; i += 32) {
    int v = 0;
    if (i < n) {
      for (int j = 0; j < d; ++j) v += B[(int64_t)i * d + j] * (int)rintf(Zt[(int64_t)j * P + p]);
      v *= first_sign;
    }
    row[i] = (int8_t)v;
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
  s.take<float>((size_t)n * d);                // Bf
  for (int k = 0; k < 3; ++k) s.take<float>((size_t)d * P);  // Zt, Mt, Vt (carved separately)
  s.take<int8_t>((size_t)n * P);               // S
  s.take<float>((size_t)ceil_div(n, kRowBlock) * P);  // l1 partials
  s.take<uint8_t>((size_t)P);                  // changed
  return s.bytes();
}

int extract_fp32(const mape_extract_args* a, cudaStream_t st) {
  const int n = a->n, d = a->d, P = a->P;
  Carver cv(a->workspace, a->workspace_bytes);
  float* Bf = cv.take<float>((size_t)n * d);
  float* Zt = cv.take<float>((size_t)d * P);
  float* Mt = cv.take<float>((size_t)d * P);
  float* Vt = cv.take<float>((size_t)d * P);
  int8_t* S = cv.take<int8_t>((size_t)n * P);
  int nblk = (int)ceil_div(n, kRowBlock);
  float* l1p = cv.take<float>((size_t)nblk * P);
  uint8_t* changed = cv.take<uint8_t>((size_t)P);
  if (!cv.ok) return MAPE_ERR_CAPACITY;

  std::vector<float2> bc;
  adam_bias_table(a, bc);

  mape_detail::launch(to_float_kernel, (unsigned)ceil_div((int64_t)n * d, 256), 256, 0, st, a->B, Bf, (int64_t)n * d);
  dim3 tb(32, 8);
  mape_detail::launch(transpose_kernel, dim3((unsigned)ceil_div(d, 32), (unsigned)ceil_div(P, 32)), tb, 0, st, a->Z, Zt, P, d);
  mape_detail::launch(transpose_kernel, dim3((unsigned)ceil_div(d, 32), (unsigned)ceil_div(P, 32)), tb, 0, st, a->M, Mt, P, d);
  mape_detail::launch(transpose_kernel, dim3((unsigned)ceil_div(d, 32), (unsigned)ceil_div(P, 32)), tb, 0, st, a->V, Vt, P, d);
  mape_detail::launch(fill_u8_kernel, (unsigned)ceil_div(P, 256), 256, 0, st, changed, 1, P);
  MAPE_LAUNCH_CHECK();

  dim3 fgrid((unsigned)ceil_div(P, kThreads), (unsigned)nblk);
  unsigned bgrid = (unsigned)ceil_div(P, kThreads);
  unsigned cgrid = (unsigned)ceil_div((int64_t)P * 32, 256);
  for (int s = 0; s < a->T; ++s) {
    const bool first = (s == 0);
    StepParams sp{a->lambda1, a->lambda2, a->lr, (float)a->beta1, (float)a->beta2, (float)(1.0 - a->beta1),
                  (float)(1.0 - a->beta2), a->eps, bc[s].x, bc[s].y};
    mape_detail::launch(forward_sign_kernel, fgrid, kThreads, 0, st, Bf, Zt, S, first && a->dbg_phi ? l1p : nullptr, n, d, P);
    mape_detail::launch(backward_adam_kernel, bgrid, kThreads, 0, st, Bf, S, Zt, Mt, Vt, changed, sp, n, d, P, l1p, nblk,
                                                     first ? a->dbg_phi : nullptr,
                                                     first ? a->dbg_grad : nullptr);
    int t = a->t0 + s + 1;
    if (t % a->period == 0)
      mape_detail::launch(collect_kernel, cgrid, 256, 0, st, a->B, Zt, a->span, changed, n, d, P, a->cand, a->ldc,
                                            a->cand_cap, a->cand_count, a->flags);
    MAPE_LAUNCH_CHECK();
  }
  mape_detail::launch(transpose_kernel, dim3((unsigned)ceil_div(P, 32), (unsigned)ceil_div(d, 32)), tb, 0, st, Zt, a->Z, d, P);
  mape_detail::launch(transpose_kernel, dim3((unsigned)ceil_div(P, 32), (unsigned)ceil_div(d, 32)), tb, 0, st, Mt, a->M, d, P);
  mape_detail::launch(transpose_kernel, dim3((unsigned)ceil_div(P, 32), (unsigned)ceil_div(d, 32)), tb, 0, st, Vt, a->V, d, P);
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
