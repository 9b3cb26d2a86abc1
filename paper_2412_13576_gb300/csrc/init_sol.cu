// Initial feasible solutions of model (1), Eq. (4) (§3.3): projected Adam on
// ||A x - b||_2^2 + lambda3 sum_i (x_i - floor x_i)(ceil x_i - x_i) over the
// box [l, u] from many starts at once; after every `period`-th step the
// rounded iterate (ties to even) is tested exactly (A round(x) = b in int64;
// the box holds by the projection) and, if it changed since the start's
// previous collection in this call, appended as a row of bytes round(x) - l.
//
// One warp per start, persistent over the T steps: the warp keeps its x in
// shared memory (the broadcast operand of both products), its lanes take the
// rows of A for r = A x - b and the coordinates for 2 A^T r, the gradient
// term of the integrality penalty, Adam and the projection.  A is held as
// FP32 in both orientations (A for the gradient, A^T for the residual, so
// that the lanes of a warp read consecutive words); in shared memory when it
// fits, else from global memory through L2.  The products are dense m x n
// CUDA-core work (m is small, a fifth of n in the workloads): FP32 SIMT, the
// precision of the paper's PyTorch version.
#include "common.cuh"

#include <cmath>
#include <vector>

namespace {

constexpr int kWarps = 4;
constexpr uint32_t kSmemLimit = 200 * 1024;

struct InitParams {
  int n, m, P, t0, T, period;
  const float* Af;    // [m x n]
  const float* At;    // [n x m]
  const int64_t* b;
  const int32_t* l;
  const int32_t* u;
  float* X;
  float* M;
  float* V;
  const float2* bias;  // (lr / (1 - beta1^t), 1 / sqrt(1 - beta2^t)) per step
  float lambda3, eps, beta1, beta2, omb1, omb2;
  uint8_t* sol;
  int lds;
  int64_t cap;
  unsigned long long* count;
  int32_t* flags;
  float* dbg_f;
  float* dbg_grad;
  int a_smem;  // 1: A and A^T are copied into shared memory
};

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(32 * kWarps) init_sol_kernel(InitParams p) {
  extern __shared__ __align__(16) float sm[];
  const int n = p.n, m = p.m;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* sAf = sm;
  float* sAt = sm + (p.a_smem ? (size_t)m * n : 0);
  float* base = sm + (p.a_smem ? 2 * (size_t)m * n : 0);
  float* xs = base + (size_t)warp * (n + m);
  float* rs = xs + n;
  if (p.a_smem) {
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
      sAf[e] = p.Af[e];
      sAt[e] = p.At[e];
    }
  }
  __syncthreads();
  const float* Af = p.a_smem ? sAf : p.Af;
  const float* At = p.a_smem ? sAt : p.At;
  const int64_t pg = (int64_t)blockIdx.x * kWarps + warp;
  if (pg >= p.P) return;  // warp-uniform; no block barrier follows
  float* X = p.X + pg * n;
  float* Mv = p.M + pg * n;
  float* Vv = p.V + pg * n;
  for (int j = lane; j < n; j += 32) xs[j] = fminf(fmaxf(X[j], (float)p.l[j]), (float)p.u[j]);
  __syncwarp();
  bool changed = true;  // the first collection of a call always counts
  for (int s = 0; s < p.T; ++s) {
    const int t = p.t0 + s + 1;
    // r = A x - b, one row per lane
    for (int i = lane; i < m; i += 32) {
      float acc = -(float)p.b[i];
      for (int j = 0; j < n; ++j) acc = fmaf(At[(size_t)j * m + i], xs[j], acc);
      rs[i] = acc;
    }
    __syncwarp();
    const bool dbg = s == 0 && (p.dbg_f || p.dbg_grad);
    float fr = 0.f;
    if (dbg && p.dbg_f)
      for (int i = lane; i < m; i += 32) fr += rs[i] * rs[i];
    const float2 ad = p.bias[s];
    bool moved = false;
    for (int j = lane; j < n; j += 32) {
      float g = 0.f;
      for (int i = 0; i < m; ++i) g = fmaf(Af[(size_t)i * n + j], rs[i], g);
      const float x = xs[j];
      const float fl = floorf(x);
      // ceil x + floor x = 2 floor x + [x not an integer]
      const float grad = 2.f * g + p.lambda3 * (2.f * fl + (x != fl ? 1.f : 0.f) - 2.f * x);
      if (dbg) {
        if (p.dbg_f) fr += p.lambda3 * (x - fl) * (ceilf(x) - x);
        if (p.dbg_grad) p.dbg_grad[pg * n + j] = grad;
      }
      const float mm = p.beta1 * Mv[j] + p.omb1 * grad;
      const float vv = p.beta2 * Vv[j] + p.omb2 * grad * grad;
      const float den = (vv > 0.f ? vv * rsqrtf(vv) : 0.f) * ad.y + p.eps;
      float xn = x - ad.x * __fdividef(mm, den);
      xn = fminf(fmaxf(xn, (float)p.l[j]), (float)p.u[j]);
      Mv[j] = mm;
      Vv[j] = vv;
      moved |= rintf(xn) != rintf(x);
      xs[j] = xn;
    }
    if (dbg && p.dbg_f) {
      fr = warp_sum_f(fr);
      if (lane == 0) p.dbg_f[pg] = fr;
    }
    changed |= __any_sync(0xffffffffu, moved);
    __syncwarp();
    if (t % p.period == 0) {
      if (changed) {
        // exact test of A round(x) = b in int64
        bool ok = true;
        for (int i = lane; i < m; i += 32) {
          long long acc = 0;
          for (int j = 0; j < n; ++j) acc += (long long)Af[(size_t)i * n + j] * (long long)rintf(xs[j]);
          ok &= acc == p.b[i];
        }
        ok = __all_sync(0xffffffffu, ok);
        long long slot = -1;
        if (ok && lane == 0) {
          const unsigned long long at = atomicAdd(p.count, 1ull);
          if ((int64_t)at < p.cap) slot = (long long)at;
          else atomicOr(p.flags, 1);
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= 0) {
          uint8_t* row = p.sol + slot * p.lds;
          for (int j = lane; j < p.lds; j += 32) row[j] = j < n ? (uint8_t)((int)rintf(xs[j]) - p.l[j]) : 0;
        }
      }
      changed = false;
    }
  }
  for (int j = lane; j < n; j += 32) X[j] = xs[j];
}

__global__ void init_operands_kernel(const int32_t* __restrict__ A, int m, int n, float* __restrict__ Af,
                                     float* __restrict__ At) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const float v = (float)A[e];
  Af[e] = v;
  At[(int64_t)j * m + i] = v;
}

}  // namespace

extern "C" size_t mape_initial_solutions_workspace_bytes(int32_t n, int32_t m, int32_t T) {
  if (n <= 0 || m <= 0 || T < 0) return 0;
  mape_detail::Sizer s;
  s.take<float>((size_t)m * n);
  s.take<float>((size_t)m * n);
  s.take<float2>((size_t)(T > 0 ? T : 1));
  return s.bytes();
}

extern "C" int mape_initial_solutions(const mape_init_args* a, void* stream) {
  using namespace mape_detail;
  if (!a) return MAPE_ERR_INVALID_ARG;
  const int n = a->n, m = a->m, P = a->P;
  if (n <= 0 || m <= 0 || P < 0 || a->T < 0 || a->t0 < 0 || a->period <= 0) return MAPE_ERR_INVALID_ARG;
  if (!a->A || !a->b || !a->l || !a->u || !a->sol_count || !a->flags) return MAPE_ERR_INVALID_ARG;
  if (P > 0 && (!a->X || !a->M || !a->V)) return MAPE_ERR_INVALID_ARG;
  if (a->lds < n || a->sol_cap < 0 || (a->sol_cap > 0 && !a->sol)) return MAPE_ERR_INVALID_ARG;
  if (n > 48 * 1024) return MAPE_ERR_SHAPE;
  if (P == 0 || a->T == 0) return MAPE_OK;
  if (a->workspace_bytes < mape_initial_solutions_workspace_bytes(n, m, a->T)) return MAPE_ERR_CAPACITY;
  cudaStream_t st = as_stream(stream);
  Carver cv(a->workspace, a->workspace_bytes);
  float* Af = cv.take<float>((size_t)m * n);
  float* At = cv.take<float>((size_t)m * n);
  float2* bias = cv.take<float2>((size_t)a->T);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  std::vector<float2> bc((size_t)a->T);
  for (int s = 0; s < a->T; ++s) {
    const double t = (double)a->t0 + s + 1;
    const double bc1 = 1.0 - std::pow(a->beta1, t), bc2 = 1.0 - std::pow(a->beta2, t);
    bc[s] = make_float2((float)((double)a->lr / bc1), (float)(1.0 / std::sqrt(bc2)));
  }
  MAPE_CUDA_TRY(cudaMemcpyAsync(bias, bc.data(), sizeof(float2) * bc.size(), cudaMemcpyHostToDevice, st));
  launch(init_operands_kernel, (unsigned)ceil_div((int64_t)m * n, 256), 256, 0, st, a->A, m, n, Af, At);
  InitParams p{};
  p.n = n; p.m = m; p.P = P; p.t0 = a->t0; p.T = a->T; p.period = a->period;
  p.Af = Af; p.At = At; p.b = a->b; p.l = a->l; p.u = a->u; p.X = a->X; p.M = a->M; p.V = a->V; p.bias = bias;
  p.lambda3 = a->lambda3; p.eps = a->eps;
  p.beta1 = (float)a->beta1; p.beta2 = (float)a->beta2;
  p.omb1 = (float)(1.0 - a->beta1); p.omb2 = (float)(1.0 - a->beta2);
  p.sol = a->sol; p.lds = a->lds; p.cap = a->sol_cap; p.count = a->sol_count; p.flags = a->flags;
  p.dbg_f = a->dbg_f; p.dbg_grad = a->dbg_grad;
  const size_t per_warp = (size_t)kWarps * (n + m) * sizeof(float);
  const size_t with_a = 2 * (size_t)m * n * sizeof(float) + per_warp;
  p.a_smem = with_a <= kSmemLimit ? 1 : 0;
  const size_t smem = p.a_smem ? with_a : per_warp;
  if (smem > kSmemLimit) return MAPE_ERR_SHAPE;
  {
    size_t lim = 0;
    const int rc = allow_max_dynamic_smem((const void*)init_sol_kernel, &lim);
    if (rc != MAPE_OK) return rc;
    if ((size_t)smem > lim) return MAPE_ERR_SHAPE;
  }
  launch(init_sol_kernel, (unsigned)ceil_div(P, kWarps), 32 * kWarps, smem, st, p);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}
