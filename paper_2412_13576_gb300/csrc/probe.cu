// Measurement of the tensor-core instruction cost on this GPU, the basis of
// the MMA-count choices of the extraction kernels (few, wide MMAs; the
// transposed forward product of the resident kernel): one thread issues a
// chain of tcgen05.mma (cta_group::1) into one or two TMEM accumulators and
// the SM clock is read around the chain, from the first issue to the
// completion of the last (tcgen05.commit on an mbarrier, waited with a bound).
// The operands are zero tiles in shared memory (K-major, no swizzle); the
// values do not change the cost.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace {
using namespace mape_tc;

// out[0]: cycles from the first issue to the last issue, out[1]: to the
// completion of the chain; out[2] = 1 when a wait gave up
__global__ void mma_issue_probe_kernel(int kind, int M, int N, int nacc, int chain, long long* out) {
  __shared__ __align__(1024) uint8_t sA[128 * 32];
  __shared__ __align__(1024) uint8_t sB[256 * 32];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_tmem;
  for (int i = threadIdx.x; i < 128 * 32; i += blockDim.x) sA[i] = 0;
  for (int i = threadIdx.x; i < 256 * 32; i += blockDim.x) sB[i] = 0;
  if (threadIdx.x == 0) mbar_init(smem_u32(&bar), 1);
  if (threadIdx.x < 32) tmem_alloc(smem_u32(&s_tmem), 512);
  mbar_init_fence();
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  if (threadIdx.x == 0) {
    // 8-row groups 256 bytes apart, the two K-adjacent core matrices 128 apart
    const uint64_t a = make_desc(smem_u32(sA), 128, 256);
    const uint64_t b = make_desc(smem_u32(sB), 128, 256);
    const uint32_t id = kind ? idesc_e4m3(M, N) : idesc_bf16(M, N);
    for (int i = 0; i < 8; ++i) {  // warm-up
      if (kind) mma_e4m3(tmem, a, b, id, i > 0);
      else mma_bf16(tmem, a, b, id, i > 0);
    }
    mma_commit(smem_u32(&bar));
    bool ok = mbar_wait_bounded(smem_u32(&bar), 0);
    const long long t0 = clock64();
    for (int i = 0; i < chain; ++i) {
      const uint32_t d = tmem + (uint32_t)((i % nacc) * N);
      if (kind) mma_e4m3(d, a, b, id, 1u);
      else mma_bf16(d, a, b, id, 1u);
    }
    mma_commit(smem_u32(&bar));
    const long long t1 = clock64();
    ok = mbar_wait_bounded(smem_u32(&bar), 1) && ok;
    const long long t2 = clock64();
    out[0] = t1 - t0;
    out[1] = t2 - t0;
    out[2] = ok ? 0 : 1;
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace

extern "C" int mape_mma_issue_probe(int32_t kind, int32_t M, int32_t N, int32_t accumulators, int32_t chain,
                                    double* issue_cycles, double* total_cycles) {
  using namespace mape_detail;
  if (!issue_cycles || !total_cycles || (kind != 0 && kind != 1) || (M != 64 && M != 128) || chain <= 0 ||
      chain > 4096 || accumulators < 1 || accumulators > 2)
    return MAPE_ERR_INVALID_ARG;
  if (N < 16 || N > 256 || N % 16 != 0 || accumulators * N > 512) return MAPE_ERR_INVALID_ARG;
  long long* d_out = nullptr;
  MAPE_CUDA_TRY(cudaMalloc(&d_out, 3 * sizeof(long long)));
  launch(mma_issue_probe_kernel, 1, 128, 0, (cudaStream_t)0, (int)kind, (int)M, (int)N, (int)accumulators,
         (int)chain, d_out);
  long long h[3] = {0, 0, 0};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(h, d_out, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d_out);
  if (e != cudaSuccess) {
    record_cuda_error(e, "mape_mma_issue_probe", __FILE__, __LINE__);
    return MAPE_ERR_CUDA;
  }
  if (h[2]) return MAPE_ERR_TIMEOUT;
  *issue_cycles = (double)h[0] / chain;
  *total_cycles = (double)h[1] / chain;
  return MAPE_OK;
}
