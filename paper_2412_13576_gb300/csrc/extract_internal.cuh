// Internal entry points shared by the extraction translation units.
#pragma once
#include <vector>
#include "common.cuh"

namespace mape_detail {
// Adam bias corrections (1 - beta1^t, 1 - beta2^t) for t = t0+1 .. t0+T,
// computed in double on the host.
void adam_bias_table(const mape_extract_args* a, std::vector<float2>& out);

size_t extract_fp32_workspace(int32_t n, int32_t d, int32_t P);
int extract_fp32(const mape_extract_args* a, cudaStream_t st);

size_t extract_tc_workspace(int32_t n, int32_t d, int32_t P, int32_t precision);
bool extract_tc_supported(int32_t n, int32_t d, int32_t precision);
int extract_tc(const mape_extract_args* a, cudaStream_t st);

// Batches of calls (same T, t0, period, precision) on the resident kernel:
// prepare uploads and synchronises; enqueue only launches kernels.
struct TcBatch;
bool extract_tc_fits(const mape_extract_args* a, bool id);
size_t extract_tc_batch_workspace(const mape_extract_args* const* items, int count);
int extract_tc_batch_prepare(const mape_extract_args* const* items, const bool* ids, int count, void* ws,
                             size_t ws_bytes, cudaStream_t st, TcBatch** out);
int extract_tc_batch_enqueue(const TcBatch* plan, cudaStream_t st);
void extract_tc_batch_free(TcBatch* plan);

bool extract_sparse_supported(int32_t n, int32_t d);
size_t extract_sparse_workspace(int32_t n, int32_t d, int32_t P);
int extract_sparse(const mape_extract_args* a, cudaStream_t st);

bool extract_stream_supported(int32_t n, int32_t d);
size_t extract_stream_workspace(int32_t n, int32_t d, int32_t P);
// forward pass of the streamed path: the tensor-core forward, or the CUDA-core
// sparse forward (SHAPE unless B is identity-topped, z is carried in full
// and Bm has density at most 1/16)
constexpr int kFwdDense = 1, kFwdSparse = 2;
int extract_stream(const mape_extract_args* a, cudaStream_t st, int fwd_mode);
// the same with the forward and gradient N-block widths chosen (64..256, multiples of 64)
int extract_stream_widths(const mape_extract_args* a, cudaStream_t st, int wF, int wG, int fwd_mode);

// Batches of calls on the streamed kernels: three launches per step for all
// calls of one basis kind.
struct StBatch;
size_t extract_stream_batch_workspace(const mape_extract_args* const* items, int count);
int extract_stream_batch_prepare(const mape_extract_args* const* items, const bool* ids, int count, void* ws,
                                 size_t ws_bytes, cudaStream_t st, StBatch** out);
int extract_stream_batch_enqueue(const StBatch* plan, cudaStream_t st);
void extract_stream_batch_free(StBatch* plan);
// identity-topped test of every call's B (one launch each, one synchronisation)
int identity_tops(const mape_extract_args* const* items, int count, int32_t* dflags, cudaStream_t st,
                  std::vector<bool>& ids);

// Optional CUDA-event timing of the extraction kernels' launches
// (mape_launch_timing): when on, timed_launch records an event pair around
// the launch on its stream; the pairs are read at mape_launch_timing_read.
bool launch_timing_on();
void timed_record(int kind, cudaEvent_t start, cudaEvent_t stop);
template <typename F>
inline void timed_launch(int kind, cudaStream_t st, F&& f) {
  if (!launch_timing_on()) {
    f();
    return;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    f();
    return;
  }
  cudaEventRecord(a, st);
  f();
  cudaEventRecord(b, st);
  timed_record(kind, a, b);
}
}  // namespace mape_detail
