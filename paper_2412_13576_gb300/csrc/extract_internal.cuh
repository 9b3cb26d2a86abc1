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

bool extract_stream_supported(int32_t n, int32_t d);
size_t extract_stream_workspace(int32_t n, int32_t d, int32_t P);
int extract_stream(const mape_extract_args* a, cudaStream_t st);
}  // namespace mape_detail
