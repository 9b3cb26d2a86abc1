// Shared helpers of the CUDA path (not used by the oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/mape.h"

#define MAPE_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) {                                  \
      mape_detail::record_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return MAPE_ERR_CUDA;                                   \
    }                                                         \
  } while (0)

#define MAPE_LAUNCH_CHECK() MAPE_CUDA_TRY(cudaGetLastError())

namespace mape_detail {

void record_cuda_error(cudaError_t e, const char* what, const char* file, int line);
// Records a plain message (an argument error worth explaining) in the same place.
void record_message(const char* what);

// Lets the kernel `func` take as much dynamic shared memory as the device
// allows (its static shared memory deducted) and returns that amount in
// *limit.  Every caller sets the same value, so that threads launching the
// same kernel with different amounts (handles of a server) never lower the
// limit under one another's launch.
int allow_max_dynamic_smem(const void* func, size_t* limit);

// Forgets the autotuned lane counts of Algorithm 1's scoring pass.
void augment_tune_clear();

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

// Carves consecutive 256-byte aligned pieces out of a caller workspace.
struct Carver {
  char* base;
  size_t cap;
  size_t used = 0;
  bool ok = true;
  Carver(void* p, size_t c) : base(static_cast<char*>(p)), cap(c) {}
  template <typename T>
  T* take(size_t count) {
    size_t off = align_up(used, 256);
    size_t bytes = count * sizeof(T);
    if (off + bytes > cap || (base == nullptr && bytes > 0)) {
      ok = false;
      used = off + bytes;
      return nullptr;
    }
    used = off + bytes;
    return reinterpret_cast<T*>(base + off);
  }
};

// Same arithmetic as Carver, without memory: the workspace size query.
struct Sizer {
  size_t used = 0;
  template <typename T>
  void take(size_t count) { used = align_up(used, 256) + count * sizeof(T); }
  size_t bytes() const { return align_up(used, 256) + 256; }
};

// Default candidate-buffer rows of a handle: one row per start and
// collection step (`collections` = T / period), at most 2^23 rows and at most
// 2 GiB per buffer (a handle holds two); the extraction runs in chunks of
// steps that fit.
inline int64_t default_cand_capacity(int64_t P, int64_t collections, int64_t ldg) {
  int64_t cap = P * (collections > 0 ? collections : 1) + P;
  cap = cap < ((int64_t)1 << 23) ? cap : ((int64_t)1 << 23);
  const int64_t by_bytes = ((int64_t)1 << 31) / (ldg > 0 ? ldg : 16);
  cap = cap < by_bytes ? cap : by_bytes;
  return cap > P + 1 ? cap : P + 1;
}

}  // namespace mape_detail

// Device-side integer helpers ------------------------------------------------

__device__ __forceinline__ int mape_sign_f(float y) { return (y > 0.f) - (y < 0.f); }

namespace mape_detail {
// Every kernel of the library is launched through launch(), which counts the
// launches (mape_launch_count).
void note_launch();
template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  kernel<<<grid, block, smem, st>>>(args...);
  note_launch();
}
}  // namespace mape_detail
