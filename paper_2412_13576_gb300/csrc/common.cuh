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
