// Internal helpers of the HRT library: status plumbing, error messages, launch checks.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "../../include/hrt.h"

namespace hrt {

// Records a printf-style message in the calling thread's error buffer and returns the status.
hrt_status fail(hrt_status s, const char* fmt, ...);

// Maps a CUDA runtime error to HRT_ERR_CUDA / HRT_ERR_OOM with a message; HRT_OK on success.
hrt_status cuda_status(cudaError_t e, const char* what);

// Environment-controlled allocation-failure injection for host-side fault tests: HRT_FAIL_ALLOC_AT=k makes
// the k-th device allocation of the process (1-based) report out-of-memory.
bool inject_alloc_failure();

// cudaMallocAsync with the fault-injection hook; bytes == 0 gives nullptr.
hrt_status device_alloc(void** p, size_t bytes, cudaStream_t stream, const char* what);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline unsigned blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

}  // namespace hrt

#define HRT_TRY(expr)                      \
  do {                                     \
    hrt_status _s = (expr);                \
    if (_s != HRT_OK) return _s;           \
  } while (0)

#define HRT_CUDA(expr) HRT_TRY(::hrt::cuda_status((expr), #expr))

#define HRT_LAUNCHED(name) HRT_TRY(::hrt::cuda_status(cudaGetLastError(), name))
