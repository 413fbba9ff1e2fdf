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

// Allocation-failure injection for host-side fault tests: HRT_FAIL_ALLOC_AT=k in the environment, or
// hrt_inject_alloc_failure(k), makes the k-th device allocation (1-based, counted from process start or from
// that call) report out-of-memory.
bool inject_alloc_failure();
// Resets the allocation count and makes the k-th device allocation from now fail (0: none); hrt_inject_alloc_failure.
void set_alloc_failure(int64_t k);

// cudaMallocAsync with the fault-injection hook; bytes == 0 gives nullptr.
hrt_status device_alloc(void** p, size_t bytes, cudaStream_t stream, const char* what);

// Waits for the work queued on s, for at most the process-wide limit set by hrt_set_host_wait_limit (no limit
// by default): HRT_ERR_TIMEOUT when it expires (the queued work keeps running), HRT_ERR_CUDA on a CUDA error.
hrt_status wait_stream(cudaStream_t s, const char* what);

// ORs 1 into *flag (device) if any of the n values at p (device) is a NaN or an infinity.
hrt_status launch_nonfinite_scan(const float* p, int64_t n, int* flag, cudaStream_t s);
hrt_status launch_nonfinite_scan(const double* p, int64_t n, int* flag, cudaStream_t s);

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
