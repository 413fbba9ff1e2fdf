// hrt_kspace_gradient_noalloc: the fused k-space kernel without any device allocation.
//
// The ordinary entry point hrt_kspace_gradient uploads its per-axis filter tables into a small device buffer
// that it allocates and frees on every call.  Some callers cannot allow that: an application that owns every
// byte of device memory through its own pool and forbids allocation once it is running, or a pipeline that
// must not allocate (or risk an allocation failure) in the middle of a time step.  For them this variant keeps
// the tables in one fixed array in device global memory, declared at file scope below.  Its size is fixed at
// build time (kNoallocMaxMesh), and every GPU that loads the library holds it until the process exits.
//
// In host code the name g_noalloc_tables is only a host-side stand-in for the device array, never a device
// address; the device address is looked up once per device with cudaGetSymbolAddress and passed to the kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "common.h"
#include "mesh_kernels.h"

namespace hrt {

// Largest mesh side the fixed array can hold: two filter sets of (n + n/2 + 1) floats each.
constexpr int64_t kNoallocMaxMesh = 2048;
constexpr int64_t kNoallocSetFloats = kNoallocMaxMesh + kNoallocMaxMesh / 2 + 1;

static __device__ __align__(256) float g_noalloc_tables[2 * kNoallocSetFloats];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_table_addr[kMaxDevices] = {};

// Device address of the fixed table array on the current device, looked up on the first call per device.
hrt_status table_address(float** out) {
  int dev = -1;
  HRT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(HRT_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_table_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_tables);
    if (e != cudaSuccess || p == nullptr) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                             "cudaGetSymbolAddress(g_noalloc_tables)");
    g_table_addr[dev] = static_cast<float*>(p);
  }
  *out = g_table_addr[dev];
  return HRT_OK;
}

}  // namespace
}  // namespace hrt

using namespace hrt;

extern "C" hrt_status hrt_kspace_gradient_noalloc(const void* rho_hat, int64_t n, double box, double pref,
                                                  const hrt_filter* f, int32_t n_out, void* out, const hrt_filter* f2,
                                                  int32_t n_second, void* second, void* stream) {
  if (n > kNoallocMaxMesh)
    return fail(HRT_ERR_INVALID_ARG, "hrt_kspace_gradient_noalloc: mesh %lld exceeds the fixed table limit %lld",
                static_cast<long long>(n), static_cast<long long>(kNoallocMaxMesh));
  // the same argument checks as hrt_kspace_gradient
  if (n < 2 || n % 2 != 0) return fail(HRT_ERR_INVALID_ARG, "mesh size %lld must be even", static_cast<long long>(n));
  if (!(box > 0.0) || !std::isfinite(box)) return fail(HRT_ERR_INVALID_ARG, "box must be positive and finite");
  if (!std::isfinite(pref)) return fail(HRT_ERR_INVALID_ARG, "non-finite prefactor");
  if (!rho_hat || !out || n_out < 1 || n_out > 3) return fail(HRT_ERR_INVALID_ARG, "bad primary output");
  if (second && (n_second < 1 || n_second > 3)) return fail(HRT_ERR_INVALID_ARG, "bad second output count");
  for (const hrt_filter* g : {f, second ? f2 : f}) {
    if (!g) return fail(HRT_ERR_INVALID_ARG, "filter is NULL");
    if (!std::isfinite(g->deconv_p) || !(g->smooth >= 0.0) || !std::isfinite(g->smooth))
      return fail(HRT_ERR_INVALID_ARG, "bad filter");
    if (g->g_table && (g->g_nk < 2 || !(g->g_kmax > 0.0))) return fail(HRT_ERR_INVALID_ARG, "bad learned table");
  }
  cudaStream_t s = as_stream(stream);
  // The tables are staged from host memory at call time; a captured graph would replay a copy from a host
  // buffer that no longer exists, so calls during stream capture are refused.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  HRT_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(HRT_ERR_STATE, "hrt_kspace_gradient_noalloc cannot be called while the stream is being captured");
  float* tables = nullptr;
  HRT_TRY(table_address(&tables));
  // Host tables, then one copy into the fixed array on the caller's stream.  The copy reads pageable host
  // memory, which the runtime consumes before cudaMemcpyAsync returns, so the vector may go out of scope.
  std::vector<float> host, wxy, wz;
  filter_tables(n, box, *f, wxy, wz);
  host.insert(host.end(), wxy.begin(), wxy.end());
  host.insert(host.end(), wz.begin(), wz.end());
  const size_t set_floats = host.size();
  if (second) {
    filter_tables(n, box, *f2, wxy, wz);
    host.insert(host.end(), wxy.begin(), wxy.end());
    host.insert(host.end(), wz.begin(), wz.end());
  }
  HRT_CUDA(cudaMemcpyAsync(tables, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  return launch_kspace(rho_hat, n, box, pref, tables, f, n_out, out, second ? tables + set_floats : nullptr, f2,
                       second ? n_second : 0, second, s);
}
