// Load callback of the batched complex-to-real FFT that turns the density spectrum into the gradient spectra on
// the fly (the fused k-space step of the Poisson solve, Sec. 2 Poisson equation and Sec. 5.2 deconvolution).
//
// Compiled separately to LTO IR (compute_100, C++ linkage: the form cuFFT's JIT link resolves by name) and linked
// into cuFFT's own kernels at plan time (cufftXtSetJITCallback).  cuFFT
// calls it exactly once per input element of a batch of n_comp half spectra; element `offset` of batch j gets
//   i k_j * scale / k^2 * Wx[ix] Wy[iy] Wz[kz] * g(|k|) * rho_hat[offset - j * elems]
// (0 at k = 0 and on the j-Nyquist plane), the same value the stand-alone k-space kernel writes.  The batch
// input buffer handed to cuFFT is only scratch: the density spectrum is read through the caller info, so cuFFT
// may overwrite its input freely.
#include <cuComplex.h>
#include <cufftXt.h>

#include "kspace_callback.h"

__device__ cufftComplex hrt_kspace_load(void* data_in, unsigned long long offset, void* caller_info,
                                                   void* shared_ptr) {
  (void)data_in;
  (void)shared_ptr;
  const hrt::KspaceCallbackInfo* ci = static_cast<const hrt::KspaceCallbackInfo*>(caller_info);
  unsigned local = static_cast<unsigned>(offset);
  int comp = 0;
  while (comp + 1 < ci->n_comp && local >= ci->elems) {  // at most two subtractions (batch <= 3)
    local -= ci->elems;
    ++comp;
  }
  // row = local / nzc exactly: local < 2^31 and nzc < 2048, magic = ceil(2^42 / nzc)
  const unsigned row = static_cast<unsigned>((static_cast<unsigned long long>(local) * ci->magic) >> 42);
  const int iz = static_cast<int>(local - row * static_cast<unsigned>(ci->nzc));
  const int ix = static_cast<int>(row >> ci->log2n);
  const int iy = static_cast<int>(row & static_cast<unsigned>(ci->n - 1));
  const int n = ci->n, half = n >> 1;
  const int nx = ix < half ? ix : ix - n;
  const int ny = iy < half ? iy : iy - n;
  const float kx = ci->kf * nx, ky = ci->kf * ny, kz = ci->kf * iz;
  const float k2 = kx * kx + ky * ky + kz * kz;
  float d;
  if (comp == 0) d = (nx == -half) ? 0.f : kx;
  else if (comp == 1) d = (ny == -half) ? 0.f : ky;
  else d = (iz == half) ? 0.f : kz;
  if (k2 == 0.f || d == 0.f) return make_cuComplex(0.f, 0.f);
  float c = ci->scale / k2 * __ldg(ci->wx + ix) * __ldg(ci->wy + iy) * __ldg(ci->wz + iz) * d;
  if (ci->g != nullptr) {
    const float t = sqrtf(k2) * ci->g_inv_dk;
    if (t < static_cast<float>(ci->g_nk - 1)) {
      const int i = static_cast<int>(t);
      const float w = t - static_cast<float>(i);
      c *= __ldg(ci->g + i) * (1.f - w) + __ldg(ci->g + i + 1) * w;
    }
  }
  const float2 v = __ldg(reinterpret_cast<const float2*>(ci->rho_hat) + local);
  return make_cuComplex(-c * v.y, c * v.x);  // i * c * v
}
