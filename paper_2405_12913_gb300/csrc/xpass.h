// The x-pass of the split Poisson solve (xpass_kernels.cu): forward x-FFT, fused k-space step and inverse x-FFTs
// of the gradient spectra on the [x][ky][kz] output of batched 2D (y, z) R2C plans.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "common.h"

namespace hrt {

// One filter set: per-axis factor tables wxy [n] (signed-frequency order) and wz [n/2 + 1], the optional learned
// factor g(|k|) (g_nk entries over [0, (g_nk - 1) / g_inv_dk]) and n_out gradient spectra (x, y[, z]) laid out
// [component][x][ky][xpass_row(n)].
struct XpassSet {
  const float* wxy;
  const float* wz;
  const float* g;
  int g_nk;
  float g_inv_dk;
  int n_out;
  float2* out;
};

// Mesh sides the x-pass supports (n = 32 R1 with R1 in {8, 16, 32}).
bool xpass_supported(int64_t n);
// Length of a kz row of the split layout (the half spectrum's n/2 + 1).
int64_t xpass_row(int64_t n);
// Twiddle table of the x-FFT for side n: [R1][32] forward factors exp(-2 pi i l k1 / n), then [32][32] inverse
// factors exp(+2 pi i n1 (lane mod R1) / n); FP64 on the host, rounded to float.
void xpass_twiddles(int64_t n, std::vector<float2>& tw);
// Bit the x-pass sets in its error word when a wait for a tile's copy timed out (the kernel then stops early).
constexpr int kXpassTimeout = 1;
// Dynamic shared memory of the x-pass for side n (three 64 KB tiles, twiddle and filter tables, barriers).
size_t xpass_smem_bytes(int64_t n);
// in: the (y, z)-transformed density [x][ky][xpass_row(n)] (16-byte aligned, as are the outputs); tw: device copy
// of xpass_twiddles(n); err: device error word (kXpassTimeout is OR-ed into it).  Set a has 2 or 3 outputs, set
// b none (n_out 0), 2 or 3.  clear (or nullptr): a buffer of clear_floats floats (16-byte aligned, a multiple of
// 4) that nothing reads or writes during the pass, set to zero by it.
hrt_status launch_xpass(const void* in, int64_t n, double box, double pref, const float2* tw, const XpassSet& a,
                        const XpassSet& b, int* err, cudaStream_t s, float* clear = nullptr,
                        int64_t clear_floats = 0);

}  // namespace hrt
