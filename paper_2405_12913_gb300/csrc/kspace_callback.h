// Caller information of the k-space load callback (kspace_callback.cu), kept in device memory by the PM object.
#pragma once

namespace hrt {

struct KspaceCallbackInfo {
  const void* rho_hat;        // density half spectrum [n][n][n/2+1] complex64
  const float* wx;            // per-axis filter factors: [n], [n], [n/2+1]
  const float* wy;
  const float* wz;
  const float* g;             // learned correction table or nullptr
  int g_nk;
  float g_inv_dk;             // (g_nk - 1) / g_kmax
  int n, nzc, log2n, n_comp;  // mesh side (power of two), n/2 + 1, log2(n), spectra in the batch
  unsigned elems;             // n * n * nzc (< 2^31)
  unsigned long long magic;   // ceil(2^42 / nzc)
  float kf, scale;            // 2 pi / box, -pref / n^3
};

}  // namespace hrt
