// Readout of the lensing observables from the distortion matrix A (Eqs. "obs_first_set" / "obs_second_set"),
// shared by the ray kernels: A = [[x, y], [z, w]] row-major.
#pragma once

#include <cuda_runtime.h>

namespace hrt {

__device__ __forceinline__ void readout(const float4 A, float& kappa, float& g1, float& g2, float& om) {
  float c1 = 0.5f * (A.x + A.w), c2 = 0.5f * (A.y - A.z), c3 = 0.5f * (A.w - A.x), c4 = 0.5f * (A.y + A.z);
  kappa = 1.f - c1;
  om = c2 / c1;
  g1 = c3 + c4 * om;
  g2 = -c4 + c3 * om;
}

}  // namespace hrt
