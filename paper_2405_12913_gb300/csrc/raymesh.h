// The ray-mesh kick operator (raymesh.cu): the context's hook into it.
#pragma once

#include <cuda_runtime.h>

#include "common.h"

namespace hrt {

// One KDK ray step over [chi_from, chi_to] whose two half kicks come from ray meshes (hrt_raymesh_ray_step);
// grad_z is read only through a tiled light cone (g.n_replicas > 0); maps == nullptr skips the readout,
// accumulate != 0 adds weight times the observables.
hrt_status raymesh_step(hrt_raymesh* rm, const hrt_rays& rays, const float* grad_x, const float* grad_y,
                        const float* grad_z, const hrt_ray_geom& g, double chi_from, double chi_to, double a_ref, double omega_m,
                        float* maps, int accumulate, float weight, cudaStream_t s);

// The configuration a workspace was created with.
const hrt_raymesh_config& raymesh_config_of(const hrt_raymesh* rm);

}  // namespace hrt
