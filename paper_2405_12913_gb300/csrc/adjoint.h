// Launch wrappers of the adjoint kernels (adjoint_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.h"
#include "mesh_kernels.h"

namespace hrt {

hrt_status launch_deposit_adjoint(const float* rho_bar, const float* disp, int64_t n_side, int64_t n, double box,
                                  float* disp_bar, cudaStream_t s);
hrt_status launch_kick_drift_adjoint(const float* grad, int64_t n, double box, int64_t n_side, const float* disp,
                                     const float* mom, double kick, double drift, const float* rho_bar,
                                     float* disp_bar, float* mom_bar, float* grad_bar, double* coef_bar,
                                     cudaStream_t s);
hrt_status launch_kspace_adjoint(const void* in, int n_in, int64_t n, double box, double pref, const float* tab,
                                 const hrt_filter* f, void* out, bool accumulate, cudaStream_t s);
// gz, gbz: the third field and its cotangent, read and written only for a tiled step (p.tiled).
hrt_status launch_ray_step_adjoint(const hrt_rays& rays, const float* gx, const float* gy, const RayStepParams& p,
                                   const hrt_rays& bar, float* gbx, float* gby, double* node_bar, double* drift_bar,
                                   cudaStream_t s, const float* gz = nullptr, float* gbz = nullptr);
hrt_status launch_power_adjoint_weight(void* spec, int64_t m, double dtheta, int nbins, double ell_min, double ell_max,
                                       const double* wbin_dev, cudaStream_t s);
hrt_status launch_ic_adjoint(const void* in, const void* w_hat, int64_t n, double box, const float* table, void* out,
                             double* table_bar, cudaStream_t s);
hrt_status launch_lpt2_kspace_adjoint(const void* in, int64_t n, double box, void* out, cudaStream_t s);
hrt_status launch_lpt2_source_adjoint(float* h, const float* sb, int64_t m, cudaStream_t s);
hrt_status launch_ic_hessian_adjoint(const void* in, const void* w_hat, int64_t n, double box, const float* table,
                                     int set, void* out, double* table_bar, cudaStream_t s);
hrt_status launch_axpy(const float* x, float* y, double alpha, int64_t m, cudaStream_t s);
hrt_status launch_dot(const float* a, const float* b, int64_t m, double* out, cudaStream_t s);

}  // namespace hrt
