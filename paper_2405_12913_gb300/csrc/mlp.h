// Launch wrappers of the learned-correction kernels (mlp_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.h"

namespace hrt {

constexpr int kMlpParams = 9473;  // W1 64x16 (3 used), b1 64, W2 64x64, b2 64, W3 64x64, b3 64, W4 64, b4 1

hrt_status launch_mlp_forward(const float* x, int rows, const void* wb, const float* wf, float* y, cudaStream_t s);
hrt_status launch_mlp_backward(const float* x, int rows, const void* wb, const float* wf, const float* gbar,
                               float* grad, cudaStream_t s);
hrt_status launch_adam(float* wf, void* wb, const float* grad, float* m, float* v, double lr, double b1, double b2,
                       double eps, int step, cudaStream_t s);
hrt_status launch_to_bf16(const float* wf, void* wb, cudaStream_t s);
hrt_status launch_correction_inputs(float* x, int rows, double dx, double a, double ln_n, cudaStream_t s);

// The correction table of a context: kCorrectionRows samples of g over |k| in [0, kCorrectionKmaxCell / cell],
// the corner of the Brillouin zone (sqrt(3) pi / cell) with a small margin.
constexpr int kCorrectionRows = 512;
constexpr double kCorrectionKmaxCell = 1.7320508075688772 * 3.141592653589793 * 1.0001;
hrt_status launch_kspace_table_adjoint(const void* gbar_hat, int n_comp, const void* rho_hat, int64_t n, double box,
                                       double pref, const float* tab, int g_nk, double g_kmax, float* table_bar,
                                       cudaStream_t s);

}  // namespace hrt
