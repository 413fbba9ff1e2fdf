// Learned force correction: a 3 -> 64 -> 64 -> 64 -> 1 multilayer perceptron g(|k| cell, a, ln N_mesh) that
// multiplies the Green's function of the ray gradient fields (the analogue of the paper's force-sharpening
// factor k/k^2 -> (k/k^2) g, Sec. 6.2), evaluated once per step on a 1D table of |k|.
//
// Forward: one warp per 16 table rows; BF16 weights and activations, FP32 accumulation on the tensor cores
// (mma.sync m16n8k16), SiLU hidden activations in FP32, output g = 1 + y.  Backward (training): FP32 matrix
// products on tiles of 32 rows in shared memory, one global atomic per parameter per tile.
// Adam update of the FP32 master weights, which are also rounded to the BF16 copy used by the forward.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "common.h"
#include "mlp.h"

namespace hrt {

// Parameter layout (FP32 master, same offsets in the BF16 copy):
//   W1 [64][16] (input dim 3 zero-padded to 16), b1 [64], W2 [64][64], b2 [64], W3 [64][64], b3 [64],
//   W4 [64] (output row), b4 [1]
constexpr int kH = 64, kIn = 16;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kH,
              kParams = kOffB4 + 1;
static_assert(kParams == kMlpParams, "parameter count");

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

// D[16x8] += A[16x16] (row major) * B[16x8] (column major), BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float d[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One dense layer on a 16-row tile held by a warp.  act: [16][K] FP32 activations in shared memory (this
// warp's tile), W: [64][K] BF16 weights in shared memory (row n = output neuron), bias FP32 [64].  Writes the
// pre-activations z [16][64] to zout (shared) for the caller's epilogue.
template <int K>
__device__ __forceinline__ void dense_tile(const float* __restrict__ act, const __nv_bfloat16* __restrict__ W,
                                           const float* __restrict__ bias, float* __restrict__ zout) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int nb = 0; nb < kH / 8; ++nb) {  // 8 output-column tiles of 8
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kb = 0; kb < K / 16; ++kb) {
      const int c0 = kb * 16 + t * 2;
      unsigned a[4];
      a[0] = pack_bf16(act[g * K + c0], act[g * K + c0 + 1]);
      a[1] = pack_bf16(act[(g + 8) * K + c0], act[(g + 8) * K + c0 + 1]);
      a[2] = pack_bf16(act[g * K + c0 + 8], act[g * K + c0 + 9]);
      a[3] = pack_bf16(act[(g + 8) * K + c0 + 8], act[(g + 8) * K + c0 + 9]);
      // B[k][n] = W[n][k]: column n = nb*8 + g, rows k = c0, c0+1 and c0+8, c0+9
      const __nv_bfloat16* wr = W + (nb * 8 + g) * K;
      unsigned b[2];
      b[0] = *reinterpret_cast<const unsigned*>(wr + c0);
      b[1] = *reinterpret_cast<const unsigned*>(wr + c0 + 8);
      mma_bf16(d, a, b);
    }
    const int col = nb * 8 + t * 2;
    zout[g * kH + col] = d[0] + bias[col];
    zout[g * kH + col + 1] = d[1] + bias[col + 1];
    zout[(g + 8) * kH + col] = d[2] + bias[col];
    zout[(g + 8) * kH + col + 1] = d[3] + bias[col + 1];
  }
}

constexpr int kWarps = 2;  // rows per block: 32 (static shared memory: weights 19 KB + tiles 16 KB)

__global__ void __launch_bounds__(32 * kWarps) mlp_forward_kernel(const float* __restrict__ x, int rows,
                                                                  const __nv_bfloat16* __restrict__ wb,
                                                                  const float* __restrict__ wf, float* __restrict__ y) {
  __shared__ __align__(16) __nv_bfloat16 sw[kOffB4 + 2];
  __shared__ float sb[3 * kH + kH + 1];  // b1, b2, b3, W4 (FP32 for the final dot), b4
  __shared__ float act[kWarps][16 * kH];
  __shared__ float z[kWarps][16 * kH];
  for (int i = threadIdx.x; i < kOffB4; i += blockDim.x) sw[i] = wb[i];
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    sb[i] = wf[kOffB1 + i];
    sb[kH + i] = wf[kOffB2 + i];
    sb[2 * kH + i] = wf[kOffB3 + i];
    sb[3 * kH + i] = __bfloat162float(wb[kOffW4 + i]);
  }
  if (threadIdx.x == 0) sb[4 * kH] = wf[kOffB4];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = (blockIdx.x * kWarps + warp) * 16;
  float* a = act[warp];
  float* zz = z[warp];
  // input tile [16][16]: features 0..2, zero padding
  for (int i = lane; i < 16 * kIn; i += 32) {
    const int r = i / kIn, c = i % kIn, row = row0 + r;
    a[i] = (c < 3 && row < rows) ? x[row * 3 + c] : 0.f;
  }
  __syncwarp();
  dense_tile<kIn>(a, sw + kOffW1, sb, zz);
  __syncwarp();
  for (int i = lane; i < 16 * kH; i += 32) a[i] = silu(zz[i]);
  __syncwarp();
  dense_tile<kH>(a, sw + kOffW2, sb + kH, zz);
  __syncwarp();
  for (int i = lane; i < 16 * kH; i += 32) a[i] = silu(zz[i]);
  __syncwarp();
  dense_tile<kH>(a, sw + kOffW3, sb + 2 * kH, zz);
  __syncwarp();
  for (int i = lane; i < 16 * kH; i += 32) a[i] = silu(zz[i]);
  __syncwarp();
  if (lane < 16) {
    const int row = row0 + lane;
    float s = sb[4 * kH];
    for (int k = 0; k < kH; ++k) s += a[lane * kH + k] * sb[3 * kH + k];
    if (row < rows) y[row] = 1.f + s;
  }
}

// Backward in FP32 (the BF16-rounded weights, as in the forward; FP32 activations) on a tile of kBwdRows rows
// per block, as matrix products in shared memory: the forward is recomputed layer by layer (Z = H W^T + b),
// then D3 = (gbar W4) o silu'(Z3), dW3 = D3^T H2, D2 = (D3 W3) o silu'(Z2), ... Thread mappings keep every
// shared access conflict-free: lane = row for the layer products (activation tiles padded to kLd columns, the
// weight row a warp-uniform broadcast), lane = input column k for the weight gradients.  Each block adds its
// tile's gradient with one global atomic per parameter.
constexpr int kBwdRows = 32, kBwdThreads = 256, kLd = kH + 1;
constexpr int kBwdSmemFloats = kH * 3 + kH + 2 * (kH * kH + kH) + kH + kBwdRows * 4 + 8 * kBwdRows * kLd;

__global__ void __launch_bounds__(kBwdThreads) mlp_backward_kernel(const float* __restrict__ x, int rows,
                                                                   const __nv_bfloat16* __restrict__ wb,
                                                                   const float* __restrict__ wf,
                                                                   const float* __restrict__ gbar,
                                                                   float* __restrict__ grad) {
  extern __shared__ float sm[];
  float* W1 = sm;                 // [64][3]
  float* B1 = W1 + kH * 3;        // [64]
  float* W2 = B1 + kH;            // [64][64] (row n = output neuron)
  float* B2 = W2 + kH * kH;
  float* W3 = B2 + kH;
  float* B3 = W3 + kH * kH;
  float* W4 = B3 + kH;            // [64]
  float* X = W4 + kH;             // [rows][3]
  float* GY = X + kBwdRows * 3;   // [rows]
  float* H1 = GY + kBwdRows;      // [rows][kLd] activations
  float* H2 = H1 + kBwdRows * kLd;
  float* H3 = H2 + kBwdRows * kLd;
  float* S1 = H3 + kBwdRows * kLd;  // silu'(Z)
  float* S2 = S1 + kBwdRows * kLd;
  float* S3 = S2 + kBwdRows * kLd;
  float* D = S3 + kBwdRows * kLd;   // deltas, ping-pong
  float* E = D + kBwdRows * kLd;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = blockIdx.x * kBwdRows;
  for (int i = tid; i < kH * 3; i += kBwdThreads) W1[i] = __bfloat162float(wb[kOffW1 + (i / 3) * kIn + i % 3]);
  for (int i = tid; i < kH * kH; i += kBwdThreads) {
    W2[i] = __bfloat162float(wb[kOffW2 + i]);
    W3[i] = __bfloat162float(wb[kOffW3 + i]);
  }
  for (int i = tid; i < kH; i += kBwdThreads) {
    B1[i] = wf[kOffB1 + i];
    B2[i] = wf[kOffB2 + i];
    B3[i] = wf[kOffB3 + i];
    W4[i] = __bfloat162float(wb[kOffW4 + i]);
  }
  for (int i = tid; i < kBwdRows * 3; i += kBwdThreads) {
    const int r = row0 + i / 3;
    X[i] = r < rows ? x[static_cast<int64_t>(r) * 3 + i % 3] : 0.f;
  }
  for (int i = tid; i < kBwdRows; i += kBwdThreads) GY[i] = row0 + i < rows ? gbar[row0 + i] : 0.f;
  __syncthreads();
  // forward recomputation; lane = row, warp -> output neurons n = warp + 8 i
  for (int i = 0; i < kH / 8; ++i) {
    const int n = warp + 8 * i;
    const float z = B1[n] + W1[n * 3] * X[lane * 3] + W1[n * 3 + 1] * X[lane * 3 + 1] + W1[n * 3 + 2] * X[lane * 3 + 2];
    H1[lane * kLd + n] = silu(z);
    S1[lane * kLd + n] = silu_grad(z);
  }
  __syncthreads();
  for (int i = 0; i < kH / 8; ++i) {
    const int n = warp + 8 * i;
    float z = B2[n];
    for (int k = 0; k < kH; ++k) z += W2[n * kH + k] * H1[lane * kLd + k];
    H2[lane * kLd + n] = silu(z);
    S2[lane * kLd + n] = silu_grad(z);
  }
  __syncthreads();
  for (int i = 0; i < kH / 8; ++i) {
    const int n = warp + 8 * i;
    float z = B3[n];
    for (int k = 0; k < kH; ++k) z += W3[n * kH + k] * H2[lane * kLd + k];
    H3[lane * kLd + n] = silu(z);
    S3[lane * kLd + n] = silu_grad(z);
  }
  __syncthreads();
  // output layer: dW4, db4 and D3 = gbar W4 o silu'(Z3)
  if (tid < kH) {
    float s = 0.f;
    for (int r = 0; r < kBwdRows; ++r) s += GY[r] * H3[r * kLd + tid];
    atomicAdd(grad + kOffW4 + tid, s);
  } else if (tid == kH) {
    float s = 0.f;
    for (int r = 0; r < kBwdRows; ++r) s += GY[r];
    atomicAdd(grad + kOffB4, s);
  }
  for (int i = 0; i < kH / 8; ++i) {
    const int n = warp + 8 * i;
    D[lane * kLd + n] = GY[lane] * W4[n] * S3[lane * kLd + n];
  }
  __syncthreads();
  // hidden layers 3 and 2: dW = D^T H_in, db = sum_r D, E = (D W) o silu'(Z_in)
  const float* h_in[2] = {H2, H1};
  const float* s_in[2] = {S2, S1};
  const float* w_l[2] = {W3, W2};
  const int off_w[2] = {kOffW3, kOffW2}, off_b[2] = {kOffB3, kOffB2};
  for (int l = 0; l < 2; ++l) {
    const float* hin = h_in[l];
    {
      const int k = tid & (kH - 1);
      for (int i = 0; i < kH / 4; ++i) {
        const int n = (tid >> 6) + 4 * i;
        float s = 0.f;
        for (int r = 0; r < kBwdRows; ++r) s += D[r * kLd + n] * hin[r * kLd + k];
        atomicAdd(grad + off_w[l] + n * kH + k, s);
      }
      if (tid < kH) {
        float s = 0.f;
        for (int r = 0; r < kBwdRows; ++r) s += D[r * kLd + tid];
        atomicAdd(grad + off_b[l] + tid, s);
      }
    }
    const float* w = w_l[l];
    for (int i = 0; i < kH / 8; ++i) {
      const int k = warp + 8 * i;
      float s = 0.f;
      for (int n = 0; n < kH; ++n) s += D[lane * kLd + n] * w[n * kH + k];
      E[lane * kLd + k] = s * s_in[l][lane * kLd + k];
    }
    __syncthreads();
    float* t = D;
    D = E;
    E = t;
  }
  // first layer: dW1 = D1^T X, db1 = sum_r D1
  if (tid < kH * 3) {
    const int n = tid / 3, k = tid % 3;
    float s = 0.f;
    for (int r = 0; r < kBwdRows; ++r) s += D[r * kLd + n] * X[r * 3 + k];
    atomicAdd(grad + kOffW1 + n * kIn + k, s);
  } else if (tid < kH * 4) {
    const int n = tid - kH * 3;
    float s = 0.f;
    for (int r = 0; r < kBwdRows; ++r) s += D[r * kLd + n];
    atomicAdd(grad + kOffB1 + n, s);
  }
}

// Adam step on the FP32 master weights (bias-corrected), then the BF16 copy; padding columns stay zero.
__global__ void adam_kernel(float* __restrict__ wf, __nv_bfloat16* __restrict__ wb, const float* __restrict__ grad,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParams) return;
  if (i < kOffB1 && (i % kIn) >= 3) {
    wb[i] = __float2bfloat16(0.f);
    return;
  }
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float w = wf[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  wf[i] = w;
  wb[i] = __float2bfloat16(w);
}

__global__ void to_bf16_kernel(const float* __restrict__ wf, __nv_bfloat16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kParams) wb[i] = __float2bfloat16((i < kOffB1 && (i % kIn) >= 3) ? 0.f : wf[i]);
}

hrt_status launch_mlp_forward(const float* x, int rows, const void* wb, const float* wf, float* y, cudaStream_t s) {
  const int blocks = (rows + 16 * kWarps - 1) / (16 * kWarps);
  mlp_forward_kernel<<<blocks, 32 * kWarps, 0, s>>>(x, rows, static_cast<const __nv_bfloat16*>(wb), wf, y);
  HRT_LAUNCHED("mlp_forward_kernel");
  return HRT_OK;
}

hrt_status launch_mlp_backward(const float* x, int rows, const void* wb, const float* wf, const float* gbar,
                               float* grad, cudaStream_t s) {
  const int smem = kBwdSmemFloats * static_cast<int>(sizeof(float));
  HRT_CUDA(cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  mlp_backward_kernel<<<(rows + kBwdRows - 1) / kBwdRows, kBwdThreads, smem, s>>>(
      x, rows, static_cast<const __nv_bfloat16*>(wb), wf, gbar, grad);
  HRT_LAUNCHED("mlp_backward_kernel");
  return HRT_OK;
}

hrt_status launch_adam(float* wf, void* wb, const float* grad, float* m, float* v, double lr, double b1, double b2,
                       double eps, int step, cudaStream_t s) {
  const float c1 = static_cast<float>(1.0 - std::pow(b1, step)), c2 = static_cast<float>(1.0 - std::pow(b2, step));
  adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(wf, static_cast<__nv_bfloat16*>(wb), grad, m, v,
                                                    static_cast<float>(lr), static_cast<float>(b1),
                                                    static_cast<float>(b2), static_cast<float>(eps), c1, c2);
  HRT_LAUNCHED("adam_kernel");
  return HRT_OK;
}

hrt_status launch_to_bf16(const float* wf, void* wb, cudaStream_t s) {
  to_bf16_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(wf, static_cast<__nv_bfloat16*>(wb));
  HRT_LAUNCHED("to_bf16_kernel");
  return HRT_OK;
}

// Inputs of the correction table at one scale factor: row i = (i dx, a, ln N_mesh), dx = |k|max cell / (rows - 1).
__global__ void correction_inputs_kernel(float* __restrict__ x, int rows, double dx, float a, float ln_n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  x[3 * i] = static_cast<float>(i * dx);
  x[3 * i + 1] = a;
  x[3 * i + 2] = ln_n;
}

hrt_status launch_correction_inputs(float* x, int rows, double dx, double a, double ln_n, cudaStream_t s) {
  correction_inputs_kernel<<<(rows + 255) / 256, 256, 0, s>>>(x, rows, dx, static_cast<float>(a),
                                                              static_cast<float>(ln_n));
  HRT_LAUNCHED("correction_inputs_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// Table adjoint of the learned k-space factor: given the half spectra of the ray-field cotangents and the
// density spectrum, table_bar[i] += sum over modes of w_kz Re(conj(gbar_j) d ghat_j / d g) times the linear
// interpolation weight of entry i (ghat_j = i d_j c0 g(|k|) rho_hat, c0 the filter without g).
// ---------------------------------------------------------------------------------------------------------
__global__ void kspace_table_adjoint_kernel(const float2* __restrict__ gbar_hat, int n_comp, const float2* __restrict__ rho_hat,
                                            int n, int nzc, float kf, float scale, int64_t elems,
                                            const float* __restrict__ wx, const float* __restrict__ wz, int g_nk,
                                            float g_inv_dk, float* __restrict__ table_bar) {
  const int iz = blockIdx.y * blockDim.x + threadIdx.x;
  const unsigned row = blockIdx.x * blockDim.y + threadIdx.y;
  if (iz >= nzc || row >= static_cast<unsigned>(n) * static_cast<unsigned>(n)) return;
  const int ix = static_cast<int>(row / static_cast<unsigned>(n));
  const int iy = static_cast<int>(row - static_cast<unsigned>(ix) * n);
  const int half = n >> 1;
  const int nx = ix < half ? ix : ix - n, ny = iy < half ? iy : iy - n;
  const float kx = kf * nx, ky = kf * ny, kz = kf * iz;
  const float k2 = kx * kx + ky * ky + kz * kz;
  if (k2 == 0.f) return;
  const float t = sqrtf(k2) * g_inv_dk;
  if (t >= static_cast<float>(g_nk - 1)) return;
  const int64_t e = static_cast<int64_t>(row) * nzc + iz;
  const float c0 = scale / k2 * __ldg(wx + ix) * __ldg(wx + iy) * __ldg(wz + iz);
  const float d[3] = {(nx == -half) ? 0.f : kx, (ny == -half) ? 0.f : ky, (iz == half) ? 0.f : kz};
  const float2 r = rho_hat[e];
  float v = 0.f;
  for (int j = 0; j < n_comp; ++j) {
    const float2 gb = gbar_hat[e + j * elems];
    // Re(conj(gb) * i d c0 r) = d c0 (gb.y r.x - gb.x r.y)
    v += d[j] * c0 * (gb.y * r.x - gb.x * r.y);
  }
  v *= (iz == 0 || iz == half) ? 1.f : 2.f;
  const int i = static_cast<int>(t);
  const float w = t - static_cast<float>(i);
  if (v != 0.f) {
    atomicAdd(table_bar + i, v * (1.f - w));
    atomicAdd(table_bar + i + 1, v * w);
  }
}

hrt_status launch_kspace_table_adjoint(const void* gbar_hat, int n_comp, const void* rho_hat, int64_t n, double box,
                                       double pref, const float* tab, int g_nk, double g_kmax, float* table_bar,
                                       cudaStream_t s) {
  const int64_t nzc = n / 2 + 1;
  dim3 block(64, 4);
  dim3 grid(static_cast<unsigned>((n * n + 3) / 4), static_cast<unsigned>((nzc + 63) / 64));
  kspace_table_adjoint_kernel<<<grid, block, 0, s>>>(
      static_cast<const float2*>(gbar_hat), n_comp, static_cast<const float2*>(rho_hat), static_cast<int>(n),
      static_cast<int>(nzc), static_cast<float>(2.0 * M_PI / box),
      static_cast<float>(-pref / (static_cast<double>(n) * n * n)), n * n * nzc, tab, tab + n, g_nk,
      static_cast<float>((g_nk - 1) / g_kmax), table_bar);
  HRT_LAUNCHED("kspace_table_adjoint_kernel");
  return HRT_OK;
}

}  // namespace hrt
