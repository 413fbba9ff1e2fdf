// Mesh kernels of the HRT hot path on sm_103a: CIC mass assignment, the fused k-space Poisson/gradient/
// deconvolution kernel, the fused particle gather + kick + drift, and the Zel'dovich IC helpers.
//
// All three mesh passes are bound by HBM bandwidth; the kernels are written for coalesced 4- and 8-byte
// accesses with the particles in Lagrangian-lattice order (neighbouring threads touch neighbouring cells,
// so the CIC atomics and gathers hit lines already resident in the 129 MB L2).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "common.h"
#include "mesh_kernels.h"

namespace hrt {

// Lower node (wrapped into [0, n)) and fraction of a coordinate given as lattice node + displacement in cells.
__device__ __forceinline__ void cic_axis(int q_node, float d_cells, int n, int& i0, float& f) {
  float fl = floorf(d_cells);
  f = d_cells - fl;
  int i = q_node + static_cast<int>(fl);
  i %= n;
  i0 = i < 0 ? i + n : i;
}

__device__ __forceinline__ int wrap_next(int i, int n) { return i + 1 == n ? 0 : i + 1; }

// ---------------------------------------------------------------------------------------------------------
// CIC mass assignment: one thread per particle, eight float32 reductions into the mesh.
// ---------------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) cic_scatter_kernel(const float* __restrict__ dx,
                                                          const float* __restrict__ dy,
                                                          const float* __restrict__ dz, int64_t np,
                                                          int n_side, int ratio, int n, float inv_cell,
                                                          float mass, float* __restrict__ rho) {
  int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= np) return;
  int qk = static_cast<int>(p % n_side);
  int64_t t = p / n_side;
  int qj = static_cast<int>(t % n_side);
  int qi = static_cast<int>(t / n_side);
  int ix, iy, iz;
  float fx, fy, fz;
  cic_axis(qi * ratio, __ldg(dx + p) * inv_cell, n, ix, fx);
  cic_axis(qj * ratio, __ldg(dy + p) * inv_cell, n, iy, fy);
  cic_axis(qk * ratio, __ldg(dz + p) * inv_cell, n, iz, fz);
  int jx = wrap_next(ix, n), jy = wrap_next(iy, n), jz = wrap_next(iz, n);
  float wx0 = (1.f - fx) * mass, wx1 = fx * mass;
  float wy0 = 1.f - fy, wy1 = fy, wz0 = 1.f - fz, wz1 = fz;
  int64_t nn = n;
  int64_t r00 = (ix * nn + iy) * nn, r01 = (ix * nn + jy) * nn, r10 = (jx * nn + iy) * nn,
          r11 = (jx * nn + jy) * nn;
  atomicAdd(rho + r00 + iz, wx0 * wy0 * wz0);
  atomicAdd(rho + r00 + jz, wx0 * wy0 * wz1);
  atomicAdd(rho + r01 + iz, wx0 * wy1 * wz0);
  atomicAdd(rho + r01 + jz, wx0 * wy1 * wz1);
  atomicAdd(rho + r10 + iz, wx1 * wy0 * wz0);
  atomicAdd(rho + r10 + jz, wx1 * wy0 * wz1);
  atomicAdd(rho + r11 + iz, wx1 * wy1 * wz0);
  atomicAdd(rho + r11 + jz, wx1 * wy1 * wz1);
}

hrt_status launch_cic_scatter(const float* disp, int64_t n_side, int64_t n, double box, float* rho,
                              cudaStream_t s) {
  int64_t np = n_side * n_side * n_side;
  size_t mesh_bytes = static_cast<size_t>(n) * n * n * sizeof(float);
  HRT_CUDA(cudaMemsetAsync(rho, 0, mesh_bytes, s));
  if (np == 0) return HRT_OK;
  float mass = static_cast<float>(static_cast<double>(n) * n * n / static_cast<double>(np));
  cic_scatter_kernel<<<blocks_for(np, 256), 256, 0, s>>>(disp, disp + np, disp + 2 * np, np,
                                                         static_cast<int>(n_side),
                                                         static_cast<int>(n / n_side), static_cast<int>(n),
                                                         static_cast<float>(n / box), mass, rho);
  HRT_LAUNCHED("cic_scatter_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// Fused k-space kernel: out_j = i d_j * scale / k^2 * Wx Wy Wz * g(|k|) * rho_hat
// Per-axis filter factors (sinc^-p exp(-k_i^2 s^2/2)) come from FP64 host tables; the Green's function,
// derivative and learned correction are evaluated per element.  Grid: x over rows (ix, iy), y over z chunks.
// ---------------------------------------------------------------------------------------------------------
struct KspaceSet {
  const float* wx;  // per-axis factor tables [n], [n], [n/2+1]
  const float* wy;
  const float* wz;
  const float* g;   // learned correction table or nullptr
  int g_nk;
  float g_inv_dk;   // (g_nk - 1) / g_kmax
  int n_out;
  float2* out;      // n_out spectra, stride elems
};

__device__ __forceinline__ float learned_g(const KspaceSet& s, float kmag) {
  if (s.g == nullptr) return 1.f;
  float t = kmag * s.g_inv_dk;
  if (t >= static_cast<float>(s.g_nk - 1)) return 1.f;
  int i = static_cast<int>(t);
  float w = t - static_cast<float>(i);
  return __ldg(s.g + i) * (1.f - w) + __ldg(s.g + i + 1) * w;
}

__global__ void __launch_bounds__(256) kspace_kernel(const float2* __restrict__ rho_hat, int n, int nzc,
                                                     float kf, float scale, int64_t elems, KspaceSet a,
                                                     KspaceSet b) {
  int iz = blockIdx.y * blockDim.x + threadIdx.x;
  int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.y + threadIdx.y;
  if (iz >= nzc || row >= static_cast<int64_t>(n) * n) return;
  int ix = static_cast<int>(row / n);
  int iy = static_cast<int>(row - static_cast<int64_t>(ix) * n);
  int half = n >> 1;
  int nx = ix < half ? ix : ix - n;
  int ny = iy < half ? iy : iy - n;
  int nz = iz;
  float kx = kf * nx, ky = kf * ny, kz = kf * nz;
  float k2 = kx * kx + ky * ky + kz * kz;
  int64_t e = row * nzc + iz;
  float2 v = rho_hat[e];
  float dx = (nx == -half) ? 0.f : kx;
  float dy = (ny == -half) ? 0.f : ky;
  float dz = (nz == half) ? 0.f : kz;
  float green = k2 > 0.f ? scale / k2 : 0.f;
  float kmag = sqrtf(k2);
  {
    float c = green * __ldg(a.wx + ix) * __ldg(a.wy + iy) * __ldg(a.wz + iz) * learned_g(a, kmag);
    float2 base = make_float2(-c * v.y, c * v.x);  // i * c * v
    a.out[e] = make_float2(dx * base.x, dx * base.y);
    if (a.n_out > 1) a.out[e + elems] = make_float2(dy * base.x, dy * base.y);
    if (a.n_out > 2) a.out[e + 2 * elems] = make_float2(dz * base.x, dz * base.y);
  }
  if (b.n_out > 0) {
    float c = green * __ldg(b.wx + ix) * __ldg(b.wy + iy) * __ldg(b.wz + iz) * learned_g(b, kmag);
    float2 base = make_float2(-c * v.y, c * v.x);
    b.out[e] = make_float2(dx * base.x, dx * base.y);
    if (b.n_out > 1) b.out[e + elems] = make_float2(dy * base.x, dy * base.y);
    if (b.n_out > 2) b.out[e + 2 * elems] = make_float2(dz * base.x, dz * base.y);
  }
}

// FP64 host tables of the separable filter factor sinc(k_i cell/2)^-p exp(-k_i^2 s^2/2) for the x (= y)
// axis (n entries, signed frequency) and the z axis (n/2 + 1 entries).
void filter_tables(int64_t n, double box, const hrt_filter& f, std::vector<float>& wxy, std::vector<float>& wz) {
  const double kf = 2.0 * M_PI / box, cell = box / n;
  auto factor = [&](int64_t ni) {
    double k = kf * ni;
    double x = 0.5 * k * cell;
    double s = x == 0.0 ? 1.0 : std::sin(x) / x;
    double w = f.deconv_p != 0.0 ? std::pow(s, -f.deconv_p) : 1.0;
    if (f.smooth > 0.0) w *= std::exp(-0.5 * k * k * f.smooth * f.smooth);
    return static_cast<float>(w);
  };
  wxy.resize(n);
  wz.resize(n / 2 + 1);
  for (int64_t i = 0; i < n; ++i) wxy[i] = factor(i < n / 2 ? i : i - n);
  for (int64_t i = 0; i <= n / 2; ++i) wz[i] = factor(i);
}

hrt_status launch_kspace(const void* rho_hat, int64_t n, double box, double pref, const float* tab_a,
                         const hrt_filter* fa, int n_a, void* out_a, const float* tab_b, const hrt_filter* fb,
                         int n_b, void* out_b, cudaStream_t s) {
  int64_t nzc = n / 2 + 1;
  int64_t elems = n * n * nzc;
  double scale = -pref / (static_cast<double>(n) * n * n);
  auto make_set = [&](const float* tab, const hrt_filter* f, int n_out, void* out) {
    KspaceSet k{};
    k.n_out = n_out;
    if (n_out == 0) return k;
    k.wx = tab;
    k.wy = tab;
    k.wz = tab + n;
    k.g = f->g_table;
    k.g_nk = f->g_nk;
    k.g_inv_dk = f->g_table ? static_cast<float>((f->g_nk - 1) / f->g_kmax) : 0.f;
    k.out = static_cast<float2*>(out);
    return k;
  };
  KspaceSet a = make_set(tab_a, fa, n_a, out_a);
  KspaceSet b = make_set(tab_b, fb, n_b, out_b);
  dim3 block(64, 4);
  dim3 grid(static_cast<unsigned>((n * n + block.y - 1) / block.y),
            static_cast<unsigned>((nzc + block.x - 1) / block.x));
  kspace_kernel<<<grid, block, 0, s>>>(static_cast<const float2*>(rho_hat), static_cast<int>(n),
                                       static_cast<int>(nzc), static_cast<float>(2.0 * M_PI / box),
                                       static_cast<float>(scale), elems, a, b);
  HRT_LAUNCHED("kspace_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// Particle gather + kick + drift: one thread per particle.
// ---------------------------------------------------------------------------------------------------------
__device__ __forceinline__ float trilinear(const float* __restrict__ f, int64_t r00, int64_t r01, int64_t r10,
                                           int64_t r11, int iz, int jz, float fx, float fy, float fz) {
  float c00 = __ldg(f + r00 + iz), c00z = __ldg(f + r00 + jz);
  float c01 = __ldg(f + r01 + iz), c01z = __ldg(f + r01 + jz);
  float c10 = __ldg(f + r10 + iz), c10z = __ldg(f + r10 + jz);
  float c11 = __ldg(f + r11 + iz), c11z = __ldg(f + r11 + jz);
  float a00 = c00 + fz * (c00z - c00), a01 = c01 + fz * (c01z - c01);
  float a10 = c10 + fz * (c10z - c10), a11 = c11 + fz * (c11z - c11);
  float b0 = a00 + fy * (a01 - a00), b1 = a10 + fy * (a11 - a10);
  return b0 + fx * (b1 - b0);
}

__global__ void __launch_bounds__(256) kick_drift_kernel(const float* __restrict__ gx,
                                                         const float* __restrict__ gy,
                                                         const float* __restrict__ gz, int n,
                                                         float inv_cell, int64_t np, int n_side, int ratio,
                                                         float* __restrict__ disp, float* __restrict__ mom,
                                                         float kick, float drift) {
  int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= np) return;
  int qk = static_cast<int>(p % n_side);
  int64_t t = p / n_side;
  int qj = static_cast<int>(t % n_side);
  int qi = static_cast<int>(t / n_side);
  float d0 = disp[p], d1 = disp[p + np], d2 = disp[p + 2 * np];
  float m0 = mom[p], m1 = mom[p + np], m2 = mom[p + 2 * np];
  int ix, iy, iz;
  float fx, fy, fz;
  cic_axis(qi * ratio, d0 * inv_cell, n, ix, fx);
  cic_axis(qj * ratio, d1 * inv_cell, n, iy, fy);
  cic_axis(qk * ratio, d2 * inv_cell, n, iz, fz);
  int jx = wrap_next(ix, n), jy = wrap_next(iy, n), jz = wrap_next(iz, n);
  int64_t nn = n;
  int64_t r00 = (ix * nn + iy) * nn, r01 = (ix * nn + jy) * nn, r10 = (jx * nn + iy) * nn,
          r11 = (jx * nn + jy) * nn;
  float a0 = trilinear(gx, r00, r01, r10, r11, iz, jz, fx, fy, fz);
  float a1 = trilinear(gy, r00, r01, r10, r11, iz, jz, fx, fy, fz);
  float a2 = trilinear(gz, r00, r01, r10, r11, iz, jz, fx, fy, fz);
  m0 -= a0 * kick;
  m1 -= a1 * kick;
  m2 -= a2 * kick;
  mom[p] = m0;
  mom[p + np] = m1;
  mom[p + 2 * np] = m2;
  if (drift != 0.f) {
    disp[p] = d0 + m0 * drift;
    disp[p + np] = d1 + m1 * drift;
    disp[p + 2 * np] = d2 + m2 * drift;
  }
}

hrt_status launch_kick_drift(const float* grad, int64_t n, double box, int64_t n_side, float* disp, float* mom,
                             double kick, double drift, cudaStream_t s) {
  int64_t np = n_side * n_side * n_side;
  if (np == 0) return HRT_OK;
  int64_t m = n * n * n;
  kick_drift_kernel<<<blocks_for(np, 256), 256, 0, s>>>(grad, grad + m, grad + 2 * m, static_cast<int>(n),
                                                        static_cast<float>(n / box), np,
                                                        static_cast<int>(n_side), static_cast<int>(n / n_side),
                                                        disp, mom, static_cast<float>(kick),
                                                        static_cast<float>(drift));
  HRT_LAUNCHED("kick_drift_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// Zel'dovich ICs: Psi_j = i d_j T(n^2) w_hat with T from an FP64 host table indexed by the integer |n|^2
// (T = D1 sqrt(P(k)/V_cell) / k^2 / n_side^3), then mom = ratio * disp.
// ---------------------------------------------------------------------------------------------------------
__global__ void ic_kspace_kernel(const float2* __restrict__ w_hat, int n, int nzc, float kf,
                                 const float* __restrict__ table, int64_t elems, float2* __restrict__ out) {
  int iz = blockIdx.y * blockDim.x + threadIdx.x;
  int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.y + threadIdx.y;
  if (iz >= nzc || row >= static_cast<int64_t>(n) * n) return;
  int ix = static_cast<int>(row / n);
  int iy = static_cast<int>(row - static_cast<int64_t>(ix) * n);
  int half = n >> 1;
  int nx = ix < half ? ix : ix - n;
  int ny = iy < half ? iy : iy - n;
  int nz = iz;
  int64_t e = row * nzc + iz;
  float c = __ldg(table + (nx * nx + ny * ny + nz * nz));
  float2 v = w_hat[e];
  float2 base = make_float2(-c * v.y, c * v.x);
  float dx = (nx == -half) ? 0.f : kf * nx;
  float dy = (ny == -half) ? 0.f : kf * ny;
  float dz = (nz == half) ? 0.f : kf * nz;
  out[e] = make_float2(dx * base.x, dx * base.y);
  out[e + elems] = make_float2(dy * base.x, dy * base.y);
  out[e + 2 * elems] = make_float2(dz * base.x, dz * base.y);
}

hrt_status launch_ic_kspace(const void* w_hat, int64_t n, double box, const float* table, void* out,
                            cudaStream_t s) {
  int64_t nzc = n / 2 + 1;
  dim3 block(64, 4);
  dim3 grid(static_cast<unsigned>((n * n + 3) / 4), static_cast<unsigned>((nzc + 63) / 64));
  ic_kspace_kernel<<<grid, block, 0, s>>>(static_cast<const float2*>(w_hat), static_cast<int>(n),
                                          static_cast<int>(nzc), static_cast<float>(2.0 * M_PI / box), table,
                                          n * n * nzc, static_cast<float2*>(out));
  HRT_LAUNCHED("ic_kspace_kernel");
  return HRT_OK;
}

__global__ void scale_copy_kernel(const float* __restrict__ in, float* __restrict__ out, float ratio, int64_t m) {
  int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < m) out[i] = ratio * in[i];
}

hrt_status launch_scale_copy(const float* in, float* out, double ratio, int64_t m, cudaStream_t s) {
  if (m == 0) return HRT_OK;
  scale_copy_kernel<<<blocks_for(m, 256), 256, 0, s>>>(in, out, static_cast<float>(ratio), m);
  HRT_LAUNCHED("scale_copy_kernel");
  return HRT_OK;
}

}  // namespace hrt
