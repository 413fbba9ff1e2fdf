// Ray kernels of the HRT hot path on sm_103a: the KDK step with the A/B recursion and readout (Alg. 1),
// the force-free drift, and the binning of the convergence power spectrum.
//
// One thread per ray.  The line-of-sight node table of the step (FP64 on the host, rounded to float32 here)
// travels in the kernel parameters, so every warp reads it by broadcast from the constant bank.  The ray
// angle stays FP64; per half shell the FP64 base position r_ref * theta is split into an integer cell and a
// float32 fraction, and each node adds a small float32 offset (r_j - r_ref) theta, so the float32
// interpolation position keeps ~1e-6-cell accuracy at any distance from the observer.
#include <cuda_runtime.h>

#include <cmath>

#include "common.h"
#include "mesh_kernels.h"
#include "readout.cuh"

namespace hrt {

struct HalfKick {
  float kx, ky;              // kick
  float j00, j01, j10, j11;  // dK/dtheta
};

__device__ __forceinline__ void base_position(double obs, double r_ref, double theta, double cell, int n,
                                              int& i0, float& f0, int theta32 = 0) {
  if (theta32) {
    // the FP32 ablation: the position and its cell split in single precision
    float uf = (static_cast<float>(obs) + static_cast<float>(r_ref) * static_cast<float>(theta)) / static_cast<float>(cell);
    uf -= static_cast<float>(n) * floorf(uf / static_cast<float>(n));
    const float flf = floorf(uf);
    i0 = static_cast<int>(flf);
    if (i0 >= n) i0 -= n;
    if (i0 < 0) i0 += n;
    f0 = uf - flf;
    return;
  }
  double u = (obs + r_ref * theta) / cell;
  u -= n * floor(u / n);
  double fl = floor(u);
  i0 = static_cast<int>(fl);
  if (i0 >= n) i0 -= n;
  f0 = static_cast<float>(u - fl);
}

// Wraps k into [0, n): one compare for the usual k within a box of [0, n), the division only beyond.
__device__ __forceinline__ int wrap_cell(int k, int n) {
  if (k >= n) {
    k -= n;
    if (k >= n) k %= n;
  } else if (k < 0) {
    k += n;
    if (k < 0) {
      k %= n;
      if (k < 0) k += n;
    }
  }
  return k;
}

__device__ __forceinline__ void node_axis(int i0, float f0, float off, int n, int& i, float& f) {
  float u = f0 + off;
  float fl = floorf(u);
  f = u - fl;
  i = wrap_cell(i0 + static_cast<int>(fl), n);
}

__device__ __forceinline__ HalfKick half_kick(const RayStepParams& p, int j0, int j1, double th_x, double th_y,
                                              double ref_r, const float* __restrict__ gx,
                                              const float* __restrict__ gy) {
  HalfKick h{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (j1 <= j0) return h;
  const int n = p.n;
  int bx, by;
  float fbx, fby;
  base_position(p.obs_x, ref_r, th_x, p.cell, n, bx, fbx, p.theta32);
  base_position(p.obs_y, ref_r, th_y, p.cell, n, by, fby, p.theta32);
  const float tx = static_cast<float>(th_x), ty = static_cast<float>(th_y);
  const int64_t nn = n;
  for (int j = j0; j < j1; ++j) {
    const float dr = p.dr[j];
    int ix, iy;
    float fx, fy;
    node_axis(bx, fbx, dr * tx, n, ix, fx);
    node_axis(by, fby, dr * ty, n, iy, fy);
    const int iz = p.kz[j];
    const int jz = iz + 1 == n ? 0 : iz + 1;
    const float fz = p.fz[j];
    const int jx = ix + 1 == n ? 0 : ix + 1, jy = iy + 1 == n ? 0 : iy + 1;
    const int64_t r00 = (ix * nn + iy) * nn, r01 = (ix * nn + jy) * nn, r10 = (jx * nn + iy) * nn,
                  r11 = (jx * nn + jy) * nn;
    // z-interpolated columns of both fields
    float ax00 = __ldg(gx + r00 + iz), ax01 = __ldg(gx + r01 + iz), ax10 = __ldg(gx + r10 + iz),
          ax11 = __ldg(gx + r11 + iz);
    float bx00 = __ldg(gx + r00 + jz), bx01 = __ldg(gx + r01 + jz), bx10 = __ldg(gx + r10 + jz),
          bx11 = __ldg(gx + r11 + jz);
    float ay00 = __ldg(gy + r00 + iz), ay01 = __ldg(gy + r01 + iz), ay10 = __ldg(gy + r10 + iz),
          ay11 = __ldg(gy + r11 + iz);
    float by00 = __ldg(gy + r00 + jz), by01 = __ldg(gy + r01 + jz), by10 = __ldg(gy + r10 + jz),
          by11 = __ldg(gy + r11 + jz);
    float x00 = ax00 + fz * (bx00 - ax00), x01 = ax01 + fz * (bx01 - ax01);
    float x10 = ax10 + fz * (bx10 - ax10), x11 = ax11 + fz * (bx11 - ax11);
    float y00 = ay00 + fz * (by00 - ay00), y01 = ay01 + fz * (by01 - ay01);
    float y10 = ay10 + fz * (by10 - ay10), y11 = ay11 + fz * (by11 - ay11);
    // bilinear value and transverse derivatives (per cell; 1/cell is folded into cwr)
    float vx0 = x00 + fy * (x01 - x00), vx1 = x10 + fy * (x11 - x10);
    float vy0 = y00 + fy * (y01 - y00), vy1 = y10 + fy * (y11 - y10);
    float vx = vx0 + fx * (vx1 - vx0), vy = vy0 + fx * (vy1 - vy0);
    float dxx = vx1 - vx0, dyx = vy1 - vy0;
    float dxy = (x01 - x00) + fx * ((x11 - x10) - (x01 - x00));
    float dyy = (y01 - y00) + fx * ((y11 - y10) - (y01 - y00));
    const float c = p.cw[j], cr = p.cwr[j];
    h.kx += c * vx;
    h.ky += c * vy;
    h.j00 += cr * dxx;
    h.j01 += cr * dxy;
    h.j10 += cr * dyx;
    h.j11 += cr * dyy;
  }
  return h;
}

// Cell and fraction on a box axis of a sky coordinate (cell i_s, fraction f_s) under sign sgn and a translation
// of sh cells: u -> sgn u + sh (mod n); a flipped point on a cell face stays on the face (lower cell).
__device__ __forceinline__ void box_axis(int i_s, float f_s, int sgn, int sh, int n, int& ib, float& fb) {
  if (sgn > 0) {
    ib = i_s + sh;
    fb = f_s;
  } else if (f_s > 0.f) {
    ib = sh - i_s - 1;
    fb = 1.f - f_s;
  } else {
    ib = sh - i_s;
    fb = 0.f;
  }
  ib = wrap_cell(ib, n);
}

__device__ __forceinline__ int pick(int axis, int a, int b, int c) { return axis == 0 ? a : (axis == 1 ? b : c); }
__device__ __forceinline__ float pickf(int axis, float a, float b, float c) { return axis == 0 ? a : (axis == 1 ? b : c); }

// Trilinear value of field f at box cell (ix, iy, iz) + (fx, fy, fz) and its derivatives (per cell) along
// the three box axes.
__device__ __forceinline__ void trilinear3(const float* __restrict__ f, int64_t r00, int64_t r01, int64_t r10,
                                           int64_t r11, int iz, int jz, float fx, float fy, float fz, float& v,
                                           float& dX, float& dY, float& dZ) {
  const float a00 = __ldg(f + r00 + iz), a01 = __ldg(f + r01 + iz), a10 = __ldg(f + r10 + iz), a11 = __ldg(f + r11 + iz);
  const float z00 = __ldg(f + r00 + jz) - a00, z01 = __ldg(f + r01 + jz) - a01, z10 = __ldg(f + r10 + jz) - a10,
              z11 = __ldg(f + r11 + jz) - a11;
  const float e00 = a00 + fz * z00, e01 = a01 + fz * z01, e10 = a10 + fz * z10, e11 = a11 + fz * z11;
  const float h0 = e01 - e00, h1 = e11 - e10;
  const float g0 = e00 + fy * h0, g1 = e10 + fy * h1;
  v = g0 + fx * (g1 - g0);
  dX = g1 - g0;
  dY = h0 + fx * (h1 - h0);
  const float q0 = z00 + fy * (z01 - z00), q1 = z10 + fy * (z11 - z10);
  dZ = q0 + fx * (q1 - q0);
}

// Half kick through a light cone tiled by rotated and translated replicas: each node is mapped into its
// replica's box frame; the sky gradient component a is sign_a times field perm_a there, and its derivative along
// sky axis b is sign_a sign_b times the box derivative along perm_b.
__device__ __forceinline__ HalfKick half_kick_tiled(const RayStepParams& p, int j0, int j1, double th_x, double th_y,
                                                    double ref_r, const float* __restrict__ gx,
                                                    const float* __restrict__ gy, const float* __restrict__ gz) {
  HalfKick h{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (j1 <= j0) return h;
  const int n = p.n;
  int bx, by;
  float fbx, fby;
  base_position(p.obs_x, ref_r, th_x, p.cell, n, bx, fbx, p.theta32);
  base_position(p.obs_y, ref_r, th_y, p.cell, n, by, fby, p.theta32);
  const float tx = static_cast<float>(th_x), ty = static_cast<float>(th_y);
  const int64_t nn = n;
  for (int j = j0; j < j1; ++j) {
    const float dr = p.dr[j];
    int ix, iy;
    float fx, fy;
    node_axis(bx, fbx, dr * tx, n, ix, fx);
    node_axis(by, fby, dr * ty, n, iy, fy);
    const int R = p.rep[j];
    const int p0 = p.rperm[R][0], p1 = p.rperm[R][1];
    const int s0 = p.rsign[R][0], s1 = p.rsign[R][1];
    int c0, c1;
    float q0, q1;
    box_axis(ix, fx, s0, p.rshift[R][0], n, c0, q0);
    box_axis(iy, fy, s1, p.rshift[R][1], n, c1, q1);
    const int c2 = p.kz[j];
    const float q2 = p.fz[j];
    // box-frame cell and fraction per box axis (axis p0 from sky x, p1 from sky y, the other from the line of sight)
    const int jx_ = pick(0 == p0 ? 0 : (0 == p1 ? 1 : 2), c0, c1, c2), jy_ = pick(1 == p0 ? 0 : (1 == p1 ? 1 : 2), c0, c1, c2),
              jz_ = pick(2 == p0 ? 0 : (2 == p1 ? 1 : 2), c0, c1, c2);
    const float gfx = pickf(0 == p0 ? 0 : (0 == p1 ? 1 : 2), q0, q1, q2), gfy = pickf(1 == p0 ? 0 : (1 == p1 ? 1 : 2), q0, q1, q2),
                gfz = pickf(2 == p0 ? 0 : (2 == p1 ? 1 : 2), q0, q1, q2);
    const int kx = jx_ + 1 == n ? 0 : jx_ + 1, ky = jy_ + 1 == n ? 0 : jy_ + 1, kz2 = jz_ + 1 == n ? 0 : jz_ + 1;
    const int64_t r00 = (jx_ * nn + jy_) * nn, r01 = (jx_ * nn + ky) * nn, r10 = (kx * nn + jy_) * nn,
                  r11 = (kx * nn + ky) * nn;
    const float* fa = p0 == 0 ? gx : (p0 == 1 ? gy : gz);
    const float* fb = p1 == 0 ? gx : (p1 == 1 ? gy : gz);
    float va, aX, aY, aZ, vb, bX, bY, bZ;
    trilinear3(fa, r00, r01, r10, r11, jz_, kz2, gfx, gfy, gfz, va, aX, aY, aZ);
    trilinear3(fb, r00, r01, r10, r11, jz_, kz2, gfx, gfy, gfz, vb, bX, bY, bZ);
    const float ss = static_cast<float>(s0 * s1);
    const float c = p.cw[j], cr = p.cwr[j];
    h.kx += c * (s0 * va);
    h.ky += c * (s1 * vb);
    h.j00 += cr * pickf(p0, aX, aY, aZ);
    h.j01 += cr * (ss * pickf(p1, aX, aY, aZ));
    h.j10 += cr * (ss * pickf(p0, bX, bY, bZ));
    h.j11 += cr * pickf(p1, bX, bY, bZ);
  }
  return h;
}

// One thread per ray.  __launch_bounds__(128, 1) leaves the register count to the compiler (72 for the direct
// gather): measured at 2048^2 rays over a 1024^3 mesh, 1.05 ms per step against 1.29 ms with 56 registers, and
// unrolling the node loop (1.13-1.49 ms) does not help; the loop waits on the latency of its gathers.
template <bool TILED>
__global__ void __launch_bounds__(128, 1) ray_step_kernel(double2* __restrict__ theta, float2* __restrict__ eta,
                                                       float4* __restrict__ Amat, float4* __restrict__ Bmat,
                                                       int64_t nr, const float* __restrict__ gx,
                                                       const float* __restrict__ gy, const __grid_constant__ RayStepParams p,
                                                       float* __restrict__ maps, const float* __restrict__ gz) {
  int64_t r;
  if (p.tile_w > 0) {
    // 16 x 8 pixel tiles in row-major tile order; a warp covers 16 x 2 neighbouring pixels
    const unsigned tiles_x = static_cast<unsigned>(p.tile_w) >> 4;
    const unsigned tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int64_t x = tx * 16 + (threadIdx.x & 15), y = ty * 8 + (threadIdx.x >> 4);
    r = y * p.tile_w + x;
  } else {
    r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  }
  if (r >= nr) return;
  double2 th = theta[r];
  float2 et = eta[r];
  float4 A = Amat[r], B = Bmat[r];

  HalfKick h = TILED ? half_kick_tiled(p, 0, p.n1, th.x, th.y, p.ref_r[0], gx, gy, gz)
                     : half_kick(p, 0, p.n1, th.x, th.y, p.ref_r[0], gx, gy);
  et.x += h.kx;
  et.y += h.ky;
  // B += J A (row-major 2x2: x = 11, y = 12, z = 21, w = 22)
  B.x += h.j00 * A.x + h.j01 * A.z;
  B.y += h.j00 * A.y + h.j01 * A.w;
  B.z += h.j10 * A.x + h.j11 * A.z;
  B.w += h.j10 * A.y + h.j11 * A.w;
  // drift: theta in FP64, A in float32
  const double d = p.drift_d;
  if (p.theta32) {
    const float df = static_cast<float>(d);
    th.x = static_cast<double>(static_cast<float>(th.x) + df * et.x);
    th.y = static_cast<double>(static_cast<float>(th.y) + df * et.y);
  } else {
    th.x += d * static_cast<double>(et.x);
    th.y += d * static_cast<double>(et.y);
  }
  A.x += p.drift * B.x;
  A.y += p.drift * B.y;
  A.z += p.drift * B.z;
  A.w += p.drift * B.w;
  h = TILED ? half_kick_tiled(p, p.n1, p.n1 + p.n2, th.x, th.y, p.ref_r[1], gx, gy, gz)
            : half_kick(p, p.n1, p.n1 + p.n2, th.x, th.y, p.ref_r[1], gx, gy);
  et.x += h.kx;
  et.y += h.ky;
  B.x += h.j00 * A.x + h.j01 * A.z;
  B.y += h.j00 * A.y + h.j01 * A.w;
  B.z += h.j10 * A.x + h.j11 * A.z;
  B.w += h.j10 * A.y + h.j11 * A.w;

  theta[r] = th;
  eta[r] = et;
  Amat[r] = A;
  Bmat[r] = B;
  if (maps != nullptr) {
    float k, g1, g2, om;
    readout(A, k, g1, g2, om);
    if (p.map_accumulate) {
      // O = sum_n n_g(chi_n) O_n (Eq. obs_accum): this step's observables with the caller's weight
      const float w = p.map_weight;
      maps[r] += w * k;
      maps[r + nr] += w * g1;
      maps[r + 2 * nr] += w * g2;
      maps[r + 3 * nr] += w * om;
    } else {
      maps[r] = k;
      maps[r + nr] = g1;
      maps[r + 2 * nr] = g2;
      maps[r + 3 * nr] = om;
    }
  }
}

hrt_status launch_ray_step(const hrt_rays& rays, const float* gx, const float* gy, const RayStepParams& p,
                           float* maps, cudaStream_t s, const float* gz) {
  if (rays.n_rays == 0) return HRT_OK;
  if (p.tiled && !gz) return fail(HRT_ERR_INVALID_ARG, "light-cone tiling needs the third gradient component");
  auto* kernel = p.tiled ? ray_step_kernel<true> : ray_step_kernel<false>;
  kernel<<<blocks_for(rays.n_rays, 128), 128, 0, s>>>(
      reinterpret_cast<double2*>(rays.theta), reinterpret_cast<float2*>(rays.eta),
      reinterpret_cast<float4*>(rays.A), reinterpret_cast<float4*>(rays.B), rays.n_rays, gx, gy, p, maps, gz);
  HRT_LAUNCHED("ray_step_kernel");
  return HRT_OK;
}

__global__ void ray_drift_kernel(double2* __restrict__ theta, const float2* __restrict__ eta,
                                 float4* __restrict__ Amat, const float4* __restrict__ Bmat, int64_t nr, double d) {
  int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (r >= nr) return;
  double2 th = theta[r];
  float2 et = eta[r];
  th.x += d * static_cast<double>(et.x);
  th.y += d * static_cast<double>(et.y);
  theta[r] = th;
  float4 A = Amat[r];
  const float4 B = Bmat[r];
  const float df = static_cast<float>(d);
  A.x += df * B.x;
  A.y += df * B.y;
  A.z += df * B.z;
  A.w += df * B.w;
  Amat[r] = A;
}

hrt_status launch_ray_drift_free(const hrt_rays& rays, double d, cudaStream_t s) {
  if (rays.n_rays == 0) return HRT_OK;
  ray_drift_kernel<<<blocks_for(rays.n_rays, 256), 256, 0, s>>>(
      reinterpret_cast<double2*>(rays.theta), reinterpret_cast<const float2*>(rays.eta),
      reinterpret_cast<float4*>(rays.A), reinterpret_cast<const float4*>(rays.B), rays.n_rays, d);
  HRT_LAUNCHED("ray_drift_kernel");
  return HRT_OK;
}

__global__ void ray_readout_kernel(const float4* __restrict__ Amat, int64_t nr, float* __restrict__ maps) {
  int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (r >= nr) return;
  float k, g1, g2, om;
  readout(Amat[r], k, g1, g2, om);
  maps[r] = k;
  maps[r + nr] = g1;
  maps[r + 2 * nr] = g2;
  maps[r + 3 * nr] = om;
}

hrt_status launch_ray_readout(const hrt_rays& rays, float* maps, cudaStream_t s) {
  if (rays.n_rays == 0) return HRT_OK;
  ray_readout_kernel<<<blocks_for(rays.n_rays, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(rays.A),
                                                                  rays.n_rays, maps);
  HRT_LAUNCHED("ray_readout_kernel");
  return HRT_OK;
}

// theta0 may be theta itself (initialisation in place)
__global__ void rays_init_kernel(double2* theta, float2* __restrict__ eta, float4* __restrict__ Amat,
                                 float4* __restrict__ Bmat, const double2* theta0, int64_t nr) {
  int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (r >= nr) return;
  theta[r] = theta0[r];
  eta[r] = make_float2(0.f, 0.f);
  Amat[r] = make_float4(1.f, 0.f, 0.f, 1.f);
  Bmat[r] = make_float4(0.f, 0.f, 0.f, 0.f);
}

hrt_status launch_rays_init(const hrt_rays& rays, const double* theta0, cudaStream_t s) {
  if (rays.n_rays == 0) return HRT_OK;
  rays_init_kernel<<<blocks_for(rays.n_rays, 256), 256, 0, s>>>(
      reinterpret_cast<double2*>(rays.theta), reinterpret_cast<float2*>(rays.eta),
      reinterpret_cast<float4*>(rays.A), reinterpret_cast<float4*>(rays.B),
      reinterpret_cast<const double2*>(theta0), rays.n_rays);
  HRT_LAUNCHED("rays_init_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// Power-spectrum binning of the m x (m/2+1) half spectrum of kappa.  Column kz = 1..m/2-1 stands for two
// modes (n and -n); kz = 0 and kz = m/2 for one.  The bin of a mode is decided in FP64 exactly as stated in
// the header.  Per-block shared accumulators, then one FP64 atomic per bin and block into sums[3][nbins].
// ---------------------------------------------------------------------------------------------------------
__global__ void power_bin_kernel(const float2* __restrict__ spec, int m, double theta_field, double p_norm,
                                 int nbins, double ln_lmin, double inv_ln_ratio, double* __restrict__ sums) {
  extern __shared__ double sh[];  // [3][nbins]
  for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) sh[i] = 0.0;
  __syncthreads();
  const int mzc = m / 2 + 1;
  const int64_t total = static_cast<int64_t>(m) * mzc;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int ix = static_cast<int>(e / mzc);
    int iz = static_cast<int>(e - static_cast<int64_t>(ix) * mzc);
    int nx = ix < m / 2 ? ix : ix - m;
    double n2 = static_cast<double>(nx) * nx + static_cast<double>(iz) * iz;
    if (n2 <= 0.0) continue;
    double ell = 2.0 * M_PI * sqrt(n2) / theta_field;
    double t = nbins * (log(ell) - ln_lmin) * inv_ln_ratio + 1e-9;
    if (!(t >= 0.0) || t >= nbins) continue;
    int b = static_cast<int>(floor(t));
    float2 v = spec[e];
    double w = (iz == 0 || iz == m / 2) ? 1.0 : 2.0;
    double pw = (static_cast<double>(v.x) * v.x + static_cast<double>(v.y) * v.y) * p_norm;
    atomicAdd(sh + b, w * pw);
    atomicAdd(sh + nbins + b, w * ell);
    atomicAdd(sh + 2 * nbins + b, w);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x)
    if (sh[i] != 0.0) atomicAdd(sums + i, sh[i]);
}

hrt_status launch_power_bin(const void* spec, int64_t m, double dtheta, int nbins, double ell_min, double ell_max,
                            double* sums, cudaStream_t s) {
  HRT_CUDA(cudaMemsetAsync(sums, 0, 3 * nbins * sizeof(double), s));
  double theta_field = m * dtheta;
  // |FFT|^2 dtheta^4 / Theta^2
  double p_norm = dtheta * dtheta * dtheta * dtheta / (theta_field * theta_field);
  int64_t total = m * (m / 2 + 1);
  unsigned blocks = blocks_for(total, 256);
  if (blocks > 4 * 152) blocks = 4 * 152;
  power_bin_kernel<<<blocks, 256, 3 * nbins * sizeof(double), s>>>(
      static_cast<const float2*>(spec), static_cast<int>(m), theta_field, p_norm, nbins, std::log(ell_min),
      1.0 / std::log(ell_max / ell_min), sums);
  HRT_LAUNCHED("power_bin_kernel");
  return HRT_OK;
}

}  // namespace hrt
