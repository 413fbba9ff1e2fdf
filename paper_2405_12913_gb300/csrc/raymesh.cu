// The ray-mesh kick operator on sm_103a (Sec. 5.2, Sec. 5.3, App. C of arXiv 2405.12913): the kick of a half
// shell is accumulated on an adaptive 2D angular mesh from the 3D gradient mesh, deconvolved and smoothed by 2D
// FFT, and interpolated to the rays.
//
// * Projection.  The 3D nodes of the planes z = kz cell inside the shell are projected to the angles
//   (X_xy - O_xy) / r and CIC-weighted onto the ray mesh.  The kernel gathers instead of scattering: each
//   ray-mesh node m sums, per plane, the few 3D nodes i within one ray-mesh cell of it, with weight
//   (1 - |i - s_m| / P)_+ per axis, where s_m = Q + m P is the node's position in 3D cells and P = r x2d / cell.
//   That is the same sum as the scatter (no atomics, deterministic).  A CTA covers 8 x 32 ray-mesh nodes; it
//   computes its per-plane base position in FP64 once and splits it into a wrapped integer cell plus a float
//   fraction, so that every thread's float offset stays small.  The two kick components travel as one complex
//   field Kx + i Ky: the filter is real and even in k, so one C2C transform pair filters both.
// * Filter.  sinc(k_x x2d / 2)^-4 sinc(k_y x2d / 2)^-4 exp(-k^2 lambda^2 / 2) with the 1 / N^2 of the inverse
//   transform, evaluated per element (x2d = iota lambda, so the Gaussian is exp(-w^2 / (2 iota^2)) in the phase
//   step w = k x2d per mesh cell).
// * Rays.  One thread per ray runs the KDK step with the A/B recursion: bilinear kick and its derivative from
//   the first half shell's mesh, drift, the same from the second; readout as in the direct ray step.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <map>

#include "common.h"
#include "cosmo.h"
#include "mesh_kernels.h"
#include "raymesh.h"
#include "readout.cuh"

struct hrt_raymesh {
  hrt_raymesh_config cfg{};
  std::map<int64_t, cufftHandle> plans;  // C2C n2d x n2d plans by side
  float2* mesh[2] = {nullptr, nullptr};  // one mesh per half shell
  int64_t cap[2] = {0, 0};               // elements allocated
  float2* mesh_bar[2] = {nullptr, nullptr};  // adjoint: cotangents of the meshes
  int64_t cap_bar[2] = {0, 0};
  double* acc = nullptr;                 // adjoint: drift and plane-weight cotangents (1 + 2 * 512 doubles)
};

namespace hrt {

constexpr int kMaxMeshPlanes = 512;
constexpr int kTileX = 8, kTileY = 32;  // ray-mesh nodes per CTA (x rows, y columns)
constexpr double kMaxCellsPerMeshCell = 64.0;
constexpr float kPif = 3.14159265358979f;

// Light-cone tiling: where a replica's sky axes x, y and z land in the box (field of the sky components, box
// stride, sign and translation in cells).
struct ReplicaMap {
  int64_t str_x, str_y, str_z;
  int sh_x, sh_y, sh_z;
  signed char sg_x, sg_y, sg_z;
  unsigned char c_x, c_y;
};

struct ProjectParams {
  int n;         // 3D mesh side
  int n2d;       // ray-mesh side
  int n_planes;
  int tiled;     // 0: the periodic box; 1: replicas (rep, rmap)
  int kz[kMaxMeshPlanes];        // plane index on the z axis, wrapped into [0, n)
  float w[kMaxMeshPlanes];       // -(2/c) r g(chi) (+-cell) cell^2 / (r^2 x2d^2)
  float pf[kMaxMeshPlanes];      // P = r x2d / cell (3D cells per ray-mesh cell)
  float inv_p[kMaxMeshPlanes];   // 1 / P
  double p[kMaxMeshPlanes];      // P in FP64 for the CTA base
  double qx[kMaxMeshPlanes];     // position of ray-mesh node 0 in 3D cells: (O - r (N/2) x2d) / cell
  double qy[kMaxMeshPlanes];
  unsigned char rep[kMaxMeshPlanes];  // replica of each plane (tiled)
  ReplicaMap rmap[kMaxReplicas];
};

__device__ __forceinline__ int wrap(int i, int n) {
  if (i >= 0 && i < n) return i;
  i %= n;
  return i < 0 ? i + n : i;
}

// Box index along the box axis that receives a sky axis: i -> sgn i + sh (mod n).
__device__ __forceinline__ int box_index(int i, int sgn, int sh, int n) { return wrap(sgn > 0 ? i + sh : sh - i, n); }

template <bool TILED>
__global__ void __launch_bounds__(kTileX * kTileY, 1) raymesh_project_kernel(const float* __restrict__ gx,
                                                                         const float* __restrict__ gy,
                                                                         const float* __restrict__ gz,
                                                                         const __grid_constant__ ProjectParams p,
                                                                         float2* __restrict__ mesh) {
  __shared__ int2 s_base[kMaxMeshPlanes];
  __shared__ float2 s_frac[kMaxMeshPlanes];
  const int mx0 = blockIdx.y * kTileX, my0 = blockIdx.x * kTileY;
  for (int q = threadIdx.x; q < p.n_planes; q += blockDim.x) {
    const double sx = p.qx[q] + mx0 * p.p[q], sy = p.qy[q] + my0 * p.p[q];
    const double fx = floor(sx), fy = floor(sy);
    // |sx|, |sy| are bounded by the host (plane table) well inside the int range
    s_base[q] = make_int2(wrap(static_cast<int>(fx), p.n), wrap(static_cast<int>(fy), p.n));
    s_frac[q] = make_float2(static_cast<float>(sx - fx), static_cast<float>(sy - fy));
  }
  __syncthreads();
  const int dmx = threadIdx.x / kTileY, dmy = threadIdx.x % kTileY;
  const int mx = mx0 + dmx, my = my0 + dmy;
  if (mx >= p.n2d || my >= p.n2d) return;
  const int n = p.n;
  const int64_t nn = n;
  float kx = 0.f, ky = 0.f;
  for (int q = 0; q < p.n_planes; ++q) {
    const float P = p.pf[q], inv = p.inv_p[q];
    const float fx = s_frac[q].x + dmx * P, fy = s_frac[q].y + dmy * P;
    const int ilo = static_cast<int>(floorf(fx - P)), ihi = static_cast<int>(ceilf(fx + P));
    const int jlo = static_cast<int>(floorf(fy - P)), jhi = static_cast<int>(ceilf(fy + P));
    const int bx = s_base[q].x, by = s_base[q].y, kz = p.kz[q];
    // sky-frame fields of the plane: the box itself, or the replica's rotated and translated view of it
    const float* fxp = gx;
    const float* fyp = gy;
    float cx = 1.f, cy = 1.f;
    int64_t zoff = kz;
    const ReplicaMap* m = nullptr;
    if (TILED) {
      m = &p.rmap[p.rep[q]];
      fxp = m->c_x == 0 ? gx : (m->c_x == 1 ? gy : gz);
      fyp = m->c_y == 0 ? gx : (m->c_y == 1 ? gy : gz);
      cx = m->sg_x;
      cy = m->sg_y;
      zoff = box_index(kz, m->sg_z, m->sh_z, n) * m->str_z;
    }
    float sx = 0.f, sy = 0.f;
    for (int i = ilo; i <= ihi; ++i) {
      const float wx = 1.f - fabsf(static_cast<float>(i) - fx) * inv;
      if (wx <= 0.f) continue;
      const int xs = wrap(bx + i, n);
      const int64_t row = TILED ? box_index(xs, m->sg_x, m->sh_x, n) * m->str_x + zoff : static_cast<int64_t>(xs) * nn;
      for (int j = jlo; j <= jhi; ++j) {
        const float wy = 1.f - fabsf(static_cast<float>(j) - fy) * inv;
        if (wy <= 0.f) continue;
        const int ys = wrap(by + j, n);
        const int64_t idx = TILED ? row + box_index(ys, m->sg_y, m->sh_y, n) * m->str_y : (row + ys) * nn + kz;
        const float ww = wx * wy;
        sx += ww * __ldg(fxp + idx);
        sy += ww * __ldg(fyp + idx);
      }
    }
    kx += p.w[q] * cx * sx;
    ky += p.w[q] * cy * sy;
  }
  mesh[static_cast<int64_t>(mx) * p.n2d + my] = make_float2(kx, ky);
}

// sinc(w / 2)^-4 exp(-w^2 / (2 iota^2)) of the signed frequency of index i, w = 2 pi f / n2d.
__device__ __forceinline__ float axis_filter(int i, int n2d, float inv_iota2) {
  const int f = i <= n2d / 2 ? i : i - n2d;
  if (f == 0) return 1.f;
  const float t = static_cast<float>(f) / static_cast<float>(n2d);
  const float s = sinpif(t) / (kPif * t);
  const float s2 = s * s;
  const float w = 2.f * kPif * t;
  return expf(-0.5f * w * w * inv_iota2) / (s2 * s2);
}

// n2d = 2^lg.
__global__ void raymesh_filter_kernel(float2* __restrict__ spec, int lg, float inv_iota2, float scale) {
  const int n2d = 1 << lg;
  const int64_t total = static_cast<int64_t>(n2d) * n2d;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(e >> lg), j = static_cast<int>(e & (n2d - 1));
    const float f = scale * axis_filter(i, n2d, inv_iota2) * axis_filter(j, n2d, inv_iota2);
    float2 v = spec[e];
    v.x *= f;
    v.y *= f;
    spec[e] = v;
  }
}

struct MeshView {
  const float2* k;  // nullptr: the half shell holds no plane (no kick)
  int n2d;
  double inv_x2d;
};

struct RayMeshParams {
  MeshView m[2];
  double drift_d;  // (chi_to - chi_from) / (c chi_mid^2)
  float drift;
  int map_accumulate;
  float map_weight;
};

struct MeshKick {
  float kx, ky;
  float j00, j01, j10, j11;  // dK/dtheta
};

__device__ __forceinline__ float2 corner(const MeshView& m, int i, int j) {
  if (i < 0 || i >= m.n2d || j < 0 || j >= m.n2d) return make_float2(0.f, 0.f);
  return __ldg(m.k + static_cast<int64_t>(i) * m.n2d + j);
}

// Bilinear kick at the angle (thx, thy) and its derivative (zero outside the mesh).
__device__ __forceinline__ MeshKick mesh_kick(const MeshView& m, double thx, double thy) {
  MeshKick h{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (m.k == nullptr) return h;
  const double half = 0.5 * m.n2d;
  const double ux = thx * m.inv_x2d + half, uy = thy * m.inv_x2d + half;
  if (!(ux > -1.0 && ux < m.n2d && uy > -1.0 && uy < m.n2d)) return h;
  const double flx = floor(ux), fly = floor(uy);
  const int ix = static_cast<int>(flx), iy = static_cast<int>(fly);
  const float fx = static_cast<float>(ux - flx), fy = static_cast<float>(uy - fly);
  const float2 v00 = corner(m, ix, iy), v01 = corner(m, ix, iy + 1), v10 = corner(m, ix + 1, iy),
               v11 = corner(m, ix + 1, iy + 1);
  const float gx = 1.f - fx, gy = 1.f - fy;
  h.kx = gx * (gy * v00.x + fy * v01.x) + fx * (gy * v10.x + fy * v11.x);
  h.ky = gx * (gy * v00.y + fy * v01.y) + fx * (gy * v10.y + fy * v11.y);
  const float s = static_cast<float>(m.inv_x2d);
  h.j00 = s * (gy * (v10.x - v00.x) + fy * (v11.x - v01.x));
  h.j01 = s * (gx * (v01.x - v00.x) + fx * (v11.x - v10.x));
  h.j10 = s * (gy * (v10.y - v00.y) + fy * (v11.y - v01.y));
  h.j11 = s * (gx * (v01.y - v00.y) + fx * (v11.y - v10.y));
  return h;
}

__global__ void __launch_bounds__(256, 1) raymesh_ray_kernel(double2* __restrict__ theta, float2* __restrict__ eta,
                                                          float4* __restrict__ Amat, float4* __restrict__ Bmat,
                                                          int64_t nr, const __grid_constant__ RayMeshParams p,
                                                          float* __restrict__ maps) {
  const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (r >= nr) return;
  double2 th = theta[r];
  float2 et = eta[r];
  float4 A = Amat[r], B = Bmat[r];
  MeshKick h = mesh_kick(p.m[0], th.x, th.y);
  et.x += h.kx;
  et.y += h.ky;
  // B += J A (row-major 2x2: x = 11, y = 12, z = 21, w = 22)
  B.x += h.j00 * A.x + h.j01 * A.z;
  B.y += h.j00 * A.y + h.j01 * A.w;
  B.z += h.j10 * A.x + h.j11 * A.z;
  B.w += h.j10 * A.y + h.j11 * A.w;
  th.x += p.drift_d * static_cast<double>(et.x);
  th.y += p.drift_d * static_cast<double>(et.y);
  A.x += p.drift * B.x;
  A.y += p.drift * B.y;
  A.z += p.drift * B.z;
  A.w += p.drift * B.w;
  h = mesh_kick(p.m[1], th.x, th.y);
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

// ---------------------------------------------------------------------------------------------------------
// Adjoint (reverse mode).  The filter is a real, even multiplier in Fourier space, so the filtered mesh is a
// self-adjoint linear map of the deposit and its transpose is the same filter.  The transpose of the projection
// is a gather per 3D node: the bilinear interpolation of the mesh cotangent at the node's projected angle,
// summed over its periodic images and times the plane weight.  The mesh geometry (lambda_lim, x2d, N) is held
// fixed: it is a discretisation choice, not a function of the fields.
// ---------------------------------------------------------------------------------------------------------

// Position of an angle on a mesh with its corner values (the forward's arithmetic).
struct MeshPos {
  bool inside;
  int ix, iy;
  float fx, fy;
  float2 v00, v01, v10, v11;
};

__device__ __forceinline__ MeshPos mesh_locate(const MeshView& m, double thx, double thy) {
  MeshPos c{};
  c.inside = false;
  if (m.k == nullptr) return c;
  const double half = 0.5 * m.n2d;
  const double ux = thx * m.inv_x2d + half, uy = thy * m.inv_x2d + half;
  if (!(ux > -1.0 && ux < m.n2d && uy > -1.0 && uy < m.n2d)) return c;
  const double flx = floor(ux), fly = floor(uy);
  c.inside = true;
  c.ix = static_cast<int>(flx);
  c.iy = static_cast<int>(fly);
  c.fx = static_cast<float>(ux - flx);
  c.fy = static_cast<float>(uy - fly);
  c.v00 = corner(m, c.ix, c.iy);
  c.v01 = corner(m, c.ix, c.iy + 1);
  c.v10 = corner(m, c.ix + 1, c.iy);
  c.v11 = corner(m, c.ix + 1, c.iy + 1);
  return c;
}

__device__ __forceinline__ void corner_add(float2* __restrict__ mbar, int n2d, int i, int j, float a, float b) {
  if (i < 0 || i >= n2d || j < 0 || j >= n2d) return;
  atomicAdd(mbar + static_cast<int64_t>(i) * n2d + j, make_float2(a, b));
}

// Transpose of one half kick at c: the kick's cotangent Kb and the cotangent Jb of dK/dtheta (J as in MeshKick,
// J[c][b] = dK_c / dtheta_b) go to the mesh cotangent through the bilinear and derivative weights, and to the
// angle cotangent thb through J^T Kb and the cross derivative d^2 K / dtheta_x dtheta_y.
__device__ __forceinline__ void mesh_kick_backward(const MeshView& m, float2* __restrict__ mbar, const MeshPos& c,
                                                   const float Kb[2], const float Jb[2][2], float thb[2]) {
  if (!c.inside) return;
  const float s = static_cast<float>(m.inv_x2d);
  const float gx = 1.f - c.fx, gy = 1.f - c.fy, fx = c.fx, fy = c.fy;
  const float j00 = s * (gy * (c.v10.x - c.v00.x) + fy * (c.v11.x - c.v01.x));
  const float j01 = s * (gx * (c.v01.x - c.v00.x) + fx * (c.v11.x - c.v10.x));
  const float j10 = s * (gy * (c.v10.y - c.v00.y) + fy * (c.v11.y - c.v01.y));
  const float j11 = s * (gx * (c.v01.y - c.v00.y) + fx * (c.v11.y - c.v10.y));
  const float hx = s * s * (c.v11.x - c.v10.x - c.v01.x + c.v00.x);
  const float hy = s * s * (c.v11.y - c.v10.y - c.v01.y + c.v00.y);
  thb[0] += j00 * Kb[0] + j10 * Kb[1] + Jb[0][1] * hx + Jb[1][1] * hy;
  thb[1] += j01 * Kb[0] + j11 * Kb[1] + Jb[0][0] * hx + Jb[1][0] * hy;
  // corner (di, dj): value weight w, weights dJx, dJy of J[.][0] and J[.][1]
  const float w[4] = {gx * gy, gx * fy, fx * gy, fx * fy};
  const float dx[4] = {-s * gy, -s * fy, s * gy, s * fy};
  const float dy[4] = {-s * gx, s * gx, -s * fx, s * fx};
  for (int k = 0; k < 4; ++k) {
    const float a = Kb[0] * w[k] + Jb[0][0] * dx[k] + Jb[0][1] * dy[k];
    const float b = Kb[1] * w[k] + Jb[1][0] * dx[k] + Jb[1][1] * dy[k];
    corner_add(mbar, m.n2d, c.ix + (k >> 1), c.iy + (k & 1), a, b);
  }
}

__device__ __forceinline__ void block_sum_add(double v, double* __restrict__ out) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out, v);
}

__global__ void __launch_bounds__(256) raymesh_ray_adjoint_kernel(
    const double2* __restrict__ theta, const float2* __restrict__ eta, const float4* __restrict__ Amat,
    const float4* __restrict__ Bmat, int64_t nr, const __grid_constant__ RayMeshParams p,
    double2* __restrict__ theta_bar, float2* __restrict__ eta_bar, float4* __restrict__ A_bar,
    float4* __restrict__ B_bar, float2* __restrict__ mbar0, float2* __restrict__ mbar1, double* __restrict__ drift_bar) {
  const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const bool active = r < nr;
  double db = 0.0;
  if (active) {
    const double2 th0 = theta[r];
    const float2 et0 = eta[r];
    const float4 A0v = Amat[r], B0v = Bmat[r];
    const float A0[2][2] = {{A0v.x, A0v.y}, {A0v.z, A0v.w}};
    const float B0[2][2] = {{B0v.x, B0v.y}, {B0v.z, B0v.w}};
    // forward recompute (the arithmetic of raymesh_ray_kernel)
    const MeshKick h1 = mesh_kick(p.m[0], th0.x, th0.y);
    const float J1[2][2] = {{h1.j00, h1.j01}, {h1.j10, h1.j11}};
    const float eta1[2] = {et0.x + h1.kx, et0.y + h1.ky};
    float B1[2][2], A1[2][2];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) B1[a][b] = B0[a][b] + (J1[a][0] * A0[0][b] + J1[a][1] * A0[1][b]);
    const double th1x = th0.x + p.drift_d * static_cast<double>(eta1[0]);
    const double th1y = th0.y + p.drift_d * static_cast<double>(eta1[1]);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) A1[a][b] = A0[a][b] + p.drift * B1[a][b];
    const MeshKick h2 = mesh_kick(p.m[1], th1x, th1y);
    const float J2[2][2] = {{h2.j00, h2.j01}, {h2.j10, h2.j11}};
    // backward
    const double2 thbv = theta_bar[r];
    const float2 etbv = eta_bar[r];
    const float4 Abv = A_bar[r], Bbv = B_bar[r];
    float Ab[2][2] = {{Abv.x, Abv.y}, {Abv.z, Abv.w}};
    float Bb[2][2] = {{Bbv.x, Bbv.y}, {Bbv.z, Bbv.w}};
    float etb[2] = {etbv.x, etbv.y};
    float thb[2] = {static_cast<float>(thbv.x), static_cast<float>(thbv.y)};
    float Jb[2][2];
    // B2 = B1 + J2 A1 and eta2 = eta1 + K2(theta1)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) Jb[a][b] = Bb[a][0] * A1[b][0] + Bb[a][1] * A1[b][1];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) Ab[a][b] += J2[0][a] * Bb[0][b] + J2[1][a] * Bb[1][b];
    mesh_kick_backward(p.m[1], mbar1, mesh_locate(p.m[1], th1x, th1y), etb, Jb, thb);
    // A1 = A0 + d B1, theta1 = theta0 + d eta1
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        Bb[a][b] += p.drift * Ab[a][b];
        db += static_cast<double>(Ab[a][b]) * B1[a][b];
      }
    etb[0] += static_cast<float>(p.drift_d) * thb[0];
    etb[1] += static_cast<float>(p.drift_d) * thb[1];
    db += static_cast<double>(thb[0]) * eta1[0] + static_cast<double>(thb[1]) * eta1[1];
    // B1 = B0 + J1 A0 and eta1 = eta0 + K1(theta0)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) Jb[a][b] = Bb[a][0] * A0[b][0] + Bb[a][1] * A0[b][1];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) Ab[a][b] += J1[0][a] * Bb[0][b] + J1[1][a] * Bb[1][b];
    mesh_kick_backward(p.m[0], mbar0, mesh_locate(p.m[0], th0.x, th0.y), etb, Jb, thb);
    theta_bar[r] = make_double2(thb[0], thb[1]);
    eta_bar[r] = make_float2(etb[0], etb[1]);
    A_bar[r] = make_float4(Ab[0][0], Ab[0][1], Ab[1][0], Ab[1][1]);
    B_bar[r] = make_float4(Bb[0][0], Bb[0][1], Bb[1][0], Bb[1][1]);
  }
  block_sum_add(db, drift_bar);
}

// Transpose of the projection: one thread per sky-frame 3D node (i, j) of plane blockIdx.z.  S is the bilinear
// interpolation of the (filtered) mesh cotangent at the node's projected angle, summed over the node's periodic
// images.  Untiled, the node is the box node and w_p S goes to the (x, y) field cotangents.  Tiled, the node lives
// in the plane's replica: sky component a was read from box field perm(a) with sign s_a at the replica's box
// node, so w_p s_a S_a goes to that field's cotangent there.  The dot product of the fields read with S adds to
// dL/dw_p.
template <bool TILED>
__global__ void __launch_bounds__(256) raymesh_project_adjoint_kernel(const float* __restrict__ gx,
                                                                     const float* __restrict__ gy,
                                                                     const float* __restrict__ gz,
                                                                     const __grid_constant__ ProjectParams p,
                                                                     const float2* __restrict__ mbar,
                                                                     float* __restrict__ gxb, float* __restrict__ gyb,
                                                                     float* __restrict__ gzb,
                                                                     double* __restrict__ plane_bar) {
  const int q = blockIdx.z;
  const int i = blockIdx.y * kTileX + threadIdx.x / kTileY, j = blockIdx.x * kTileY + threadIdx.x % kTileY;
  const int n = p.n, n2d = p.n2d;
  double part = 0.0;
  if (i < n && j < n) {
    const double P = p.p[q], inv = 1.0 / P;
    // u = (node + image n - Q) / P on each axis; the images whose u reaches (-1, n2d)
    const double ux0 = (i - p.qx[q]) * inv, uy0 = (j - p.qy[q]) * inv, step = n * inv;
    const int ia0 = static_cast<int>(ceil((-1.0 - ux0) / step)), ia1 = static_cast<int>(floor((n2d - ux0) / step));
    const int ib0 = static_cast<int>(ceil((-1.0 - uy0) / step)), ib1 = static_cast<int>(floor((n2d - uy0) / step));
    float sx = 0.f, sy = 0.f;
    for (int ia = ia0; ia <= ia1; ++ia) {
      const double ux = ux0 + ia * step;
      if (!(ux > -1.0 && ux < n2d)) continue;
      const double flx = floor(ux);
      const int mx = static_cast<int>(flx);
      const float fx = static_cast<float>(ux - flx);
      for (int ib = ib0; ib <= ib1; ++ib) {
        const double uy = uy0 + ib * step;
        if (!(uy > -1.0 && uy < n2d)) continue;
        const double fly = floor(uy);
        const int my = static_cast<int>(fly);
        const float fy = static_cast<float>(uy - fly);
        const float w[4] = {(1.f - fx) * (1.f - fy), (1.f - fx) * fy, fx * (1.f - fy), fx * fy};
        for (int k = 0; k < 4; ++k) {
          const int a = mx + (k >> 1), b = my + (k & 1);
          if (a < 0 || a >= n2d || b < 0 || b >= n2d) continue;
          const float2 v = __ldg(mbar + static_cast<int64_t>(a) * n2d + b);
          sx += w[k] * v.x;
          sy += w[k] * v.y;
        }
      }
    }
    if ((sx != 0.f || sy != 0.f) && TILED) {
      const ReplicaMap& m = p.rmap[p.rep[q]];
      const int64_t idx = box_index(i, m.sg_x, m.sh_x, n) * m.str_x + box_index(j, m.sg_y, m.sh_y, n) * m.str_y +
                          box_index(p.kz[q], m.sg_z, m.sh_z, n) * m.str_z;
      const float* fxp = m.c_x == 0 ? gx : (m.c_x == 1 ? gy : gz);
      const float* fyp = m.c_y == 0 ? gx : (m.c_y == 1 ? gy : gz);
      float* bxp = m.c_x == 0 ? gxb : (m.c_x == 1 ? gyb : gzb);
      float* byp = m.c_y == 0 ? gxb : (m.c_y == 1 ? gyb : gzb);
      const float tx = m.sg_x * sx, ty = m.sg_y * sy;
      atomicAdd(bxp + idx, p.w[q] * tx);
      atomicAdd(byp + idx, p.w[q] * ty);
      part = static_cast<double>(__ldg(fxp + idx)) * tx + static_cast<double>(__ldg(fyp + idx)) * ty;
    } else if (sx != 0.f || sy != 0.f) {
      const int64_t idx = (static_cast<int64_t>(i) * n + j) * n + p.kz[q];
      atomicAdd(gxb + idx, p.w[q] * sx);
      atomicAdd(gyb + idx, p.w[q] * sy);
      part = static_cast<double>(__ldg(gx + idx)) * sx + static_cast<double>(__ldg(gy + idx)) * sy;
    }
  }
  block_sum_add(part, plane_bar + q);
}

// ---------------------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------------------

static hrt_status cufft_check(cufftResult r, const char* what) {
  if (r == CUFFT_SUCCESS) return HRT_OK;
  return fail(r == CUFFT_ALLOC_FAILED ? HRT_ERR_OOM : HRT_ERR_CUDA, "cuFFT %s failed (%d)", what, static_cast<int>(r));
}

static hrt_status check_config(const hrt_raymesh_config& c) {
  if (!(c.iota > 0.0 && c.iota <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "iota must be in (0, 1]");
  if (!(c.p_min >= 0.0) || !std::isfinite(c.p_min)) return fail(HRT_ERR_INVALID_ARG, "p_min must be >= 0");
  if (!(c.mu > 0.0) || !std::isfinite(c.mu)) return fail(HRT_ERR_INVALID_ARG, "mu must be > 0");
  if (c.m_pix < 1) return fail(HRT_ERR_INVALID_ARG, "m_pix must be >= 1");
  if (c.n2d_max < 0 || c.n2d_max > 32768) return fail(HRT_ERR_INVALID_ARG, "n2d_max must be in [0, 32768]");
  return HRT_OK;
}

// lambda_lim, x2d and the power-of-two side of the ray mesh of the half shell [chi_a, chi_b) (App. C).
static hrt_status geometry(const hrt_raymesh_config& c, double chi_a, double chi_b, double cell, double& lam,
                           double& x2d, int64_t& n2d) {
  HRT_TRY(check_config(c));
  const double rsum = std::fabs(chi_a) + std::fabs(chi_b);
  if (!(cell > 0.0) || !(rsum > 0.0) || !std::isfinite(rsum)) return fail(HRT_ERR_INVALID_ARG, "bad shell or cell");
  lam = std::max(2.0 * cell / rsum, c.mu);
  x2d = c.iota * lam;
  const double need = std::ceil(static_cast<double>(c.m_pix) * c.mu / x2d + c.p_min / c.iota);
  const int64_t cap = c.n2d_max > 0 ? c.n2d_max : 8192;
  n2d = 1;
  while (n2d < need) {
    n2d *= 2;
    if (n2d > cap) return fail(HRT_ERR_INVALID_ARG, "ray mesh of side >= %.0f exceeds n2d_max = %lld", need,
                               static_cast<long long>(cap));
  }
  return HRT_OK;
}

// Plane table of the half shell (FP64 on the host): the node planes z = kz cell with
// min(chi_a, chi_b) <= chi = z - O_z < max(chi_a, chi_b), chi > 0, inside the geometry's window.
static hrt_status plane_table(const hrt_ray_geom& g, double chi_a, double chi_b, double a_ref, double omega_m,
                              double x2d, int64_t n2d, ProjectParams& p, double* w64 = nullptr,
                              double* chi64 = nullptr) {
  const double cell = g.box / g.n;
  const double lo = std::min(chi_a, chi_b), hi = std::max(chi_a, chi_b);
  const double sgn = chi_b >= chi_a ? 1.0 : -1.0;
  const double oz = g.observer[2];
  Cosmo cosmo(omega_m);
  const double d1_ref = a_ref > 0.0 ? cosmo.D1(a_ref) : 1.0;
  p.n = static_cast<int>(g.n);
  p.n2d = static_cast<int>(n2d);
  p.n_planes = 0;
  p.tiled = g.n_replicas > 0 ? 1 : 0;
  if (p.tiled) {
    if (g.n_replicas > kMaxReplicas || !g.replica_perm || !g.replica_sign || !g.replica_shift)
      return fail(HRT_ERR_INVALID_ARG, "tiling needs 1..%d replicas with their perm, sign and shift tables", kMaxReplicas);
    const int64_t nn = g.n;
    auto stride = [nn](int b) { return b == 0 ? nn * nn : (b == 1 ? nn : int64_t{1}); };
    for (int k = 0; k < g.n_replicas; ++k) {
      const int32_t* pm = g.replica_perm + 3 * k;
      const int32_t* sg = g.replica_sign + 3 * k;
      const int32_t* sh = g.replica_shift + 3 * k;
      int seen = 0;
      for (int a = 0; a < 3; ++a) {
        if (pm[a] < 0 || pm[a] > 2 || (sg[a] != 1 && sg[a] != -1) || sh[a] < 0 || sh[a] >= g.n)
          return fail(HRT_ERR_INVALID_ARG, "replica %d: bad axis, sign or shift", k);
        seen |= 1 << pm[a];
      }
      if (seen != 7) return fail(HRT_ERR_INVALID_ARG, "replica %d: the axes are not a permutation", k);
      ReplicaMap& m = p.rmap[k];
      m.c_x = static_cast<unsigned char>(pm[0]);
      m.c_y = static_cast<unsigned char>(pm[1]);
      m.str_x = stride(pm[0]);
      m.str_y = stride(pm[1]);
      m.str_z = stride(pm[2]);
      m.sg_x = static_cast<signed char>(sg[0]);
      m.sg_y = static_cast<signed char>(sg[1]);
      m.sg_z = static_cast<signed char>(sg[2]);
      m.sh_x = sh[pm[0]];
      m.sh_y = sh[pm[1]];
      m.sh_z = sh[pm[2]];
    }
  }
  const int64_t k0 = static_cast<int64_t>(std::ceil((oz + lo) / cell)) - 1;
  const int64_t k1 = static_cast<int64_t>(std::ceil((oz + hi) / cell));
  for (int64_t kz = k0; kz <= k1; ++kz) {
    const double chi = kz * cell - oz;
    if (!(lo <= chi && chi < hi && chi > 0.0)) continue;
    if (!(g.window_lo <= chi && chi < g.window_hi)) continue;
    if (p.n_planes >= kMaxMeshPlanes) return fail(HRT_ERR_INVALID_ARG, "more than %d mesh planes in a half shell", kMaxMeshPlanes);
    const double r = chi;
    double gw = 1.0;
    if (a_ref > 0.0) {
      const double a = cosmo.a_of_chi(chi);
      gw = cosmo.D1(a) / d1_ref * a_ref / a;
    }
    const double P = r * x2d / cell;
    if (P > kMaxCellsPerMeshCell) return fail(HRT_ERR_INVALID_ARG, "a ray-mesh cell spans %.1f mesh cells (> %.0f)", P, kMaxCellsPerMeshCell);
    const double qx = (g.observer[0] - r * (0.5 * n2d) * x2d) / cell;
    const double qy = (g.observer[1] - r * (0.5 * n2d) * x2d) / cell;
    // the CTA bases qx + m0 P must stay well inside the int range
    if (std::fabs(qx) + n2d * P > 1.0e9 || std::fabs(qy) + n2d * P > 1.0e9) return fail(HRT_ERR_INVALID_ARG, "ray mesh too far from the box");
    int64_t rep = 0;
    if (p.tiled) {
      // the plane z = kz cell lies in replica floor(kz / n)
      rep = kz >= 0 ? kz / g.n : -1;
      if (rep < 0 || rep >= g.n_replicas)
        return fail(HRT_ERR_INVALID_ARG, "mesh plane at chi = %g is outside the %d replicas", chi, g.n_replicas);
    }
    const int q = p.n_planes++;
    p.rep[q] = static_cast<unsigned char>(rep);
    int64_t kzw = kz % g.n;
    if (kzw < 0) kzw += g.n;
    p.kz[q] = static_cast<int>(kzw);
    const double wq = -(2.0 / kCLight) * r * gw * sgn * cell * cell * cell / (r * r * x2d * x2d);
    p.w[q] = static_cast<float>(wq);
    if (w64) w64[q] = wq;
    if (chi64) chi64[q] = chi;
    p.pf[q] = static_cast<float>(P);
    p.inv_p[q] = static_cast<float>(1.0 / P);
    p.p[q] = P;
    p.qx[q] = qx;
    p.qy[q] = qy;
  }
  return HRT_OK;
}

static hrt_status check_geom(const hrt_ray_geom* g, bool tiled) {
  if (!g) return fail(HRT_ERR_INVALID_ARG, "geometry is NULL");
  if (g->n < 2 || g->n > 8192 || !(g->box > 0.0)) return fail(HRT_ERR_INVALID_ARG, "bad mesh or box");
  if (!tiled && g->n_replicas != 0) return fail(HRT_ERR_INVALID_ARG, "a tiled geometry needs the tiled call (three fields)");
  if (tiled && g->n_replicas < 1) return fail(HRT_ERR_INVALID_ARG, "the tiled call needs n_replicas >= 1");
  return HRT_OK;
}

static hrt_status ensure_mesh(hrt_raymesh* rm, int h, int64_t elems, cudaStream_t s) {
  if (rm->cap[h] >= elems) return HRT_OK;
  if (rm->mesh[h]) {
    cudaFreeAsync(rm->mesh[h], s);
    rm->mesh[h] = nullptr;
    rm->cap[h] = 0;
  }
  HRT_TRY(device_alloc(reinterpret_cast<void**>(&rm->mesh[h]), static_cast<size_t>(elems) * sizeof(float2), s, "ray mesh"));
  rm->cap[h] = elems;
  return HRT_OK;
}

static hrt_status plan_for(hrt_raymesh* rm, int64_t n2d, cudaStream_t s, cufftHandle& plan) {
  auto it = rm->plans.find(n2d);
  if (it == rm->plans.end()) {
    cufftHandle h;
    HRT_TRY(cufft_check(cufftPlan2d(&h, static_cast<int>(n2d), static_cast<int>(n2d), CUFFT_C2C), "plan"));
    it = rm->plans.emplace(n2d, h).first;
  }
  plan = it->second;
  return cufft_check(cufftSetStream(plan, s), "set stream");
}

// In place: C2C forward, the deconvolution and smoothing (with the 1 / N^2 of the inverse), C2C inverse.  The
// same operation is its own transpose (real, even multiplier).
static hrt_status filter_mesh(hrt_raymesh* rm, float2* mesh, int64_t n2d, cudaStream_t s) {
  cufftHandle plan;
  HRT_TRY(plan_for(rm, n2d, s, plan));
  auto* c = reinterpret_cast<cufftComplex*>(mesh);
  HRT_TRY(cufft_check(cufftExecC2C(plan, c, c, CUFFT_FORWARD), "forward"));
  const int64_t total = n2d * n2d;
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 152 * 16));
  int lg = 0;
  while ((int64_t{1} << lg) < n2d) ++lg;
  raymesh_filter_kernel<<<blocks, 256, 0, s>>>(mesh, lg,
                                               static_cast<float>(1.0 / (rm->cfg.iota * rm->cfg.iota)),
                                               static_cast<float>(1.0 / static_cast<double>(total)));
  HRT_LAUNCHED("raymesh_filter_kernel");
  return cufft_check(cufftExecC2C(plan, c, c, CUFFT_INVERSE), "inverse");
}

// Builds the filtered ray mesh of the half shell [chi_a, chi_b) in rm->mesh[h]; view.k == nullptr when the
// shell holds no plane.
static hrt_status build_mesh(hrt_raymesh* rm, int h, const float* gx, const float* gy, const float* gz,
                             const hrt_ray_geom& g, double chi_a, double chi_b, double a_ref, double omega_m,
                             cudaStream_t s, MeshView& view) {
  static thread_local ProjectParams p;
  double lam, x2d;
  int64_t n2d;
  HRT_TRY(geometry(rm->cfg, chi_a, chi_b, g.box / g.n, lam, x2d, n2d));
  HRT_TRY(plane_table(g, chi_a, chi_b, a_ref, omega_m, x2d, n2d, p));
  view.n2d = static_cast<int>(n2d);
  view.inv_x2d = 1.0 / x2d;
  view.k = nullptr;
  if (p.n_planes == 0) return HRT_OK;
  HRT_TRY(ensure_mesh(rm, h, n2d * n2d, s));
  float2* mesh = rm->mesh[h];
  const dim3 grid(static_cast<unsigned>((n2d + kTileY - 1) / kTileY), static_cast<unsigned>((n2d + kTileX - 1) / kTileX));
  if (p.tiled) {
    if (!gz) return fail(HRT_ERR_INVALID_ARG, "light-cone tiling needs the third gradient component");
    raymesh_project_kernel<true><<<grid, kTileX * kTileY, 0, s>>>(gx, gy, gz, p, mesh);
  } else {
    raymesh_project_kernel<false><<<grid, kTileX * kTileY, 0, s>>>(gx, gy, gz, p, mesh);
  }
  HRT_LAUNCHED("raymesh_project_kernel");
  HRT_TRY(filter_mesh(rm, mesh, n2d, s));
  view.k = mesh;
  return HRT_OK;
}

const hrt_raymesh_config& raymesh_config_of(const hrt_raymesh* rm) { return rm->cfg; }

hrt_status raymesh_step(hrt_raymesh* rm, const hrt_rays& rays, const float* gx, const float* gy, const float* gz,
                        const hrt_ray_geom& g, double chi_from, double chi_to, double a_ref, double omega_m,
                        float* maps, int accumulate, float weight, cudaStream_t s) {
  const double chi_mid = 0.5 * (chi_from + chi_to);
  if (!(chi_mid > 0.0)) return fail(HRT_ERR_INVALID_ARG, "shell midpoint must be at chi > 0");
  RayMeshParams p{};
  HRT_TRY(build_mesh(rm, 0, gx, gy, gz, g, chi_from, chi_mid, a_ref, omega_m, s, p.m[0]));
  HRT_TRY(build_mesh(rm, 1, gx, gy, gz, g, chi_mid, chi_to, a_ref, omega_m, s, p.m[1]));
  p.drift_d = (chi_to - chi_from) / (kCLight * chi_mid * chi_mid);
  p.drift = static_cast<float>(p.drift_d);
  p.map_accumulate = accumulate;
  p.map_weight = weight;
  if (rays.n_rays == 0) return HRT_OK;
  raymesh_ray_kernel<<<blocks_for(rays.n_rays, 256), 256, 0, s>>>(
      reinterpret_cast<double2*>(rays.theta), reinterpret_cast<float2*>(rays.eta), reinterpret_cast<float4*>(rays.A),
      reinterpret_cast<float4*>(rays.B), rays.n_rays, p, maps);
  HRT_LAUNCHED("raymesh_ray_kernel");
  return HRT_OK;
}

static hrt_status ensure_bar(hrt_raymesh* rm, int h, int64_t elems, cudaStream_t s) {
  if (!rm->acc) HRT_TRY(device_alloc(reinterpret_cast<void**>(&rm->acc), (1 + 2 * kMaxMeshPlanes) * sizeof(double), s, "adjoint sums"));
  if (rm->cap_bar[h] >= elems) return HRT_OK;
  if (rm->mesh_bar[h]) {
    cudaFreeAsync(rm->mesh_bar[h], s);
    rm->mesh_bar[h] = nullptr;
    rm->cap_bar[h] = 0;
  }
  HRT_TRY(device_alloc(reinterpret_cast<void**>(&rm->mesh_bar[h]), static_cast<size_t>(elems) * sizeof(float2), s, "ray-mesh cotangent"));
  rm->cap_bar[h] = elems;
  return HRT_OK;
}

// Transpose of filter + projection for one half shell: mbar (filtered-mesh cotangent, overwritten) to the field
// cotangents and dL/dw_p (device, per plane); gz, gzb are read only through a tiled light cone.
static hrt_status shell_adjoint(hrt_raymesh* rm, const float* gx, const float* gy, const float* gz,
                                const ProjectParams& p, float2* mbar, float* gxb, float* gyb, float* gzb,
                                double* plane_bar, cudaStream_t s) {
  if (p.n_planes == 0) return HRT_OK;
  HRT_TRY(filter_mesh(rm, mbar, p.n2d, s));
  const dim3 grid(static_cast<unsigned>((p.n + kTileY - 1) / kTileY), static_cast<unsigned>((p.n + kTileX - 1) / kTileX),
                  static_cast<unsigned>(p.n_planes));
  auto* kernel = p.tiled ? raymesh_project_adjoint_kernel<true> : raymesh_project_adjoint_kernel<false>;
  kernel<<<grid, kTileX * kTileY, 0, s>>>(gx, gy, gz, p, mbar, gxb, gyb, gzb, plane_bar);
  HRT_LAUNCHED("raymesh_project_adjoint_kernel");
  return HRT_OK;
}

static hrt_status read_sums(hrt_raymesh* rm, double* host, size_t count, cudaStream_t s) {
  HRT_TRY(cuda_status(cudaMemcpyAsync(host, rm->acc, count * sizeof(double), cudaMemcpyDeviceToHost, s), "adjoint sums"));
  return cuda_status(cudaStreamSynchronize(s), "adjoint sync");
}

static hrt_status kick_adjoint_call(hrt_raymesh* rm, const float* gx, const float* gy, const float* gz,
                                    const float* mesh_bar, const hrt_ray_geom* geom, double chi_a, double chi_b,
                                    double a_ref, double omega_m, float* gxb, float* gyb, float* gzb,
                                    double* plane_bar_host, void* stream) {
  if (!rm || !gx || !gy || !mesh_bar || !gxb || !gyb) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if ((gz == nullptr) != (gzb == nullptr)) return fail(HRT_ERR_INVALID_ARG, "grad_z and gz_bar go together");
  HRT_TRY(check_geom(geom, gz != nullptr));
  if (!(omega_m > 0.0 && omega_m <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "omega_m must be in (0, 1]");
  cudaStream_t s = as_stream(stream);
  static thread_local ProjectParams p;
  double lam, x2d;
  int64_t n2d;
  HRT_TRY(geometry(rm->cfg, chi_a, chi_b, geom->box / geom->n, lam, x2d, n2d));
  HRT_TRY(plane_table(*geom, chi_a, chi_b, a_ref, omega_m, x2d, n2d, p));
  HRT_TRY(ensure_bar(rm, 0, n2d * n2d, s));
  HRT_TRY(cuda_status(cudaMemsetAsync(rm->acc, 0, (1 + 2 * kMaxMeshPlanes) * sizeof(double), s), "clear sums"));
  HRT_TRY(cuda_status(cudaMemcpyAsync(rm->mesh_bar[0], mesh_bar, static_cast<size_t>(n2d) * n2d * sizeof(float2),
                                      cudaMemcpyDeviceToDevice, s), "copy mesh cotangent"));
  HRT_TRY(shell_adjoint(rm, gx, gy, gz, p, rm->mesh_bar[0], gxb, gyb, gzb, rm->acc + 1, s));
  std::vector<double> h(1 + kMaxMeshPlanes);
  HRT_TRY(read_sums(rm, h.data(), h.size(), s));
  if (plane_bar_host)
    for (int q = 0; q < p.n_planes; ++q) plane_bar_host[q] += h[1 + q];
  return HRT_OK;
}

static hrt_status step_adjoint_call(hrt_raymesh* rm, const hrt_rays* rays, const float* gx, const float* gy,
                                    const float* gz, const hrt_ray_geom* geom, double chi_from, double chi_to,
                                    double a_ref, double omega_m, const hrt_rays* bar, float* gxb, float* gyb,
                                    float* gzb, double* plane_bar_host, double* drift_bar_host, void* stream) {
  if (!rm || !gx || !gy || !gxb || !gyb || !rays || !bar) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if ((gz == nullptr) != (gzb == nullptr)) return fail(HRT_ERR_INVALID_ARG, "grad_z and gz_bar go together");
  if (rays->n_rays < 0 || bar->n_rays != rays->n_rays ||
      (rays->n_rays > 0 && (!rays->theta || !rays->eta || !rays->A || !rays->B || !bar->theta || !bar->eta ||
                            !bar->A || !bar->B)))
    return fail(HRT_ERR_INVALID_ARG, "bad ray state or cotangent");
  HRT_TRY(check_geom(geom, gz != nullptr));
  if (!(omega_m > 0.0 && omega_m <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "omega_m must be in (0, 1]");
  const double chi_mid = 0.5 * (chi_from + chi_to);
  if (!(chi_mid > 0.0)) return fail(HRT_ERR_INVALID_ARG, "shell midpoint must be at chi > 0");
  cudaStream_t s = as_stream(stream);
  RayMeshParams rp{};
  HRT_TRY(build_mesh(rm, 0, gx, gy, gz, *geom, chi_from, chi_mid, a_ref, omega_m, s, rp.m[0]));
  HRT_TRY(build_mesh(rm, 1, gx, gy, gz, *geom, chi_mid, chi_to, a_ref, omega_m, s, rp.m[1]));
  rp.drift_d = (chi_to - chi_from) / (kCLight * chi_mid * chi_mid);
  rp.drift = static_cast<float>(rp.drift_d);
  for (int h = 0; h < 2; ++h) {
    const int64_t e = static_cast<int64_t>(rp.m[h].n2d) * rp.m[h].n2d;
    HRT_TRY(ensure_bar(rm, h, e, s));
    HRT_TRY(cuda_status(cudaMemsetAsync(rm->mesh_bar[h], 0, static_cast<size_t>(e) * sizeof(float2), s), "clear cotangent"));
  }
  HRT_TRY(cuda_status(cudaMemsetAsync(rm->acc, 0, (1 + 2 * kMaxMeshPlanes) * sizeof(double), s), "clear sums"));
  if (rays->n_rays > 0) {
    raymesh_ray_adjoint_kernel<<<blocks_for(rays->n_rays, 256), 256, 0, s>>>(
        reinterpret_cast<const double2*>(rays->theta), reinterpret_cast<const float2*>(rays->eta),
        reinterpret_cast<const float4*>(rays->A), reinterpret_cast<const float4*>(rays->B), rays->n_rays, rp,
        reinterpret_cast<double2*>(bar->theta), reinterpret_cast<float2*>(bar->eta), reinterpret_cast<float4*>(bar->A),
        reinterpret_cast<float4*>(bar->B), rm->mesh_bar[0], rm->mesh_bar[1], rm->acc);
    HRT_LAUNCHED("raymesh_ray_adjoint_kernel");
  }
  static thread_local ProjectParams p;
  const double lo[2] = {chi_from, chi_mid}, hi[2] = {chi_mid, chi_to};
  int counts[2] = {0, 0};
  for (int h = 0; h < 2; ++h) {
    if (rp.m[h].k == nullptr) continue;
    double lam, x2d;
    int64_t n2d;
    HRT_TRY(geometry(rm->cfg, lo[h], hi[h], geom->box / geom->n, lam, x2d, n2d));
    HRT_TRY(plane_table(*geom, lo[h], hi[h], a_ref, omega_m, x2d, n2d, p));
    counts[h] = p.n_planes;
    HRT_TRY(shell_adjoint(rm, gx, gy, gz, p, rm->mesh_bar[h], gxb, gyb, gzb, rm->acc + 1 + h * kMaxMeshPlanes, s));
  }
  std::vector<double> sums(1 + 2 * kMaxMeshPlanes);
  HRT_TRY(read_sums(rm, sums.data(), sums.size(), s));
  if (drift_bar_host) drift_bar_host[0] += sums[0];
  if (plane_bar_host)
    for (int h = 0; h < 2; ++h)
      for (int q = 0; q < counts[h]; ++q) plane_bar_host[h * kMaxMeshPlanes + q] += sums[1 + h * kMaxMeshPlanes + q];
  return HRT_OK;
}

static hrt_status kick_call(hrt_raymesh* rm, const float* grad_x, const float* grad_y, const float* grad_z,
                            const hrt_ray_geom* geom, double chi_a, double chi_b, double a_ref, double omega_m,
                            float* mesh, void* stream) {
  if (!rm || !grad_x || !grad_y || !mesh) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  HRT_TRY(check_geom(geom, grad_z != nullptr));
  if (!(omega_m > 0.0 && omega_m <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "omega_m must be in (0, 1]");
  cudaStream_t s = as_stream(stream);
  MeshView v{};
  HRT_TRY(build_mesh(rm, 0, grad_x, grad_y, grad_z, *geom, chi_a, chi_b, a_ref, omega_m, s, v));
  const size_t bytes = static_cast<size_t>(v.n2d) * v.n2d * sizeof(float2);
  if (v.k == nullptr) return cuda_status(cudaMemsetAsync(mesh, 0, bytes, s), "clear ray mesh");
  return cuda_status(cudaMemcpyAsync(mesh, v.k, bytes, cudaMemcpyDeviceToDevice, s), "copy ray mesh");
}

static hrt_status step_call(hrt_raymesh* rm, const hrt_rays* rays, const float* grad_x, const float* grad_y,
                            const float* grad_z, const hrt_ray_geom* geom, double chi_from, double chi_to,
                            double a_ref, double omega_m, float* maps, void* stream) {
  if (!rm || !grad_x || !grad_y) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (!rays) return fail(HRT_ERR_INVALID_ARG, "rays is NULL");
  if (rays->n_rays < 0 || (rays->n_rays > 0 && (!rays->theta || !rays->eta || !rays->A || !rays->B)))
    return fail(HRT_ERR_INVALID_ARG, "bad ray state");
  HRT_TRY(check_geom(geom, grad_z != nullptr));
  if (!(omega_m > 0.0 && omega_m <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "omega_m must be in (0, 1]");
  return raymesh_step(rm, *rays, grad_x, grad_y, grad_z, *geom, chi_from, chi_to, a_ref, omega_m, maps, 0, 1.f,
                      as_stream(stream));
}

}  // namespace hrt

using namespace hrt;

extern "C" {

hrt_status hrt_raymesh_geometry(const hrt_raymesh_config* cfg, double chi_a, double chi_b, double cell,
                                double* lambda_lim, double* x2d, int64_t* n2d) {
  if (!cfg || !lambda_lim || !x2d || !n2d) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  return geometry(*cfg, chi_a, chi_b, cell, *lambda_lim, *x2d, *n2d);
}

hrt_status hrt_raymesh_create(const hrt_raymesh_config* cfg, hrt_raymesh** out) {
  if (!cfg || !out) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  HRT_TRY(check_config(*cfg));
  auto* rm = new hrt_raymesh;
  rm->cfg = *cfg;
  *out = rm;
  return HRT_OK;
}

hrt_status hrt_raymesh_destroy(hrt_raymesh* rm) {
  if (!rm) return HRT_OK;
  cudaDeviceSynchronize();
  for (auto& kv : rm->plans) cufftDestroy(kv.second);
  for (int h = 0; h < 2; ++h)
    if (rm->mesh[h]) cudaFreeAsync(rm->mesh[h], nullptr);
  cudaDeviceSynchronize();
  cudaGetLastError();
  delete rm;
  return HRT_OK;
}

hrt_status hrt_raymesh_kick(hrt_raymesh* rm, const float* grad_x, const float* grad_y, const hrt_ray_geom* geom,
                            double chi_a, double chi_b, double a_ref, double omega_m, float* mesh, void* stream) {
  return kick_call(rm, grad_x, grad_y, nullptr, geom, chi_a, chi_b, a_ref, omega_m, mesh, stream);
}

hrt_status hrt_raymesh_kick_tiled(hrt_raymesh* rm, const float* grad_x, const float* grad_y, const float* grad_z,
                                  const hrt_ray_geom* geom, double chi_a, double chi_b, double a_ref, double omega_m,
                                  float* mesh, void* stream) {
  if (!grad_z) return fail(HRT_ERR_INVALID_ARG, "grad_z is NULL");
  return kick_call(rm, grad_x, grad_y, grad_z, geom, chi_a, chi_b, a_ref, omega_m, mesh, stream);
}

hrt_status hrt_raymesh_ray_step(hrt_raymesh* rm, const hrt_rays* rays, const float* grad_x, const float* grad_y,
                                const hrt_ray_geom* geom, double chi_from, double chi_to, double a_ref,
                                double omega_m, float* maps, void* stream) {
  return step_call(rm, rays, grad_x, grad_y, nullptr, geom, chi_from, chi_to, a_ref, omega_m, maps, stream);
}

hrt_status hrt_raymesh_ray_step_tiled(hrt_raymesh* rm, const hrt_rays* rays, const float* grad_x, const float* grad_y,
                                      const float* grad_z, const hrt_ray_geom* geom, double chi_from, double chi_to,
                                      double a_ref, double omega_m, float* maps, void* stream) {
  if (!grad_z) return fail(HRT_ERR_INVALID_ARG, "grad_z is NULL");
  return step_call(rm, rays, grad_x, grad_y, grad_z, geom, chi_from, chi_to, a_ref, omega_m, maps, stream);
}

hrt_status hrt_raymesh_kick_adjoint(hrt_raymesh* rm, const float* grad_x, const float* grad_y, const float* mesh_bar,
                                    const hrt_ray_geom* geom, double chi_a, double chi_b, double a_ref, double omega_m,
                                    float* gx_bar, float* gy_bar, double* plane_bar_host, void* stream) {
  return kick_adjoint_call(rm, grad_x, grad_y, nullptr, mesh_bar, geom, chi_a, chi_b, a_ref, omega_m, gx_bar, gy_bar,
                           nullptr, plane_bar_host, stream);
}

hrt_status hrt_raymesh_kick_tiled_adjoint(hrt_raymesh* rm, const float* grad_x, const float* grad_y,
                                          const float* grad_z, const float* mesh_bar, const hrt_ray_geom* geom,
                                          double chi_a, double chi_b, double a_ref, double omega_m, float* gx_bar,
                                          float* gy_bar, float* gz_bar, double* plane_bar_host, void* stream) {
  if (!grad_z || !gz_bar) return fail(HRT_ERR_INVALID_ARG, "the tiled adjoint needs grad_z and gz_bar");
  return kick_adjoint_call(rm, grad_x, grad_y, grad_z, mesh_bar, geom, chi_a, chi_b, a_ref, omega_m, gx_bar, gy_bar,
                           gz_bar, plane_bar_host, stream);
}

hrt_status hrt_raymesh_ray_step_adjoint(hrt_raymesh* rm, const hrt_rays* rays, const float* grad_x, const float* grad_y,
                                        const hrt_ray_geom* geom, double chi_from, double chi_to, double a_ref,
                                        double omega_m, const hrt_rays* bar, float* gx_bar, float* gy_bar,
                                        double* plane_bar_host, double* drift_bar_host, void* stream) {
  return step_adjoint_call(rm, rays, grad_x, grad_y, nullptr, geom, chi_from, chi_to, a_ref, omega_m, bar, gx_bar,
                           gy_bar, nullptr, plane_bar_host, drift_bar_host, stream);
}

hrt_status hrt_raymesh_ray_step_tiled_adjoint(hrt_raymesh* rm, const hrt_rays* rays, const float* grad_x,
                                              const float* grad_y, const float* grad_z, const hrt_ray_geom* geom,
                                              double chi_from, double chi_to, double a_ref, double omega_m,
                                              const hrt_rays* bar, float* gx_bar, float* gy_bar, float* gz_bar,
                                              double* plane_bar_host, double* drift_bar_host, void* stream) {
  if (!grad_z || !gz_bar) return fail(HRT_ERR_INVALID_ARG, "the tiled adjoint needs grad_z and gz_bar");
  return step_adjoint_call(rm, rays, grad_x, grad_y, grad_z, geom, chi_from, chi_to, a_ref, omega_m, bar, gx_bar,
                           gy_bar, gz_bar, plane_bar_host, drift_bar_host, stream);
}

hrt_status hrt_raymesh_step_planes(const hrt_raymesh_config* cfg, const hrt_ray_geom* geom, double chi_from,
                                   double chi_to, double a_ref, double omega_m, int32_t* n1_host, int32_t* n2_host,
                                   double* chi_host, double* w_host, double* drift_host) {
  if (!cfg || !n1_host || !n2_host || !chi_host || !w_host || !drift_host) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  HRT_TRY(check_geom(geom, false));
  if (!(omega_m > 0.0 && omega_m <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "omega_m must be in (0, 1]");
  const double chi_mid = 0.5 * (chi_from + chi_to);
  if (!(chi_mid > 0.0)) return fail(HRT_ERR_INVALID_ARG, "shell midpoint must be at chi > 0");
  static thread_local ProjectParams p;
  const double lo[2] = {chi_from, chi_mid}, hi[2] = {chi_mid, chi_to};
  int32_t* counts[2] = {n1_host, n2_host};
  const double cell = geom->box / geom->n;
  for (int h = 0; h < 2; ++h) {
    double lam, x2d;
    int64_t n2d;
    HRT_TRY(geometry(*cfg, lo[h], hi[h], cell, lam, x2d, n2d));
    HRT_TRY(plane_table(*geom, lo[h], hi[h], a_ref, omega_m, x2d, n2d, p, w_host + h * kMaxMeshPlanes,
                        chi_host + h * kMaxMeshPlanes));
    *counts[h] = p.n_planes;
  }
  drift_host[0] = (chi_to - chi_from) / (kCLight * chi_mid * chi_mid);
  return HRT_OK;
}

}  // extern "C"
