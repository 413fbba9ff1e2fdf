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
__global__ void __launch_bounds__(kTileX * kTileY) raymesh_project_kernel(const float* __restrict__ gx,
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

__global__ void __launch_bounds__(256) raymesh_ray_kernel(double2* __restrict__ theta, float2* __restrict__ eta,
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
                              double x2d, int64_t n2d, ProjectParams& p) {
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
    p.w[q] = static_cast<float>(-(2.0 / kCLight) * r * gw * sgn * cell * cell * cell / (r * r * x2d * x2d));
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
  HRT_TRY(cufft_check(cufftExecC2C(plan, c, c, CUFFT_INVERSE), "inverse"));
  view.k = mesh;
  return HRT_OK;
}

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

}  // extern "C"
