// Mesh kernels of the HRT hot path on sm_103a: CIC mass assignment, the fused k-space Poisson/gradient/
// deconvolution kernel (3D path), the fused particle gather + kick + drift + deposit, its shared-memory-tile
// variant on brick-sorted particles, and the Zel'dovich and 2LPT IC helpers.
//
// The mesh passes are bound by HBM bandwidth or by the latency of their gathers; the kernels are written for
// coalesced accesses with neighbouring threads on neighbouring cells, so that the gathers and the deposit's
// 16-byte vector reductions hit lines already resident in the 129 MB L2.  Particles come in one of two storage
// orders: fresh particles in Lagrangian-lattice order, walked in Morton-ordered bricks of lattice sites, and the
// context's particles in cell order (re-sorted by mesh cell every few steps, sort_kernels.cu), where a
// slot -> lattice-site map gives each thread its site.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"
#include "kspace_callback.h"
#include "mesh_kernels.h"
#include "tma.h"

namespace hrt {

// Lower node (wrapped into [0, n)) and fraction of a coordinate given as lattice node + displacement in cells.
__device__ __forceinline__ void cic_axis(int q_node, float d_cells, int n, int& i0, float& f) {
  float fl = floorf(d_cells);
  f = d_cells - fl;
  int i = q_node + static_cast<int>(fl);
  if (static_cast<unsigned>(i) >= static_cast<unsigned>(n)) {  // rare: more than one box away or negative
    i %= n;
    if (i < 0) i += n;
  }
  i0 = i;
}

__device__ __forceinline__ int wrap_next(int i, int n) { return i + 1 == n ? 0 : i + 1; }

// Particle launch geometry.  Storage stays in row-major lattice order; only the thread -> particle map changes.
// Brick mode (n_side a power of two >= 32): each block of 256 threads takes a brick of 2 x 4 x 32 lattice sites
// (one warp = 32 consecutive sites along z = 128 contiguous bytes per array), and consecutive blocks walk the
// bricks in Z (Morton) order, so the blocks resident at one time cover a compact region of the mesh whose fields
// and density lines stay in L2 despite the particles' displacements.  Otherwise blockIdx.x enumerates lattice
// rows (qi, qj) and blockIdx.y * blockDim.x + threadIdx.x the site along the row.
struct Lattice {
  int n_side, ratio, n;
  float inv_cell;
  int brick_mode;
  int lbx, lby, lbz;  // log2 of the brick counts per axis (brick mode)
  // particles stored in cell order: slot i holds lattice particle order[i] (nullptr: lattice order)
  const int32_t* order;
  int64_t n_particles;
  int lns;  // log2(n_side) when n_side is a power of two (lattice index by shifts), else -1
};

// Lattice site (qi, qj, qk) of lattice particle index lag (row-major, qk fastest).
__device__ __forceinline__ void lattice_site(const Lattice& L, unsigned lag, int& qi, int& qj, int& qk) {
  if (L.lns >= 0) {
    const unsigned mask = (1u << L.lns) - 1u;
    qk = static_cast<int>(lag & mask);
    qj = static_cast<int>((lag >> L.lns) & mask);
    qi = static_cast<int>(lag >> (2 * L.lns));
    return;
  }
  const unsigned ns = static_cast<unsigned>(L.n_side);
  qk = static_cast<int>(lag % ns);
  const unsigned row = lag / ns;
  qj = static_cast<int>(row % ns);
  qi = static_cast<int>(row / ns);
}

__device__ __forceinline__ void morton_decode(unsigned code, int lbx, int lby, int lbz, int& bx, int& by, int& bz) {
  bx = by = bz = 0;
  int sx = 0, sy = 0, sz = 0;
  // bits are dealt round-robin z, y, x to the axes that still have bits left
  while (sx < lbx || sy < lby || sz < lbz) {
    if (sz < lbz) { bz |= static_cast<int>(code & 1u) << sz; ++sz; code >>= 1; }
    if (sy < lby) { by |= static_cast<int>(code & 1u) << sy; ++sy; code >>= 1; }
    if (sx < lbx) { bx |= static_cast<int>(code & 1u) << sx; ++sx; code >>= 1; }
  }
}

__device__ __forceinline__ bool particle_of_thread(const Lattice& L, int64_t& p, int& qi, int& qj, int& qk) {
  if (L.order) {
    // one thread per storage slot; the lattice site comes from the slot's particle index
    p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (p >= L.n_particles) return false;
    lattice_site(L, static_cast<unsigned>(__ldg(L.order + p)), qi, qj, qk);
    return true;
  }
  if (L.brick_mode) {
    int bx, by, bz;
    morton_decode(blockIdx.x, L.lbx, L.lby, L.lbz, bx, by, bz);
    const int t = threadIdx.x;
    qi = bx * 2 + (t >> 7);
    qj = by * 4 + ((t >> 5) & 3);
    qk = bz * 32 + (t & 31);
  } else {
    qk = blockIdx.y * blockDim.x + threadIdx.x;
    if (qk >= L.n_side) return false;
    const unsigned row = blockIdx.x;
    qi = static_cast<int>(row / static_cast<unsigned>(L.n_side));
    qj = static_cast<int>(row - static_cast<unsigned>(qi) * L.n_side);
  }
  p = (static_cast<int64_t>(qi) * L.n_side + qj) * L.n_side + qk;
  return true;
}

static inline int ilog2_exact(int64_t v) {
  int l = 0;
  while ((int64_t{1} << l) < v) ++l;
  return (int64_t{1} << l) == v ? l : -1;
}

static inline bool brick_ok(int64_t n_side) { return n_side >= 32 && ilog2_exact(n_side) >= 0; }

static inline dim3 particle_grid(int64_t n_side, int threads, const int32_t* order = nullptr) {
  if (order) return dim3(static_cast<unsigned>((n_side * n_side * n_side + threads - 1) / threads), 1);
  if (brick_ok(n_side) && threads == 256) return dim3(static_cast<unsigned>(n_side * n_side * n_side / 256), 1);
  return dim3(static_cast<unsigned>(n_side * n_side), static_cast<unsigned>((n_side + threads - 1) / threads));
}

// Adds w0 to cell (col + iz) and w1 to cell (col + jz), jz = iz + 1 or 0 at the periodic wrap.  Mesh sides that
// are multiples of 4 (col is then a multiple of 4 as well): one 16-byte vector reduction on the aligned group of
// four cells that holds iz, carrying w1 too unless jz starts the next group (iz mod 4 = 3, the wrap included),
// which takes a second, predicated one; so a warp issues two reductions per pair of rows whatever the cells of
// its lanes, where the 8-byte and scalar forms below, taken by lanes of either parity, issue three.  Other sides:
// z-adjacent pairs starting on an even cell use one 8-byte reduction, the rest two scalar ones.
__device__ __forceinline__ void deposit_pair(float* __restrict__ rho, size_t col, int iz, int jz, float w0, float w1,
                                             int n) {
  if ((n & 3) == 0) {
    const int s = iz & 3;
    float4 v;
    v.x = s == 0 ? w0 : 0.f;
    v.y = s == 1 ? w0 : (s == 0 ? w1 : 0.f);
    v.z = s == 2 ? w0 : (s == 1 ? w1 : 0.f);
    v.w = s == 3 ? w0 : (s == 2 ? w1 : 0.f);
    atomicAdd(reinterpret_cast<float4*>(rho + col + (iz - s)), v);
    if (s == 3) atomicAdd(reinterpret_cast<float4*>(rho + col + jz), make_float4(w1, 0.f, 0.f, 0.f));
    return;
  }
  if (jz == iz + 1 && (iz & 1) == 0) {
    atomicAdd(reinterpret_cast<float2*>(rho + col + iz), make_float2(w0, w1));
  } else {
    atomicAdd(rho + col + iz, w0);
    atomicAdd(rho + col + jz, w1);
  }
}

__device__ __forceinline__ void deposit_cic(float* __restrict__ rho, int n, int ix, int iy, int iz, float fx,
                                            float fy, float fz, float mass) {
  const int jx = wrap_next(ix, n), jy = wrap_next(iy, n), jz = wrap_next(iz, n);
  const float wx0 = (1.f - fx) * mass, wx1 = fx * mass;
  const float wy0 = 1.f - fy, wy1 = fy, wz0 = 1.f - fz, wz1 = fz;
  const size_t c00 = static_cast<size_t>(static_cast<unsigned>(ix * n + iy)) * n;
  const size_t c01 = static_cast<size_t>(static_cast<unsigned>(ix * n + jy)) * n;
  const size_t c10 = static_cast<size_t>(static_cast<unsigned>(jx * n + iy)) * n;
  const size_t c11 = static_cast<size_t>(static_cast<unsigned>(jx * n + jy)) * n;
  deposit_pair(rho, c00, iz, jz, wx0 * wy0 * wz0, wx0 * wy0 * wz1, n);
  deposit_pair(rho, c01, iz, jz, wx0 * wy1 * wz0, wx0 * wy1 * wz1, n);
  deposit_pair(rho, c10, iz, jz, wx1 * wy0 * wz0, wx1 * wy0 * wz1, n);
  deposit_pair(rho, c11, iz, jz, wx1 * wy1 * wz0, wx1 * wy1 * wz1, n);
}

// ---------------------------------------------------------------------------------------------------------
// CIC mass assignment: one thread per particle, four pairs of float32 reductions into the mesh.
// ---------------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) cic_scatter_kernel(const float* __restrict__ disp, int64_t np, Lattice L,
                                                          float mass, float* __restrict__ rho) {
  int64_t p;
  int qi, qj, qk;
  if (!particle_of_thread(L, p, qi, qj, qk)) return;
  int ix, iy, iz;
  float fx, fy, fz;
  cic_axis(qi * L.ratio, __ldg(disp + p) * L.inv_cell, L.n, ix, fx);
  cic_axis(qj * L.ratio, __ldg(disp + np + p) * L.inv_cell, L.n, iy, fy);
  cic_axis(qk * L.ratio, __ldg(disp + 2 * np + p) * L.inv_cell, L.n, iz, fz);
  deposit_cic(rho, L.n, ix, iy, iz, fx, fy, fz, mass);
}

// The same deposit with warp-aggregated atomics, the form that pays off when many particles of a warp share a
// target: lanes whose pair (or first cell) coincides find each other with __match_any_sync, the lowest lane
// of each group adds the group's sum.  Kept as the measured alternative to plain reductions: in lattice (brick)
// order few lanes of a warp share a target at 2 mesh cells per particle spacing, so the matching and the shuffles
// cost more than the atomics they save.
__device__ __forceinline__ void deposit_pair_warp(float* __restrict__ rho, size_t col, int iz, int jz, float w0,
                                                  float w1) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool vec = (jz == iz + 1 && (iz & 1) == 0);
  const unsigned long long addr = reinterpret_cast<unsigned long long>(rho + col + iz);
  const unsigned grp = __match_any_sync(full, vec ? addr : (addr | (1ull << 63)));
  float s0 = w0, s1 = w1;
  if (__any_sync(full, __popc(grp) > 1)) {
    for (int l = 0; l < 32; ++l) {
      const float v0 = __shfl_sync(full, w0, l), v1 = __shfl_sync(full, w1, l);
      if (l != lane && ((grp >> l) & 1u)) {
        s0 += v0;
        s1 += v1;
      }
    }
  }
  if (lane != __ffs(grp) - 1) return;
  if (vec) {
    atomicAdd(reinterpret_cast<float2*>(rho + col + iz), make_float2(s0, s1));
  } else {
    atomicAdd(rho + col + iz, s0);
    atomicAdd(rho + col + jz, s1);
  }
}

// Brick mode only (every warp full, as the warp intrinsics above need).
__global__ void __launch_bounds__(256) cic_scatter_warp_kernel(const float* __restrict__ disp, int64_t np, Lattice L,
                                                               float mass, float* __restrict__ rho) {
  int64_t p;
  int qi, qj, qk;
  particle_of_thread(L, p, qi, qj, qk);
  int ix, iy, iz;
  float fx, fy, fz;
  cic_axis(qi * L.ratio, __ldg(disp + p) * L.inv_cell, L.n, ix, fx);
  cic_axis(qj * L.ratio, __ldg(disp + np + p) * L.inv_cell, L.n, iy, fy);
  cic_axis(qk * L.ratio, __ldg(disp + 2 * np + p) * L.inv_cell, L.n, iz, fz);
  const int n = L.n;
  const int jx = wrap_next(ix, n), jy = wrap_next(iy, n), jz = wrap_next(iz, n);
  const float wx0 = (1.f - fx) * mass, wx1 = fx * mass;
  const float wy0 = 1.f - fy, wy1 = fy, wz0 = 1.f - fz, wz1 = fz;
  const size_t c00 = static_cast<size_t>(static_cast<unsigned>(ix * n + iy)) * n;
  const size_t c01 = static_cast<size_t>(static_cast<unsigned>(ix * n + jy)) * n;
  const size_t c10 = static_cast<size_t>(static_cast<unsigned>(jx * n + iy)) * n;
  const size_t c11 = static_cast<size_t>(static_cast<unsigned>(jx * n + jy)) * n;
  deposit_pair_warp(rho, c00, iz, jz, wx0 * wy0 * wz0, wx0 * wy0 * wz1);
  deposit_pair_warp(rho, c01, iz, jz, wx0 * wy1 * wz0, wx0 * wy1 * wz1);
  deposit_pair_warp(rho, c10, iz, jz, wx1 * wy0 * wz0, wx1 * wy0 * wz1);
  deposit_pair_warp(rho, c11, iz, jz, wx1 * wy1 * wz0, wx1 * wy1 * wz1);
}

static Lattice make_lattice(int64_t n_side, int64_t n, double box, const int32_t* order = nullptr) {
  Lattice L{static_cast<int>(n_side), static_cast<int>(n / n_side), static_cast<int>(n), static_cast<float>(n / box),
            0, 0, 0, 0, order, n_side * n_side * n_side, ilog2_exact(n_side)};
  if (brick_ok(n_side)) {
    const int l = ilog2_exact(n_side);
    L.brick_mode = 1;
    L.lbx = l - 1;  // bricks of 2 sites along x
    L.lby = l - 2;  // 4 along y
    L.lbz = l - 5;  // 32 along z
  }
  return L;
}

static float particle_mass(int64_t n_side, int64_t n) {
  return static_cast<float>(static_cast<double>(n) * n * n / (static_cast<double>(n_side) * n_side * n_side));
}

hrt_status launch_cic_scatter_warp(const float* disp, int64_t n_side, int64_t n, double box, float* rho,
                                   cudaStream_t s) {
  if (!brick_ok(n_side)) return fail(HRT_ERR_INVALID_ARG, "the warp-aggregated deposit needs n_side a power of two >= 32");
  const int64_t np = n_side * n_side * n_side;
  HRT_CUDA(cudaMemsetAsync(rho, 0, static_cast<size_t>(n) * n * n * sizeof(float), s));
  cic_scatter_warp_kernel<<<particle_grid(n_side, 256), 256, 0, s>>>(disp, np, make_lattice(n_side, n, box),
                                                                     particle_mass(n_side, n), rho);
  HRT_LAUNCHED("cic_scatter_warp_kernel");
  return HRT_OK;
}

hrt_status launch_cic_scatter(const float* disp, int64_t n_side, int64_t n, double box, float* rho,
                              cudaStream_t s, const int32_t* order, bool rho_zeroed) {
  int64_t np = n_side * n_side * n_side;
  size_t mesh_bytes = static_cast<size_t>(n) * n * n * sizeof(float);
  if (!rho_zeroed) HRT_CUDA(cudaMemsetAsync(rho, 0, mesh_bytes, s));
  if (np == 0) return HRT_OK;
  cic_scatter_kernel<<<particle_grid(n_side, 256, order), 256, 0, s>>>(disp, np, make_lattice(n_side, n, box, order),
                                                                       particle_mass(n_side, n), rho);
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

// One half-spectrum element: v = rho_hat[e] at integer frequency (ix, iy, iz) -> the gradient spectra of both sets.
__device__ __forceinline__ void kspace_element(float2 v, int n, float kf, float scale, int64_t elems,
                                               const KspaceSet& a, const KspaceSet& b, int ix, int iy, int iz,
                                               int64_t e) {
  const int half = n >> 1;
  const int nx = ix < half ? ix : ix - n;
  const int ny = iy < half ? iy : iy - n;
  const int nz = iz;
  const float kx = kf * nx, ky = kf * ny, kz = kf * nz;
  const float k2 = kx * kx + ky * ky + kz * kz;
  const float dx = (nx == -half) ? 0.f : kx;
  const float dy = (ny == -half) ? 0.f : ky;
  const float dz = (nz == half) ? 0.f : kz;
  const float green = k2 > 0.f ? scale / k2 : 0.f;
  const float kmag = sqrtf(k2);
  {
    const float c = green * __ldg(a.wx + ix) * __ldg(a.wy + iy) * __ldg(a.wz + iz) * learned_g(a, kmag);
    const float2 base = make_float2(-c * v.y, c * v.x);  // i * c * v
    a.out[e] = make_float2(dx * base.x, dx * base.y);
    if (a.n_out > 1) a.out[e + elems] = make_float2(dy * base.x, dy * base.y);
    if (a.n_out > 2) a.out[e + 2 * elems] = make_float2(dz * base.x, dz * base.y);
  }
  if (b.n_out > 0) {
    const float c = green * __ldg(b.wx + ix) * __ldg(b.wy + iy) * __ldg(b.wz + iz) * learned_g(b, kmag);
    const float2 base = make_float2(-c * v.y, c * v.x);
    b.out[e] = make_float2(dx * base.x, dx * base.y);
    if (b.n_out > 1) b.out[e + elems] = make_float2(dy * base.x, dy * base.y);
    if (b.n_out > 2) b.out[e + 2 * elems] = make_float2(dz * base.x, dz * base.y);
  }
}

// Grid: x over rows (ix, iy) in groups of blockDim.y; y over chunks of kKspacePer * blockDim.x along kz in
// [0, n/2).  Each thread loads its kKspacePer elements (strided by blockDim.x, so every load is coalesced)
// before computing, to keep several loads in flight; the Nyquist column kz = n/2 is done by the thread that
// holds kz = 0.
constexpr int kKspacePer = 4;

__global__ void __launch_bounds__(256) kspace_kernel(const float2* __restrict__ rho_hat, int n, int nzc, float kf,
                                                     float scale, int64_t elems, KspaceSet a, KspaceSet b) {
  const unsigned row = blockIdx.x * blockDim.y + threadIdx.y;
  if (row >= static_cast<unsigned>(n) * static_cast<unsigned>(n)) return;
  const int ix = static_cast<int>(row / static_cast<unsigned>(n));
  const int iy = static_cast<int>(row - static_cast<unsigned>(ix) * n);
  const int64_t e0 = static_cast<int64_t>(row) * nzc;
  const int z0 = blockIdx.y * (blockDim.x * kKspacePer) + threadIdx.x;
  float2 v[kKspacePer];
#pragma unroll
  for (int j = 0; j < kKspacePer; ++j) {
    const int iz = z0 + j * blockDim.x;
    v[j] = iz < nzc - 1 ? __ldg(rho_hat + e0 + iz) : make_float2(0.f, 0.f);
  }
  const bool nyquist = z0 == 0;
  const float2 vn = nyquist ? __ldg(rho_hat + e0 + nzc - 1) : make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < kKspacePer; ++j) {
    const int iz = z0 + j * blockDim.x;
    if (iz < nzc - 1) kspace_element(v[j], n, kf, scale, elems, a, b, ix, iy, iz, e0 + iz);
  }
  if (nyquist) kspace_element(vn, n, kf, scale, elems, a, b, ix, iy, nzc - 1, e0 + nzc - 1);
}

__global__ void set_callback_info_kernel(KspaceCallbackInfo* dst, KspaceCallbackInfo v) { *dst = v; }

hrt_status launch_set_callback_info(KspaceCallbackInfo* dst, const KspaceCallbackInfo& v, cudaStream_t s) {
  set_callback_info_kernel<<<1, 1, 0, s>>>(dst, v);
  HRT_LAUNCHED("set_callback_info_kernel");
  return HRT_OK;
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
            static_cast<unsigned>((nzc - 1 + block.x * kKspacePer - 1) / (block.x * kKspacePer)));
  kspace_kernel<<<grid, block, 0, s>>>(static_cast<const float2*>(rho_hat), static_cast<int>(n),
                                       static_cast<int>(nzc), static_cast<float>(2.0 * M_PI / box),
                                       static_cast<float>(scale), elems, a, b);
  HRT_LAUNCHED("kspace_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// Particle gather + kick + drift: one thread per particle.
// ---------------------------------------------------------------------------------------------------------
// Trilinear interpolation of the eight corner values (cYX: lower/upper node along y then x; the z suffix marks
// the upper node along z).
__device__ __forceinline__ float trilerp(float c00, float c00z, float c01, float c01z, float c10, float c10z,
                                         float c11, float c11z, float fx, float fy, float fz) {
  float a00 = c00 + fz * (c00z - c00), a01 = c01 + fz * (c01z - c01);
  float a10 = c10 + fz * (c10z - c10), a11 = c11 + fz * (c11z - c11);
  float b0 = a00 + fy * (a01 - a00), b1 = a10 + fy * (a11 - a10);
  return b0 + fx * (b1 - b0);
}

__device__ __forceinline__ float trilinear(const float* __restrict__ f, int64_t r00, int64_t r01, int64_t r10,
                                           int64_t r11, int iz, int jz, float fx, float fy, float fz) {
  return trilerp(__ldg(f + r00 + iz), __ldg(f + r00 + jz), __ldg(f + r01 + iz), __ldg(f + r01 + jz),
                 __ldg(f + r10 + iz), __ldg(f + r10 + jz), __ldg(f + r11 + iz), __ldg(f + r11 + jz), fx, fy, fz);
}

// The update of one particle (slot p, lattice site q, displacement d and momentum m as loaded): gather, kick,
// drift, stores, and with DEPOSIT the CIC deposit of the drifted particle into rho.
template <bool DEPOSIT>
__device__ __forceinline__ void update_particle(const float* __restrict__ gx, const float* __restrict__ gy,
                                                const float* __restrict__ gz, const Lattice& L, int64_t np, int64_t p,
                                                int qi, int qj, int qk, float d0, float d1, float d2, float m0,
                                                float m1, float m2, float* __restrict__ disp, float* __restrict__ mom,
                                                float kick, float drift, float mass, float* __restrict__ rho) {
  const int n = L.n;
  int ix, iy, iz;
  float fx, fy, fz;
  const int bx = qi * L.ratio, by = qj * L.ratio, bz = qk * L.ratio;
  cic_axis(bx, d0 * L.inv_cell, n, ix, fx);
  cic_axis(by, d1 * L.inv_cell, n, iy, fy);
  cic_axis(bz, d2 * L.inv_cell, n, iz, fz);
  const int jx = wrap_next(ix, n), jy = wrap_next(iy, n), jz = wrap_next(iz, n);
  const int64_t r00 = static_cast<int64_t>(static_cast<unsigned>(ix * n + iy)) * n;
  const int64_t r01 = static_cast<int64_t>(static_cast<unsigned>(ix * n + jy)) * n;
  const int64_t r10 = static_cast<int64_t>(static_cast<unsigned>(jx * n + iy)) * n;
  const int64_t r11 = static_cast<int64_t>(static_cast<unsigned>(jx * n + jy)) * n;
  const float a0 = trilinear(gx, r00, r01, r10, r11, iz, jz, fx, fy, fz);
  const float a1 = trilinear(gy, r00, r01, r10, r11, iz, jz, fx, fy, fz);
  const float a2 = trilinear(gz, r00, r01, r10, r11, iz, jz, fx, fy, fz);
  m0 -= a0 * kick;
  m1 -= a1 * kick;
  m2 -= a2 * kick;
  mom[p] = m0;
  mom[p + np] = m1;
  mom[p + 2 * np] = m2;
  if (drift != 0.f) {
    d0 += m0 * drift;
    d1 += m1 * drift;
    d2 += m2 * drift;
    disp[p] = d0;
    disp[p + np] = d1;
    disp[p + 2 * np] = d2;
  }
  if (DEPOSIT) {
    cic_axis(bx, d0 * L.inv_cell, n, ix, fx);
    cic_axis(by, d1 * L.inv_cell, n, iy, fy);
    cic_axis(bz, d2 * L.inv_cell, n, iz, fz);
    deposit_cic(rho, n, ix, iy, iz, fx, fy, fz, mass);
  }
}

// One thread per particle.  With DEPOSIT the drifted particle is deposited at once into rho (zeroed before
// the launch), which fuses the CIC mass assignment of the next force into the update and saves re-reading the
// positions.  Four blocks per SM with up to 64 registers each: measured at 1024^3, 5.88 ms against 6.02 ms with
// the compiler's own choice (56 registers), 6.04 / 6.09 ms at five / six blocks (48 / 40 registers) and 6.36 ms
// at three; the kernel waits on the latency of its loads, so registers for loads in flight beat more warps.
template <bool DEPOSIT>
__global__ void __launch_bounds__(256, 4) kick_drift_kernel(const float* __restrict__ gx, const float* __restrict__ gy,
                                                         const float* __restrict__ gz, Lattice L, int64_t np,
                                                         float* __restrict__ disp, float* __restrict__ mom,
                                                         float kick, float drift, float mass, float* __restrict__ rho) {
  int64_t p;
  int qi, qj, qk;
  if (!particle_of_thread(L, p, qi, qj, qk)) return;
  update_particle<DEPOSIT>(gx, gy, gz, L, np, p, qi, qj, qk, disp[p], disp[p + np], disp[p + 2 * np], mom[p],
                           mom[p + np], mom[p + 2 * np], disp, mom, kick, drift, mass, rho);
}

// ---------------------------------------------------------------------------------------------------------
// The kick-drift-deposit on brick-sorted particles: one block per 8 x 8 x 32-cell brick of the sort.  The block
// copies the fields of its tile (the brick plus one cell of drift and one of stencil on the upper side of each
// axis, z rounded to 16 bytes: 10 x 10 x 36 cells) into shared memory, gathers from there, and deposits the
// drifted particles into a density tile of the same box with shared-memory atomics, which it then adds to the
// mesh with 16-byte vector reductions (all-zero groups skipped).  Tiles inside the mesh arrive by TMA (one 3D
// box per field, completing on an mbarrier with a bounded wait); tiles that wrap around the periodic boundary,
// about 5 % of the bricks at 1024^3, by 16-byte cp.async copies of their rows.  A particle whose gather or deposit
// stencil leaves the tile (it moved below its brick since the sort, or more than a cell above) takes the global
// path for that part; bricks with fewer than kTileMinParticles particles take the global path entirely.  Every
// particle's arithmetic is that of kick_drift_kernel, so momenta and displacements are the same bit for bit;
// the density differs only in the order of its float additions.
// ---------------------------------------------------------------------------------------------------------
constexpr int kTileX = kBrickXY + 2, kTileY = kBrickXY + 2, kTileZ = kBrickZ + 4;
constexpr int kTileCells = kTileX * kTileY * kTileZ;
constexpr int kFieldStride = (kTileCells + 31) / 32 * 32;  // floats per field tile: 128-byte aligned TMA boxes
constexpr int kTileQuads = kTileZ / 4;                      // 16-byte groups per tile row
constexpr int kTileMinParticles = 32;
constexpr int kTileThreads = 256;
// three field tiles, the density tile, the mbarrier, and slack for aligning the base to 128 bytes
constexpr size_t kTileSmem = sizeof(float) * (3 * kFieldStride + kTileCells) + 16 + 128;

// Tensor maps of the three gradient fields (3D, z innermost, boxes of one tile).
struct FieldMaps {
  CUtensorMap m[3];
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(gmem) : "memory");
}

// Offset of tile position (dx, dy, dz) in [0, tile) from tile origin (x0, y0, z0): cells wrap periodically.
__device__ __forceinline__ int tile_wrap(int v, int n) { return v >= n ? v - n : v; }

__global__ void __launch_bounds__(kTileThreads, 3)
    kick_drift_tiled_kernel(const __grid_constant__ FieldMaps maps, int use_tma, const float* __restrict__ gx,
                            const float* __restrict__ gy, const float* __restrict__ gz, Lattice L, int64_t np,
                            const int32_t* __restrict__ key_start, float* __restrict__ disp, float* __restrict__ mom,
                            float kick, float drift, float mass, float* __restrict__ rho, int* __restrict__ err) {
  extern __shared__ unsigned char tile_raw[];
  float* ft = reinterpret_cast<float*>(tile_raw + ((128 - (tma::smem_u32(tile_raw) & 127)) & 127));
  // ft: [3][kFieldStride] with [kTileX][kTileY][kTileZ] in each; rt: [kTileX][kTileY][kTileZ]
  float* rt = ft + 3 * kFieldStride;
  const uint32_t bar = tma::smem_u32(rt + kTileCells);
  const int n = L.n, tid = threadIdx.x;
  const int nb = n / kBrickXY;
  const unsigned b = blockIdx.x;
  const int by = static_cast<int>(b % nb), bx = static_cast<int>((b / nb) % nb), bz = static_cast<int>(b / nb / nb);
  const int x0 = bx * kBrickXY, y0 = by * kBrickXY, z0 = bz * kBrickZ;
  // the slot range, clamped into [0, np] so that any offsets stay in bounds
  const int64_t s = min(max(int64_t{__ldg(key_start + static_cast<int64_t>(b) * kBrickKeys)}, int64_t{0}), np);
  const int64_t e = b + 1 < gridDim.x
                        ? min(max(int64_t{__ldg(key_start + static_cast<int64_t>(b + 1) * kBrickKeys)}, s), np)
                        : np;
  const bool tiled = e - s >= kTileMinParticles;
  // TMA boxes for tiles inside the mesh, row copies for tiles that wrap
  const bool by_tma = tiled && use_tma && x0 + kTileX <= n && y0 + kTileY <= n && z0 + kTileZ <= n;
  if (by_tma) {
    if (tid == 0) {
      tma::mbar_init(bar, 1);
      tma::fence_mbar_init();
      tma::mbar_expect_tx(bar, 3 * kTileCells * sizeof(float));
      for (int c = 0; c < 3; ++c) tma::load_3d(tma::smem_u32(ft + c * kFieldStride), &maps.m[c], z0, y0, x0, bar);
    }
  }
  if (tiled) {
    float4* rt4 = reinterpret_cast<float4*>(rt);
    for (int i = tid; i < kTileCells / 4; i += kTileThreads) rt4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (tiled && !by_tma) {
    for (int i = tid; i < 3 * kTileX * kTileY * kTileQuads; i += kTileThreads) {
      const int r = i / kTileQuads, q = i - r * kTileQuads;
      const int f = r / (kTileX * kTileY), rem = r - f * (kTileX * kTileY);
      const int dx = rem / kTileY, dy = rem - dx * kTileY;
      const float* src = f == 0 ? gx : (f == 1 ? gy : gz);
      const size_t off = static_cast<size_t>(static_cast<unsigned>(tile_wrap(x0 + dx, n) * n + tile_wrap(y0 + dy, n))) * n +
                         tile_wrap(z0 + 4 * q, n);
      cp_async16(ft + f * kFieldStride + rem * kTileZ + 4 * q, src + off);
    }
  }
  // a field tile this thread may read (false after a timed-out wait: the thread takes the global path)
  bool fields_ok = tiled;
  const float* gf[3] = {gx, gy, gz};
  for (int64_t base = s; base < e; base += kTileThreads) {
    const int64_t p = base + tid;
    const bool act = p < e;
    float d0 = 0.f, d1 = 0.f, d2 = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f;
    int qi = 0, qj = 0, qk = 0;
    if (act) {
      d0 = disp[p];
      d1 = disp[p + np];
      d2 = disp[p + 2 * np];
      m0 = mom[p];
      m1 = mom[p + np];
      m2 = mom[p + 2 * np];
      lattice_site(L, static_cast<unsigned>(__ldg(L.order + p)), qi, qj, qk);
    }
    if (tiled && base == s) {
      if (by_tma) {
        // the mbarrier was initialised by thread 0 before its loads; the barrier below orders every other
        // thread's first probe after that
        __syncthreads();
        if (!tma::mbar_wait(bar, 0)) {
          fields_ok = false;
          atomicOr(err, kTileTimeout);
        }
      } else {
        asm volatile("cp.async.wait_all;" ::: "memory");
      }
      __syncthreads();
    }
    if (act) {
      int ix, iy, iz;
      float fx, fy, fz;
      const int bxl = qi * L.ratio, byl = qj * L.ratio, bzl = qk * L.ratio;
      cic_axis(bxl, d0 * L.inv_cell, n, ix, fx);
      cic_axis(byl, d1 * L.inv_cell, n, iy, fy);
      cic_axis(bzl, d2 * L.inv_cell, n, iz, fz);
      int ox = ix - x0, oy = iy - y0, oz = iz - z0;
      ox += ox < 0 ? n : 0;
      oy += oy < 0 ? n : 0;
      oz += oz < 0 ? n : 0;
      float a[3];
      if (fields_ok && ox < kTileX - 1 && oy < kTileY - 1 && oz < kTileZ - 1) {
        const float* t = ft + (ox * kTileY + oy) * kTileZ + oz;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float* u = t + c * kFieldStride;
          a[c] = trilerp(u[0], u[1], u[kTileZ], u[kTileZ + 1], u[kTileY * kTileZ], u[kTileY * kTileZ + 1],
                         u[kTileY * kTileZ + kTileZ], u[kTileY * kTileZ + kTileZ + 1], fx, fy, fz);
        }
      } else {
        const int jx = wrap_next(ix, n), jy = wrap_next(iy, n), jz = wrap_next(iz, n);
        const int64_t r00 = static_cast<int64_t>(static_cast<unsigned>(ix * n + iy)) * n;
        const int64_t r01 = static_cast<int64_t>(static_cast<unsigned>(ix * n + jy)) * n;
        const int64_t r10 = static_cast<int64_t>(static_cast<unsigned>(jx * n + iy)) * n;
        const int64_t r11 = static_cast<int64_t>(static_cast<unsigned>(jx * n + jy)) * n;
#pragma unroll
        for (int c = 0; c < 3; ++c) a[c] = trilinear(gf[c], r00, r01, r10, r11, iz, jz, fx, fy, fz);
      }
      m0 -= a[0] * kick;
      m1 -= a[1] * kick;
      m2 -= a[2] * kick;
      mom[p] = m0;
      mom[p + np] = m1;
      mom[p + 2 * np] = m2;
      if (drift != 0.f) {
        d0 += m0 * drift;
        d1 += m1 * drift;
        d2 += m2 * drift;
        disp[p] = d0;
        disp[p + np] = d1;
        disp[p + 2 * np] = d2;
      }
      cic_axis(bxl, d0 * L.inv_cell, n, ix, fx);
      cic_axis(byl, d1 * L.inv_cell, n, iy, fy);
      cic_axis(bzl, d2 * L.inv_cell, n, iz, fz);
      ox = ix - x0;
      oy = iy - y0;
      oz = iz - z0;
      ox += ox < 0 ? n : 0;
      oy += oy < 0 ? n : 0;
      oz += oz < 0 ? n : 0;
      if (tiled && ox < kTileX - 1 && oy < kTileY - 1 && oz < kTileZ - 1) {
        const float wx0 = (1.f - fx) * mass, wx1 = fx * mass;
        const float wy0 = 1.f - fy, wy1 = fy, wz0 = 1.f - fz, wz1 = fz;
        float* t = rt + (ox * kTileY + oy) * kTileZ + oz;
        atomicAdd(t, wx0 * wy0 * wz0);
        atomicAdd(t + 1, wx0 * wy0 * wz1);
        atomicAdd(t + kTileZ, wx0 * wy1 * wz0);
        atomicAdd(t + kTileZ + 1, wx0 * wy1 * wz1);
        atomicAdd(t + kTileY * kTileZ, wx1 * wy0 * wz0);
        atomicAdd(t + kTileY * kTileZ + 1, wx1 * wy0 * wz1);
        atomicAdd(t + kTileY * kTileZ + kTileZ, wx1 * wy1 * wz0);
        atomicAdd(t + kTileY * kTileZ + kTileZ + 1, wx1 * wy1 * wz1);
      } else {
        deposit_cic(rho, n, ix, iy, iz, fx, fy, fz, mass);
      }
    }
  }
  if (!tiled) return;
  // a thread whose wait timed out lets the copies land before the block's shared memory goes away (again a
  // bounded wait)
  if (by_tma && !fields_ok) tma::mbar_wait(bar, 0);
  __syncthreads();
  const float4* rt4 = reinterpret_cast<const float4*>(rt);
  for (int i = tid; i < kTileCells / 4; i += kTileThreads) {
    const float4 v = rt4[i];
    if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) continue;
    const int r = i / kTileQuads, q = i - r * kTileQuads;
    const int dx = r / kTileY, dy = r - dx * kTileY;
    const size_t off = static_cast<size_t>(static_cast<unsigned>(tile_wrap(x0 + dx, n) * n + tile_wrap(y0 + dy, n))) * n +
                       tile_wrap(z0 + 4 * q, n);
    atomicAdd(reinterpret_cast<float4*>(rho + off), v);
  }
}

// Error word of the stateless calls (a timed-out tile wait changes no result: the block takes the global path).
__device__ int g_tile_err;

hrt_status launch_kick_drift_tiled(const float* grad, int64_t n, double box, int64_t n_side, float* disp, float* mom,
                                   double kick, double drift, float* rho_out, const int32_t* order,
                                   const int32_t* key_start, cudaStream_t s, int mode, int* err, bool rho_zeroed) {
  if (!particle_bricks_ok(n) || !order || !key_start || !rho_out)
    return fail(HRT_ERR_INVALID_ARG, "the tiled kick-drift-deposit needs brick-sorted particles and a density");
  const int64_t np = n_side * n_side * n_side;
  const int64_t m = n * n * n;
  if (!rho_zeroed) HRT_CUDA(cudaMemsetAsync(rho_out, 0, static_cast<size_t>(m) * sizeof(float), s));
  if (np == 0) return HRT_OK;
  if (!err) HRT_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_tile_err));
  FieldMaps maps{};
  if (mode == kTilesTma) {
    EncodeTiled enc = nullptr;
    HRT_TRY(tensor_map_encoder(&enc));
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(n)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(n) * sizeof(float),
                                   static_cast<cuuint64_t>(n) * n * sizeof(float)};
    const cuuint32_t tbox[3] = {kTileZ, kTileY, kTileX};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int c = 0; c < 3; ++c) {
      const CUresult r = enc(&maps.m[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(grad + c * m), dims,
                             strides, tbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return fail(HRT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    }
  }
  HRT_CUDA(cudaFuncSetAttribute(kick_drift_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kTileSmem)));
  const Lattice L = make_lattice(n_side, n, box, order);
  const unsigned bricks = static_cast<unsigned>(m / (kBrickXY * kBrickXY * kBrickZ));
  kick_drift_tiled_kernel<<<bricks, kTileThreads, kTileSmem, s>>>(
      maps, mode == kTilesTma ? 1 : 0, grad, grad + m, grad + 2 * m, L, np, key_start, disp, mom,
      static_cast<float>(kick), static_cast<float>(drift), particle_mass(n_side, n), rho_out, err);
  HRT_LAUNCHED("kick_drift_tiled_kernel");
  return HRT_OK;
}

hrt_status launch_kick_drift(const float* grad, int64_t n, double box, int64_t n_side, float* disp, float* mom,
                             double kick, double drift, cudaStream_t s, float* rho_out, const int32_t* order,
                             bool rho_zeroed) {
  int64_t np = n_side * n_side * n_side;
  int64_t m = n * n * n;
  if (rho_out && !rho_zeroed) HRT_CUDA(cudaMemsetAsync(rho_out, 0, static_cast<size_t>(m) * sizeof(float), s));
  if (np == 0) return HRT_OK;
  const Lattice L = make_lattice(n_side, n, box, order);
  const dim3 grid = particle_grid(n_side, 256, order);
  if (rho_out) {
    kick_drift_kernel<true><<<grid, 256, 0, s>>>(grad, grad + m, grad + 2 * m, L, np, disp, mom,
                                                 static_cast<float>(kick), static_cast<float>(drift),
                                                 particle_mass(n_side, n), rho_out);
  } else {
    kick_drift_kernel<false><<<grid, 256, 0, s>>>(grad, grad + m, grad + 2 * m, L, np, disp, mom,
                                                  static_cast<float>(kick), static_cast<float>(drift), 0.f, nullptr);
  }
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

// ---------------------------------------------------------------------------------------------------------
// Second-order Lagrangian ICs (2LPT): with c = table(|n|^2) = sqrt(P / V_cell) / k^2 / n^3 (unit growth), the
// Hessian spectra of phi1 are d_i d_j c w_hat (set 0: xx, yy, zz; set 1: xy, xz, yz); the source
// S = sum_{i<j} (phi1_ii phi1_jj - phi1_ij^2) is formed in real space; Psi2 = grad phi2 with lap phi2 = S is
// -i d_j S_hat / (k^2 n^3).  Derivative factors are zero on their Nyquist planes.
// ---------------------------------------------------------------------------------------------------------
__global__ void ic_hessian_kernel(const float2* __restrict__ w_hat, int n, int nzc, float kf,
                                  const float* __restrict__ table, int64_t elems, int set, float2* __restrict__ out) {
  const int iz = blockIdx.y * blockDim.x + threadIdx.x;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.y + threadIdx.y;
  if (iz >= nzc || row >= static_cast<int64_t>(n) * n) return;
  const int ix = static_cast<int>(row / n);
  const int iy = static_cast<int>(row - static_cast<int64_t>(ix) * n);
  const int half = n >> 1;
  const int nx = ix < half ? ix : ix - n, ny = iy < half ? iy : iy - n, nz = iz;
  const int64_t e = row * nzc + iz;
  const float c = __ldg(table + (nx * nx + ny * ny + nz * nz));
  const float2 v = w_hat[e];
  const float dx = (nx == -half) ? 0.f : kf * nx;
  const float dy = (ny == -half) ? 0.f : kf * ny;
  const float dz = (nz == half) ? 0.f : kf * nz;
  const float f0 = set == 0 ? dx * dx : dx * dy;
  const float f1 = set == 0 ? dy * dy : dx * dz;
  const float f2 = set == 0 ? dz * dz : dy * dz;
  out[e] = make_float2(f0 * c * v.x, f0 * c * v.y);
  out[e + elems] = make_float2(f1 * c * v.x, f1 * c * v.y);
  out[e + 2 * elems] = make_float2(f2 * c * v.x, f2 * c * v.y);
}

hrt_status launch_ic_hessian(const void* w_hat, int64_t n, double box, const float* table, int set, void* out,
                             cudaStream_t s) {
  const int64_t nzc = n / 2 + 1;
  dim3 block(64, 4);
  dim3 grid(static_cast<unsigned>((n * n + 3) / 4), static_cast<unsigned>((nzc + 63) / 64));
  ic_hessian_kernel<<<grid, block, 0, s>>>(static_cast<const float2*>(w_hat), static_cast<int>(n),
                                           static_cast<int>(nzc), static_cast<float>(2.0 * M_PI / box), table,
                                           n * n * nzc, set, static_cast<float2*>(out));
  HRT_LAUNCHED("ic_hessian_kernel");
  return HRT_OK;
}

// h: six fields of m values (xx, yy, zz, xy, xz, yz); out may alias h (field xx).
__global__ void lpt2_source_kernel(const float* h, int64_t m, float* out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= m) return;
  const float xx = h[i], yy = h[i + m], zz = h[i + 2 * m], xy = h[i + 3 * m], xz = h[i + 4 * m], yz = h[i + 5 * m];
  out[i] = (xx * yy - xy * xy) + (xx * zz - xz * xz) + (yy * zz - yz * yz);
}

hrt_status launch_lpt2_source(const float* h, int64_t m, float* out, cudaStream_t s) {
  lpt2_source_kernel<<<blocks_for(m, 256), 256, 0, s>>>(h, m, out);
  HRT_LAUNCHED("lpt2_source_kernel");
  return HRT_OK;
}

__global__ void lpt2_kspace_kernel(const float2* __restrict__ s_hat, int n, int nzc, float kf, float inv_n3,
                                   int64_t elems, float2* __restrict__ out) {
  const int iz = blockIdx.y * blockDim.x + threadIdx.x;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.y + threadIdx.y;
  if (iz >= nzc || row >= static_cast<int64_t>(n) * n) return;
  const int ix = static_cast<int>(row / n);
  const int iy = static_cast<int>(row - static_cast<int64_t>(ix) * n);
  const int half = n >> 1;
  const int nx = ix < half ? ix : ix - n, ny = iy < half ? iy : iy - n, nz = iz;
  const int64_t e = row * nzc + iz;
  const float k2 = kf * kf * static_cast<float>(nx * nx + ny * ny + nz * nz);
  const float c = k2 > 0.f ? inv_n3 / k2 : 0.f;
  const float2 v = s_hat[e];
  const float2 base = make_float2(c * v.y, -c * v.x);  // -i S_hat / (k^2 n^3)
  const float dx = (nx == -half) ? 0.f : kf * nx;
  const float dy = (ny == -half) ? 0.f : kf * ny;
  const float dz = (nz == half) ? 0.f : kf * nz;
  out[e] = make_float2(dx * base.x, dx * base.y);
  out[e + elems] = make_float2(dy * base.x, dy * base.y);
  out[e + 2 * elems] = make_float2(dz * base.x, dz * base.y);
}

hrt_status launch_lpt2_kspace(const void* s_hat, int64_t n, double box, void* out, cudaStream_t s) {
  const int64_t nzc = n / 2 + 1;
  dim3 block(64, 4);
  dim3 grid(static_cast<unsigned>((n * n + 3) / 4), static_cast<unsigned>((nzc + 63) / 64));
  lpt2_kspace_kernel<<<grid, block, 0, s>>>(static_cast<const float2*>(s_hat), static_cast<int>(n),
                                            static_cast<int>(nzc), static_cast<float>(2.0 * M_PI / box),
                                            static_cast<float>(1.0 / (static_cast<double>(n) * n * n)), n * n * nzc,
                                            static_cast<float2*>(out));
  HRT_LAUNCHED("lpt2_kspace_kernel");
  return HRT_OK;
}

// disp = d1 psi1 + d2 psi2, mom = c1 psi1 + c2 psi2 (disp may alias psi1).
__global__ void lpt_combine_kernel(const float* psi1, const float* __restrict__ psi2, int64_t m, float d1, float d2,
                                   float c1, float c2, float* disp, float* __restrict__ mom) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= m) return;
  const float a = psi1[i], b = psi2[i];
  disp[i] = d1 * a + d2 * b;
  mom[i] = c1 * a + c2 * b;
}

hrt_status launch_lpt_combine(const float* psi1, const float* psi2, int64_t m, double d1, double d2, double c1,
                              double c2, float* disp, float* mom, cudaStream_t s) {
  lpt_combine_kernel<<<blocks_for(m, 256), 256, 0, s>>>(psi1, psi2, m, static_cast<float>(d1), static_cast<float>(d2),
                                                        static_cast<float>(c1), static_cast<float>(c2), disp, mom);
  HRT_LAUNCHED("lpt_combine_kernel");
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

// ---------------------------------------------------------------------------------------------------------
// Non-finite scan (opt-in checks of the context): one warp vote per 32 values, one atomic per warp that saw one.
// ---------------------------------------------------------------------------------------------------------
template <typename T>
__global__ void nonfinite_scan_kernel(const T* __restrict__ p, int64_t n, int* __restrict__ flag) {
  bool bad = false;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    bad |= !isfinite(p[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

template <typename T>
static hrt_status scan(const T* p, int64_t n, int* flag, cudaStream_t s) {
  if (n <= 0) return HRT_OK;
  int dev = 0, sms = 0;
  HRT_TRY(cuda_status(cudaGetDevice(&dev), "cudaGetDevice"));
  HRT_TRY(cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count"));
  const unsigned grid = std::min<unsigned>(blocks_for(n, 256), static_cast<unsigned>(sms) * 8);
  nonfinite_scan_kernel<T><<<grid, 256, 0, s>>>(p, n, flag);
  HRT_LAUNCHED("nonfinite_scan_kernel");
  return HRT_OK;
}

hrt_status launch_nonfinite_scan(const float* p, int64_t n, int* flag, cudaStream_t s) { return scan(p, n, flag, s); }
hrt_status launch_nonfinite_scan(const double* p, int64_t n, int* flag, cudaStream_t s) { return scan(p, n, flag, s); }

}  // namespace hrt
