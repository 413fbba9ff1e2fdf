// Adjoint (reverse-mode) kernels of the HRT hot path: the vector-Jacobian products of the CIC deposit, the
// k-space Poisson/gradient kernel, the particle kick-drift and the ray KDK step with its A/B recursion, plus
// the kappa power-spectrum and Zel'dovich-IC adjoints.  Each kernel recomputes what it needs of the forward
// step from the pre-step state (no forward intermediates are stored) and accumulates
//   - field cotangents into the adjoint meshes with float32 reductions (the transposes of the CIC gathers),
//   - cotangents of the host coefficients (kick and drift factors, line-of-sight node weights and positions)
//     into FP64 accumulators, so the host can chain them with the FP64 derivatives of those coefficients.
#include <cuda_runtime.h>

#include <cmath>

#include "adjoint.h"
#include "common.h"
#include "mesh_kernels.h"

namespace hrt {

__device__ __forceinline__ void axis_split(int base, float d_cells, int n, int& i0, float& f) {
  float fl = floorf(d_cells);
  f = d_cells - fl;
  int i = base + static_cast<int>(fl);
  if (static_cast<unsigned>(i) >= static_cast<unsigned>(n)) {
    i %= n;
    if (i < 0) i += n;
  }
  i0 = i;
}

__device__ __forceinline__ int nxt(int i, int n) { return i + 1 == n ? 0 : i + 1; }

// Corner c = (a, b, e) in bits (a = x bit 2, b = y bit 1, e = z bit 0) of the cell with lower node (ix, iy, iz).
struct Cell {
  int64_t idx[8];
  float fx, fy, fz;
};

__device__ __forceinline__ void make_cell(int ix, int iy, int iz, float fx, float fy, float fz, int n, Cell& c) {
  const int jx = nxt(ix, n), jy = nxt(iy, n), jz = nxt(iz, n);
  const int64_t nn = n;
  const int64_t r[4] = {(ix * nn + iy) * nn, (ix * nn + jy) * nn, (jx * nn + iy) * nn, (jx * nn + jy) * nn};
  for (int k = 0; k < 4; ++k) {
    c.idx[2 * k] = r[k] + iz;
    c.idx[2 * k + 1] = r[k] + jz;
  }
  c.fx = fx;
  c.fy = fy;
  c.fz = fz;
}

// Trilinear weight of corner k and its derivatives with respect to the fractional coordinates.
__device__ __forceinline__ float wgt(int k, float fx, float fy, float fz) {
  return ((k & 4) ? fx : 1.f - fx) * ((k & 2) ? fy : 1.f - fy) * ((k & 1) ? fz : 1.f - fz);
}
__device__ __forceinline__ float dw(int k, int axis, float fx, float fy, float fz) {
  const float sx = (k & 4) ? 1.f : -1.f, sy = (k & 2) ? 1.f : -1.f, sz = (k & 1) ? 1.f : -1.f;
  const float wx = (k & 4) ? fx : 1.f - fx, wy = (k & 2) ? fy : 1.f - fy, wz = (k & 1) ? fz : 1.f - fz;
  return axis == 0 ? sx * wy * wz : (axis == 1 ? wx * sy * wz : wx * wy * sz);
}
__device__ __forceinline__ void block_add_double(double v, double* dst) {
  // warp reduction, then one atomic per warp
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dst, v);
}

// ---------------------------------------------------------------------------------------------------------
// Particles: lattice mapping (row mode only: adjoint workloads are small) and the kick-drift adjoint.
// ---------------------------------------------------------------------------------------------------------
struct AdjLattice {
  int n_side, ratio, n;
  float inv_cell;
  int64_t np;
};

__device__ __forceinline__ bool adj_particle(const AdjLattice& L, int64_t& p, int& qi, int& qj, int& qk) {
  p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= L.np) return false;
  qk = static_cast<int>(p % L.n_side);
  const int64_t t = p / L.n_side;
  qj = static_cast<int>(t % L.n_side);
  qi = static_cast<int>(t / L.n_side);
  return true;
}

__device__ __forceinline__ void cell_of(const AdjLattice& L, int qi, int qj, int qk, float d0, float d1, float d2,
                                        Cell& c) {
  int ix, iy, iz;
  float fx, fy, fz;
  axis_split(qi * L.ratio, d0 * L.inv_cell, L.n, ix, fx);
  axis_split(qj * L.ratio, d1 * L.inv_cell, L.n, iy, fy);
  axis_split(qk * L.ratio, d2 * L.inv_cell, L.n, iz, fz);
  make_cell(ix, iy, iz, fx, fy, fz, L.n, c);
}

// disp_bar += mass * sum_c rho_bar[c] d w_c / d x   (transpose of the CIC deposit)
__global__ void deposit_adjoint_kernel(const float* __restrict__ rho_bar, const float* __restrict__ disp, AdjLattice L,
                                       float mass, float* __restrict__ disp_bar) {
  int64_t p;
  int qi, qj, qk;
  if (!adj_particle(L, p, qi, qj, qk)) return;
  Cell c;
  cell_of(L, qi, qj, qk, disp[p], disp[p + L.np], disp[p + 2 * L.np], c);
  float g[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < 8; ++k) {
    const float r = __ldg(rho_bar + c.idx[k]);
    for (int a = 0; a < 3; ++a) g[a] += r * dw(k, a, c.fx, c.fy, c.fz);
  }
  const float s = mass * L.inv_cell;
  for (int a = 0; a < 3; ++a) disp_bar[p + a * L.np] += s * g[a];
}

// Kick-drift adjoint.  Forward: m' = m - K g(x), d' = d + D m', x = q + d; optionally the deposit of d'.
// In: d, m (pre-step), d_bar and m_bar holding the cotangents of d', m' (overwritten with those of d, m).
__global__ void kick_drift_adjoint_kernel(const float* __restrict__ gx, const float* __restrict__ gy,
                                          const float* __restrict__ gz, AdjLattice L, const float* __restrict__ disp,
                                          const float* __restrict__ mom, float kick, float drift,
                                          const float* __restrict__ rho_bar, float mass, float* __restrict__ disp_bar,
                                          float* __restrict__ mom_bar, float* __restrict__ gbx, float* __restrict__ gby,
                                          float* __restrict__ gbz, double* __restrict__ coef_bar) {
  int64_t p;
  int qi, qj, qk;
  double kbar = 0.0, dbar = 0.0;
  if (adj_particle(L, p, qi, qj, qk)) {
    const int64_t np = L.np;
    const float d[3] = {disp[p], disp[p + np], disp[p + 2 * np]};
    const float m[3] = {mom[p], mom[p + np], mom[p + 2 * np]};
    Cell c;
    cell_of(L, qi, qj, qk, d[0], d[1], d[2], c);
    const float* f[3] = {gx, gy, gz};
    float g[3] = {0.f, 0.f, 0.f}, G[3][3] = {{0.f}};  // G[a][b] = d g_a / d f_b (per cell)
    for (int k = 0; k < 8; ++k) {
      const float w = wgt(k, c.fx, c.fy, c.fz);
      const float dwk[3] = {dw(k, 0, c.fx, c.fy, c.fz), dw(k, 1, c.fx, c.fy, c.fz), dw(k, 2, c.fx, c.fy, c.fz)};
      for (int a = 0; a < 3; ++a) {
        const float v = __ldg(f[a] + c.idx[k]);
        g[a] += w * v;
        for (int b = 0; b < 3; ++b) G[a][b] += dwk[b] * v;
      }
    }
    float m1[3], d1[3];
    for (int a = 0; a < 3; ++a) {
      m1[a] = m[a] - kick * g[a];
      d1[a] = d[a] + drift * m1[a];
    }
    float db[3] = {disp_bar[p], disp_bar[p + np], disp_bar[p + 2 * np]};
    float mb[3] = {mom_bar[p], mom_bar[p + np], mom_bar[p + 2 * np]};
    if (rho_bar != nullptr) {  // transpose of the fused deposit at the drifted position
      Cell c1;
      cell_of(L, qi, qj, qk, d1[0], d1[1], d1[2], c1);
      for (int k = 0; k < 8; ++k) {
        const float r = __ldg(rho_bar + c1.idx[k]);
        for (int a = 0; a < 3; ++a) db[a] += mass * L.inv_cell * r * dw(k, a, c1.fx, c1.fy, c1.fz);
      }
    }
    float mt[3];
    for (int a = 0; a < 3; ++a) {
      mt[a] = mb[a] + drift * db[a];
      dbar += static_cast<double>(m1[a]) * db[a];
      kbar -= static_cast<double>(g[a]) * mt[a];
    }
    // field cotangents: g_a = sum_k w_k v_ak  ->  v_bar_ak += -K w_k mt_a
    float* fb[3] = {gbx, gby, gbz};
    for (int k = 0; k < 8; ++k) {
      const float w = -kick * wgt(k, c.fx, c.fy, c.fz);
      for (int a = 0; a < 3; ++a) atomicAdd(fb[a] + c.idx[k], w * mt[a]);
    }
    for (int b = 0; b < 3; ++b) {
      float s = 0.f;
      for (int a = 0; a < 3; ++a) s += G[a][b] * mt[a];
      disp_bar[p + b * np] = db[b] - kick * L.inv_cell * s;
      mom_bar[p + b * np] = mt[b];
    }
  }
  block_add_double(kbar, coef_bar);
  block_add_double(dbar, coef_bar + 1);
}

hrt_status launch_deposit_adjoint(const float* rho_bar, const float* disp, int64_t n_side, int64_t n, double box,
                                  float* disp_bar, cudaStream_t s) {
  const int64_t np = n_side * n_side * n_side;
  AdjLattice L{static_cast<int>(n_side), static_cast<int>(n / n_side), static_cast<int>(n),
               static_cast<float>(n / box), np};
  const float mass = static_cast<float>(static_cast<double>(n) * n * n / static_cast<double>(np));
  deposit_adjoint_kernel<<<blocks_for(np, 256), 256, 0, s>>>(rho_bar, disp, L, mass, disp_bar);
  HRT_LAUNCHED("deposit_adjoint_kernel");
  return HRT_OK;
}

hrt_status launch_kick_drift_adjoint(const float* grad, int64_t n, double box, int64_t n_side, const float* disp,
                                     const float* mom, double kick, double drift, const float* rho_bar,
                                     float* disp_bar, float* mom_bar, float* grad_bar, double* coef_bar,
                                     cudaStream_t s) {
  const int64_t np = n_side * n_side * n_side, m = n * n * n;
  AdjLattice L{static_cast<int>(n_side), static_cast<int>(n / n_side), static_cast<int>(n),
               static_cast<float>(n / box), np};
  const float mass = static_cast<float>(static_cast<double>(n) * n * n / static_cast<double>(np));
  kick_drift_adjoint_kernel<<<blocks_for(np, 256), 256, 0, s>>>(
      grad, grad + m, grad + 2 * m, L, disp, mom, static_cast<float>(kick), static_cast<float>(drift), rho_bar, mass,
      disp_bar, mom_bar, grad_bar, grad_bar + m, grad_bar + 2 * m, coef_bar);
  HRT_LAUNCHED("kick_drift_adjoint_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// k-space adjoint: out = sum_j conj(H_j) in_j with H_j = i d_j * scale / k^2 * Wx Wy Wz g(|k|); conj(H_j) = -H_j.
// ---------------------------------------------------------------------------------------------------------
__global__ void kspace_adjoint_kernel(const float2* __restrict__ in, int n, int nzc, float kf, float scale,
                                      int64_t elems, const float* __restrict__ wx, const float* __restrict__ wz,
                                      const float* __restrict__ gtab, int g_nk, float g_inv_dk, int n_in,
                                      int accumulate, float2* __restrict__ out) {
  const int iz = blockIdx.y * blockDim.x + threadIdx.x;
  const unsigned row = blockIdx.x * blockDim.y + threadIdx.y;
  if (iz >= nzc || row >= static_cast<unsigned>(n) * static_cast<unsigned>(n)) return;
  const int ix = static_cast<int>(row / static_cast<unsigned>(n));
  const int iy = static_cast<int>(row - static_cast<unsigned>(ix) * n);
  const int half = n >> 1;
  const int nx = ix < half ? ix : ix - n, ny = iy < half ? iy : iy - n;
  const float kx = kf * nx, ky = kf * ny, kz = kf * iz;
  const float k2 = kx * kx + ky * ky + kz * kz;
  const int64_t e = static_cast<int64_t>(row) * nzc + iz;
  float c = k2 > 0.f ? scale / k2 * __ldg(wx + ix) * __ldg(wx + iy) * __ldg(wz + iz) : 0.f;
  if (gtab != nullptr && k2 > 0.f) {
    const float t = sqrtf(k2) * g_inv_dk;
    if (t < static_cast<float>(g_nk - 1)) {
      const int i = static_cast<int>(t);
      const float w = t - static_cast<float>(i);
      c *= __ldg(gtab + i) * (1.f - w) + __ldg(gtab + i + 1) * w;
    }
  }
  const float d[3] = {(nx == -half) ? 0.f : kx, (ny == -half) ? 0.f : ky, (iz == half) ? 0.f : kz};
  float2 acc = make_float2(0.f, 0.f);
  for (int j = 0; j < n_in; ++j) {
    const float2 v = in[e + j * elems];
    const float cd = -c * d[j];  // -(i c d) v = (c d v.y, -c d v.x)
    acc.x += -cd * v.y;
    acc.y += cd * v.x;
  }
  if (accumulate) {
    const float2 o = out[e];
    acc.x += o.x;
    acc.y += o.y;
  }
  out[e] = acc;
}

hrt_status launch_kspace_adjoint(const void* in, int n_in, int64_t n, double box, double pref, const float* tab,
                                 const hrt_filter* f, void* out, bool accumulate, cudaStream_t s) {
  const int64_t nzc = n / 2 + 1;
  const double scale = -pref / (static_cast<double>(n) * n * n);
  dim3 block(64, 4);
  dim3 grid(static_cast<unsigned>((n * n + 3) / 4), static_cast<unsigned>((nzc + 63) / 64));
  kspace_adjoint_kernel<<<grid, block, 0, s>>>(
      static_cast<const float2*>(in), static_cast<int>(n), static_cast<int>(nzc), static_cast<float>(2.0 * M_PI / box),
      static_cast<float>(scale), n * n * nzc, tab, tab + n, f->g_table, f->g_nk,
      f->g_table ? static_cast<float>((f->g_nk - 1) / f->g_kmax) : 0.f, n_in, accumulate ? 1 : 0,
      static_cast<float2*>(out));
  HRT_LAUNCHED("kspace_adjoint_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// Ray KDK step adjoint.
// ---------------------------------------------------------------------------------------------------------
struct RayNodeSample {
  Cell c;
  float v[2];        // value of (gx, gy)
  float D[2][3];     // d v_a / d f_b (per cell), b = x, y, z
  float S[2][3][3];  // mixed second derivatives d^2 v_a / d f_b d f_c
};

// Mesh columns of node j: row offsets of the four (x, y) corners (ix,iy), (ix,jy), (jx,iy), (jx,jy), the two z
// planes and the fractional position (the same arithmetic as the forward kernel).
struct NodeCols {
  int64_t r[4];
  int iz, jz;
  float fx, fy, fz;
};

__device__ __forceinline__ void node_cols(const RayStepParams& p, int j, int bx, float fbx, int by, float fby,
                                          float tx, float ty, NodeCols& c) {
  const int n = p.n;
  int ix, iy;
  axis_split(bx, fbx + p.dr[j] * tx, n, ix, c.fx);
  axis_split(by, fby + p.dr[j] * ty, n, iy, c.fy);
  c.iz = p.kz[j];
  c.jz = nxt(c.iz, n);
  c.fz = p.fz[j];
  const int jx = nxt(ix, n), jy = nxt(iy, n);
  const int64_t nn = n;
  c.r[0] = (ix * nn + iy) * nn;
  c.r[1] = (ix * nn + jy) * nn;
  c.r[2] = (jx * nn + iy) * nn;
  c.r[3] = (jx * nn + jy) * nn;
}

// Trilinear interpolant of one field at a node and its derivatives in the fractional position: value v,
// gradient (dx, dy, dz) and the mixed second derivatives (the pure ones vanish for a trilinear interpolant),
// by successive linear interpolation in z, y, x.
struct NodeField {
  float v, dx, dy, dz, sxy, sxz, syz;
};

__device__ __forceinline__ NodeField node_field(const float* __restrict__ f, const NodeCols& c) {
  float lo[4], dzc[4], e[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    lo[q] = __ldg(f + c.r[q] + c.iz);
    dzc[q] = __ldg(f + c.r[q] + c.jz) - lo[q];
    e[q] = lo[q] + c.fz * dzc[q];
  }
  NodeField o;
  const float h0 = e[1] - e[0], h1 = e[3] - e[2];  // d/dfy at x = 0, 1
  const float g0 = e[0] + c.fy * h0, g1 = e[2] + c.fy * h1;
  o.v = g0 + c.fx * (g1 - g0);
  o.dx = g1 - g0;
  o.dy = h0 + c.fx * (h1 - h0);
  o.sxy = h1 - h0;
  const float z0 = dzc[0] + c.fy * (dzc[1] - dzc[0]), z1 = dzc[2] + c.fy * (dzc[3] - dzc[2]);
  o.dz = z0 + c.fx * (z1 - z0);
  o.sxz = z1 - z0;
  o.syz = (dzc[1] - dzc[0]) + c.fx * ((dzc[3] - dzc[2]) - (dzc[1] - dzc[0]));
  return o;
}

__device__ __forceinline__ void base_pos(double obs, double r_ref, double theta, double cell, int n, int& i0,
                                         float& f0) {
  double u = (obs + r_ref * theta) / cell;
  u -= n * floor(u / n);
  double fl = floor(u);
  i0 = static_cast<int>(fl);
  if (i0 >= n) i0 -= n;
  f0 = static_cast<float>(u - fl);
}

// Forward half kick (K, J) at theta, as in the forward kernel.
__device__ void half_forward(const RayStepParams& p, int j0, int j1, double thx, double thy, double ref_r,
                             const float* __restrict__ gx, const float* __restrict__ gy, float K[2], float J[2][2]) {
  K[0] = K[1] = 0.f;
  J[0][0] = J[0][1] = J[1][0] = J[1][1] = 0.f;
  if (j1 <= j0) return;
  int bx, by;
  float fbx, fby;
  base_pos(p.obs_x, ref_r, thx, p.cell, p.n, bx, fbx);
  base_pos(p.obs_y, ref_r, thy, p.cell, p.n, by, fby);
  const float tx = static_cast<float>(thx), ty = static_cast<float>(thy);
  const float* f[2] = {gx, gy};
  for (int j = j0; j < j1; ++j) {
    NodeCols c;
    node_cols(p, j, bx, fbx, by, fby, tx, ty, c);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const NodeField o = node_field(f[a], c);
      K[a] += p.cw[j] * o.v;
      J[a][0] += p.cwr[j] * o.dx;
      J[a][1] += p.cwr[j] * o.dy;
    }
  }
}

// Backward of one half kick: given Kbar, Jbar, accumulate theta_bar (FP64-free float32), field cotangents and the
// node-coefficient cotangents (per block, in shared memory: [3][n_nodes] = cw_bar, cwr_bar, chi_bar).
__device__ void half_backward(const RayStepParams& p, int j0, int j1, double thx, double thy, double ref_r,
                              const float* __restrict__ gx, const float* __restrict__ gy, const float Kb[2],
                              const float Jb[2][2], float* __restrict__ gbx, float* __restrict__ gby, float thb[2],
                              float* __restrict__ sh_nodes, int n_nodes, bool active) {
  if (j1 <= j0) return;
  int bx = 0, by = 0;
  float fbx = 0.f, fby = 0.f;
  if (active) {
    base_pos(p.obs_x, ref_r, thx, p.cell, p.n, bx, fbx);
    base_pos(p.obs_y, ref_r, thy, p.cell, p.n, by, fby);
  }
  const float tx = static_cast<float>(thx), ty = static_cast<float>(thy);
  const float inv_cell = static_cast<float>(1.0 / p.cell);
  const float* f[2] = {gx, gy};
  float* fb[2] = {gbx, gby};
  const int lane = threadIdx.x & 31;
  for (int j = j0; j < j1; ++j) {
    float cwb = 0.f, cwrb = 0.f, chib = 0.f;
    NodeCols c{};
    float t[2][4][2] = {};  // field cotangent per field, (x, y) corner and z plane
    if (active) {
      node_cols(p, j, bx, fbx, by, fby, tx, ty, c);
      const float cw = p.cw[j], cwr = p.cwr[j];
      float fbar_x = 0.f, fbar_y = 0.f, fbar_z = 0.f;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const NodeField o = node_field(f[a], c);
        // K_a = cw v_a and J_ab = cwr d_b v_a (b = x, y): cotangent weights of v, dx v, dy v
        const float al = cw * Kb[a], bex = cwr * Jb[a][0], bey = cwr * Jb[a][1];
        // field cotangents: w_k = WX WY WZ, d w_k / d fx = SX WY WZ, ... -> per (x, y) corner, times WZ
        const float ux = 1.f - c.fx, uy = 1.f - c.fy;
        const float q[4] = {al * ux * uy - bex * uy - bey * ux, al * ux * c.fy - bex * c.fy + bey * ux,
                            al * c.fx * uy + bex * uy - bey * c.fx, al * c.fx * c.fy + bex * c.fy + bey * c.fx};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          t[a][k][0] = (1.f - c.fz) * q[k];
          t[a][k][1] = c.fz * q[k];
        }
        // cotangent of the fractional position (the mixed second derivatives couple the J terms)
        fbar_x += al * o.dx + bey * o.sxy;
        fbar_y += al * o.dy + bex * o.sxy;
        fbar_z += al * o.dz + bex * o.sxz + bey * o.syz;
        cwb += Kb[a] * o.v;
        cwrb += Jb[a][0] * o.dx + Jb[a][1] * o.dy;
      }
      // f_x = (O_x + chi_j theta_x) / cell - cell index: d f_x / d theta_x = chi_j / cell, d f / d chi_j = theta/cell
      const float r_over_cell = static_cast<float>(ref_r / p.cell) + p.dr[j];
      thb[0] += fbar_x * r_over_cell;
      thb[1] += fbar_y * r_over_cell;
      chib = (fbar_x * tx + fbar_y * ty + fbar_z) * inv_cell;
    }
    // Neighbouring rays of a warp mostly share the node's mesh cell: lanes with the same cell that follow
    // each other form a segment, the segment's cotangents are summed by a segmented shuffle reduction and its
    // first lane issues the 16 atomics (a cell that reappears later in the warp starts a new segment).
    const long long key = active ? static_cast<long long>(c.r[0] + c.iz) : -1ll - lane;
    const long long prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned above = lane == 31 ? 0u : heads & (0xffffffffu << (lane + 1));
    const int seg_end = above ? __ffs(above) - 2 : 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1)
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int z = 0; z < 2; ++z) {
            const float u = __shfl_down_sync(0xffffffffu, t[a][k][z], d);
            if (lane + d <= seg_end) t[a][k][z] += u;
          }
    if (head && active) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (t[a][k][0] != 0.f) atomicAdd(fb[a] + c.r[k] + c.iz, t[a][k][0]);
          if (t[a][k][1] != 0.f) atomicAdd(fb[a] + c.r[k] + c.jz, t[a][k][1]);
        }
    }
    // block reduction of the node cotangents into shared memory
    for (int o = 16; o > 0; o >>= 1) {
      cwb += __shfl_down_sync(0xffffffffu, cwb, o);
      cwrb += __shfl_down_sync(0xffffffffu, cwrb, o);
      chib += __shfl_down_sync(0xffffffffu, chib, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(sh_nodes + j, cwb);
      atomicAdd(sh_nodes + n_nodes + j, cwrb);
      atomicAdd(sh_nodes + 2 * n_nodes + j, chib);
    }
  }
}

// ---- light-cone tiling (the forward's half_kick_tiled): the node's sky-frame cell and fraction per sky axis map
// to a box axis through the replica's axis permutation, sign and translation.
__device__ __forceinline__ void box_axis_t(int i_s, float f_s, int sgn, int sh, int n, int& ib, float& fb) {
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
  ib %= n;
  if (ib < 0) ib += n;
}

// Box-frame columns of tiled node j (as node_cols), the replica's axes p[3] (box axis of sky x, y, line of
// sight) and signs sg[3].
__device__ __forceinline__ void node_cols_tiled(const RayStepParams& p, int j, int bx, float fbx, int by, float fby,
                                                float tx, float ty, NodeCols& c, int pa[3], int sg[3]) {
  const int n = p.n;
  int ix, iy;
  float fx, fy;
  axis_split(bx, fbx + p.dr[j] * tx, n, ix, fx);
  axis_split(by, fby + p.dr[j] * ty, n, iy, fy);
  const int R = p.rep[j];
  pa[0] = p.rperm[R][0];
  pa[1] = p.rperm[R][1];
  pa[2] = 3 - pa[0] - pa[1];
  sg[0] = p.rsign[R][0];
  sg[1] = p.rsign[R][1];
  sg[2] = p.rsign[R][2];
  int cb[3];
  float fb[3];
  box_axis_t(ix, fx, sg[0], p.rshift[R][0], n, cb[pa[0]], fb[pa[0]]);
  box_axis_t(iy, fy, sg[1], p.rshift[R][1], n, cb[pa[1]], fb[pa[1]]);
  cb[pa[2]] = p.kz[j];
  fb[pa[2]] = p.fz[j];
  c.fx = fb[0];
  c.fy = fb[1];
  c.fz = fb[2];
  c.iz = cb[2];
  c.jz = nxt(cb[2], n);
  const int jx = nxt(cb[0], n), jy = nxt(cb[1], n);
  const int64_t nn = n;
  c.r[0] = (cb[0] * nn + cb[1]) * nn;
  c.r[1] = (cb[0] * nn + jy) * nn;
  c.r[2] = (jx * nn + cb[1]) * nn;
  c.r[3] = (jx * nn + jy) * nn;
}

__device__ __forceinline__ float nf_d(const NodeField& o, int a) { return a == 0 ? o.dx : (a == 1 ? o.dy : o.dz); }
// mixed second derivative along box axes a != b (zero for a == b: the interpolant is linear per axis)
__device__ __forceinline__ float nf_s(const NodeField& o, int a, int b) {
  if (a == b) return 0.f;
  const int m = a + b;  // 1: xy, 2: xz, 3: yz
  return m == 1 ? o.sxy : (m == 2 ? o.sxz : o.syz);
}

__device__ void half_forward_tiled(const RayStepParams& p, int j0, int j1, double thx, double thy, double ref_r,
                                   const float* __restrict__ gx, const float* __restrict__ gy,
                                   const float* __restrict__ gz, float K[2], float J[2][2]) {
  K[0] = K[1] = 0.f;
  J[0][0] = J[0][1] = J[1][0] = J[1][1] = 0.f;
  if (j1 <= j0) return;
  int bx, by;
  float fbx, fby;
  base_pos(p.obs_x, ref_r, thx, p.cell, p.n, bx, fbx);
  base_pos(p.obs_y, ref_r, thy, p.cell, p.n, by, fby);
  const float tx = static_cast<float>(thx), ty = static_cast<float>(thy);
  const float* f3[3] = {gx, gy, gz};
  for (int j = j0; j < j1; ++j) {
    NodeCols c;
    int pa[3], sg[3];
    node_cols_tiled(p, j, bx, fbx, by, fby, tx, ty, c, pa, sg);
    const NodeField oa = node_field(f3[pa[0]], c), ob = node_field(f3[pa[1]], c);
    const float ss = static_cast<float>(sg[0] * sg[1]);
    K[0] += p.cw[j] * (sg[0] * oa.v);
    K[1] += p.cw[j] * (sg[1] * ob.v);
    J[0][0] += p.cwr[j] * nf_d(oa, pa[0]);
    J[0][1] += p.cwr[j] * (ss * nf_d(oa, pa[1]));
    J[1][0] += p.cwr[j] * (ss * nf_d(ob, pa[0]));
    J[1][1] += p.cwr[j] * nf_d(ob, pa[1]);
  }
}

// Backward of one tiled half kick (as half_backward): the sky components are sign-weighted box fields g_{p0},
// g_{p1}, and the derivative of sky axis b is sign_b d / d(box axis p_b).
__device__ void half_backward_tiled(const RayStepParams& p, int j0, int j1, double thx, double thy, double ref_r,
                                    const float* __restrict__ gx, const float* __restrict__ gy,
                                    const float* __restrict__ gz, const float Kb[2], const float Jb[2][2],
                                    float* __restrict__ gbx, float* __restrict__ gby, float* __restrict__ gbz,
                                    float thb[2], float* __restrict__ sh_nodes, int n_nodes, bool active) {
  if (j1 <= j0) return;
  int bx = 0, by = 0;
  float fbx = 0.f, fby = 0.f;
  if (active) {
    base_pos(p.obs_x, ref_r, thx, p.cell, p.n, bx, fbx);
    base_pos(p.obs_y, ref_r, thy, p.cell, p.n, by, fby);
  }
  const float tx = static_cast<float>(thx), ty = static_cast<float>(thy);
  const float inv_cell = static_cast<float>(1.0 / p.cell);
  const float* f3[3] = {gx, gy, gz};
  float* fb3[3] = {gbx, gby, gbz};
  const int lane = threadIdx.x & 31;
  for (int j = j0; j < j1; ++j) {
    float cwb = 0.f, cwrb = 0.f, chib = 0.f;
    NodeCols c{};
    int pa[3] = {0, 1, 2}, sg[3] = {1, 1, 1};
    float t[2][4][2] = {};  // cotangent per sky field (x, y), box (x, y) corner and box z plane
    if (active) {
      node_cols_tiled(p, j, bx, fbx, by, fby, tx, ty, c, pa, sg);
      const float cw = p.cw[j], cwr = p.cwr[j];
      const float ss = static_cast<float>(sg[0] * sg[1]);
      const NodeField o[2] = {node_field(f3[pa[0]], c), node_field(f3[pa[1]], c)};
      // per sky field: value weight al and derivative weights be[box axis]
      float al[2] = {cw * sg[0] * Kb[0], cw * sg[1] * Kb[1]};
      float be[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
      be[0][pa[0]] += cwr * Jb[0][0];
      be[0][pa[1]] += cwr * ss * Jb[0][1];
      be[1][pa[0]] += cwr * ss * Jb[1][0];
      be[1][pa[1]] += cwr * Jb[1][1];
      const float w0[3] = {1.f - c.fx, 1.f - c.fy, 1.f - c.fz}, w1[3] = {c.fx, c.fy, c.fz};
      float F[3] = {0.f, 0.f, 0.f};  // dL / d(box fraction)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int z = 0; z < 2; ++z) {
            const int ax = k >> 1, ay = k & 1;
            const float wx = ax ? w1[0] : w0[0], wy = ay ? w1[1] : w0[1], wz = z ? w1[2] : w0[2];
            const float sx = ax ? 1.f : -1.f, sy = ay ? 1.f : -1.f, sz = z ? 1.f : -1.f;
            t[a][k][z] = al[a] * wx * wy * wz + be[a][0] * sx * wy * wz + be[a][1] * wx * sy * wz + be[a][2] * wx * wy * sz;
          }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          F[q] += al[a] * nf_d(o[a], q);
#pragma unroll
          for (int r = 0; r < 3; ++r) F[q] += be[a][r] * nf_s(o[a], q, r);
        }
      }
      cwb = Kb[0] * sg[0] * o[0].v + Kb[1] * sg[1] * o[1].v;
      cwrb = Jb[0][0] * nf_d(o[0], pa[0]) + Jb[0][1] * ss * nf_d(o[0], pa[1]) + Jb[1][0] * ss * nf_d(o[1], pa[0]) +
             Jb[1][1] * nf_d(o[1], pa[1]);
      const float r_over_cell = static_cast<float>(ref_r / p.cell) + p.dr[j];
      thb[0] += F[pa[0]] * sg[0] * r_over_cell;
      thb[1] += F[pa[1]] * sg[1] * r_over_cell;
      chib = (F[pa[0]] * sg[0] * tx + F[pa[1]] * sg[1] * ty + F[pa[2]] * sg[2]) * inv_cell;
    }
    // the warp-segmented reduction of the field cotangents (as half_backward); a segment needs the same cell and
    // the same replica axes
    const long long key = active ? static_cast<long long>(c.r[0] + c.iz) * 8 + pa[0] * 3 + pa[1] : -1ll - lane;
    const long long prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned above = lane == 31 ? 0u : heads & (0xffffffffu << (lane + 1));
    const int seg_end = above ? __ffs(above) - 2 : 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1)
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int z = 0; z < 2; ++z) {
            const float u = __shfl_down_sync(0xffffffffu, t[a][k][z], d);
            if (lane + d <= seg_end) t[a][k][z] += u;
          }
    if (head && active) {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        float* fbp = fb3[pa[a]];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (t[a][k][0] != 0.f) atomicAdd(fbp + c.r[k] + c.iz, t[a][k][0]);
          if (t[a][k][1] != 0.f) atomicAdd(fbp + c.r[k] + c.jz, t[a][k][1]);
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      cwb += __shfl_down_sync(0xffffffffu, cwb, o);
      cwrb += __shfl_down_sync(0xffffffffu, cwrb, o);
      chib += __shfl_down_sync(0xffffffffu, chib, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(sh_nodes + j, cwb);
      atomicAdd(sh_nodes + n_nodes + j, cwrb);
      atomicAdd(sh_nodes + 2 * n_nodes + j, chib);
    }
  }
}

template <bool TILED>
__global__ void __launch_bounds__(128) ray_step_adjoint_kernel(
    const double2* __restrict__ theta, const float2* __restrict__ eta, const float4* __restrict__ Amat,
    const float4* __restrict__ Bmat, int64_t nr, const float* __restrict__ gx, const float* __restrict__ gy,
    const __grid_constant__ RayStepParams p, double2* __restrict__ theta_bar, float2* __restrict__ eta_bar,
    float4* __restrict__ A_bar, float4* __restrict__ B_bar, float* __restrict__ gbx, float* __restrict__ gby,
    double* __restrict__ node_bar, double* __restrict__ drift_bar, const float* __restrict__ gz,
    float* __restrict__ gbz) {
  extern __shared__ float sh[];  // [3][n_nodes]
  const int n_nodes = p.n1 + p.n2;
  for (int i = threadIdx.x; i < 3 * n_nodes; i += blockDim.x) sh[i] = 0.f;
  __syncthreads();
  int64_t r;
  if (p.tile_w > 0) {
    // 16 x 8 pixel tiles, as in the forward kernel (neighbouring rays share mesh cells and cache lines)
    const unsigned tiles_x = static_cast<unsigned>(p.tile_w) >> 4;
    const unsigned tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    r = (ty * 8 + (threadIdx.x >> 4)) * static_cast<int64_t>(p.tile_w) + tx * 16 + (threadIdx.x & 15);
  } else {
    r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  }
  const bool active = r < nr;
  double db = 0.0;
  double2 th0 = active ? theta[r] : make_double2(0.0, 0.0);
  const float2 et0 = active ? eta[r] : make_float2(0.f, 0.f);
  const float4 A0v = active ? Amat[r] : make_float4(1.f, 0.f, 0.f, 1.f);
  const float4 B0v = active ? Bmat[r] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float A0[2][2] = {{A0v.x, A0v.y}, {A0v.z, A0v.w}};
  const float B0[2][2] = {{B0v.x, B0v.y}, {B0v.z, B0v.w}};
  // ---- forward recompute
  float K1[2], J1[2][2], K2[2], J2[2][2];
  if (active) {
    if (TILED) half_forward_tiled(p, 0, p.n1, th0.x, th0.y, p.ref_r[0], gx, gy, gz, K1, J1);
    else half_forward(p, 0, p.n1, th0.x, th0.y, p.ref_r[0], gx, gy, K1, J1);
  }
  float eta1[2] = {et0.x + (active ? K1[0] : 0.f), et0.y + (active ? K1[1] : 0.f)};
  float B1[2][2], A1[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) B1[a][b] = B0[a][b] + (active ? J1[a][0] * A0[0][b] + J1[a][1] * A0[1][b] : 0.f);
  const double d = p.drift_d;
  const double th1x = th0.x + d * eta1[0], th1y = th0.y + d * eta1[1];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) A1[a][b] = A0[a][b] + p.drift * B1[a][b];
  if (active) {
    if (TILED) half_forward_tiled(p, p.n1, p.n1 + p.n2, th1x, th1y, p.ref_r[1], gx, gy, gz, K2, J2);
    else half_forward(p, p.n1, p.n1 + p.n2, th1x, th1y, p.ref_r[1], gx, gy, K2, J2);
  }
  // ---- backward
  const double2 thbv = active ? theta_bar[r] : make_double2(0.0, 0.0);
  const float2 etbv = active ? eta_bar[r] : make_float2(0.f, 0.f);
  const float4 Abv = active ? A_bar[r] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 Bbv = active ? B_bar[r] : make_float4(0.f, 0.f, 0.f, 0.f);
  float Ab[2][2] = {{Abv.x, Abv.y}, {Abv.z, Abv.w}};
  float Bb[2][2] = {{Bbv.x, Bbv.y}, {Bbv.z, Bbv.w}};
  float etb[2] = {etbv.x, etbv.y};
  float thb1[2] = {static_cast<float>(thbv.x), static_cast<float>(thbv.y)};
  // B2 = B1 + J2 A1: J2_bar = B_bar A1^T, A1_bar += J2^T B_bar
  float Jb[2][2], Kb[2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) Jb[a][b] = Bb[a][0] * A1[b][0] + Bb[a][1] * A1[b][1];
  if (active)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) Ab[a][b] += J2[0][a] * Bb[0][b] + J2[1][a] * Bb[1][b];
  Kb[0] = etb[0];
  Kb[1] = etb[1];
  // second half kick at theta1: half_backward adds dK/dtheta^T K_bar (= J2^T K_bar) and the second-derivative
  // terms of J2 to theta1_bar
  if (TILED)
    half_backward_tiled(p, p.n1, p.n1 + p.n2, th1x, th1y, p.ref_r[1], gx, gy, gz, Kb, Jb, gbx, gby, gbz, thb1, sh,
                        n_nodes, active);
  else
    half_backward(p, p.n1, p.n1 + p.n2, th1x, th1y, p.ref_r[1], gx, gy, Kb, Jb, gbx, gby, thb1, sh, n_nodes, active);
  // A1 = A0 + d B1
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      Bb[a][b] += p.drift * Ab[a][b];
      db += static_cast<double>(Ab[a][b]) * B1[a][b];
    }
  // theta1 = theta0 + d eta1
  etb[0] += static_cast<float>(d) * thb1[0];
  etb[1] += static_cast<float>(d) * thb1[1];
  db += static_cast<double>(thb1[0]) * eta1[0] + static_cast<double>(thb1[1]) * eta1[1];
  float thb0[2] = {thb1[0], thb1[1]};
  // B1 = B0 + J1 A0
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) Jb[a][b] = Bb[a][0] * A0[b][0] + Bb[a][1] * A0[b][1];
  if (active)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) Ab[a][b] += J1[0][a] * Bb[0][b] + J1[1][a] * Bb[1][b];
  Kb[0] = etb[0];
  Kb[1] = etb[1];
  if (TILED)
    half_backward_tiled(p, 0, p.n1, th0.x, th0.y, p.ref_r[0], gx, gy, gz, Kb, Jb, gbx, gby, gbz, thb0, sh, n_nodes,
                        active);
  else
    half_backward(p, 0, p.n1, th0.x, th0.y, p.ref_r[0], gx, gy, Kb, Jb, gbx, gby, thb0, sh, n_nodes, active);
  if (active) {
    theta_bar[r] = make_double2(thb0[0], thb0[1]);
    eta_bar[r] = make_float2(etb[0], etb[1]);
    A_bar[r] = make_float4(Ab[0][0], Ab[0][1], Ab[1][0], Ab[1][1]);
    B_bar[r] = make_float4(Bb[0][0], Bb[0][1], Bb[1][0], Bb[1][1]);
  }
  block_add_double(db, drift_bar);
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * n_nodes; i += blockDim.x)
    if (sh[i] != 0.f) atomicAdd(node_bar + (i / n_nodes) * kMaxRayNodes + i % n_nodes, static_cast<double>(sh[i]));
}

hrt_status launch_ray_step_adjoint(const hrt_rays& rays, const float* gx, const float* gy, const RayStepParams& p,
                                   const hrt_rays& bar, float* gbx, float* gby, double* node_bar, double* drift_bar,
                                   cudaStream_t s, const float* gz, float* gbz) {
  if (rays.n_rays == 0) return HRT_OK;
  if (p.tiled && (!gz || !gbz)) return fail(HRT_ERR_INVALID_ARG, "a tiled ray step needs the third field and its cotangent");
  const size_t smem = 3 * static_cast<size_t>(p.n1 + p.n2) * sizeof(float);
  auto* kernel = p.tiled ? ray_step_adjoint_kernel<true> : ray_step_adjoint_kernel<false>;
  if (smem > 48 * 1024)
    HRT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  kernel<<<blocks_for(rays.n_rays, 128), 128, smem, s>>>(
      reinterpret_cast<const double2*>(rays.theta), reinterpret_cast<const float2*>(rays.eta),
      reinterpret_cast<const float4*>(rays.A), reinterpret_cast<const float4*>(rays.B), rays.n_rays, gx, gy, p,
      reinterpret_cast<double2*>(bar.theta), reinterpret_cast<float2*>(bar.eta), reinterpret_cast<float4*>(bar.A),
      reinterpret_cast<float4*>(bar.B), gbx, gby, node_bar, drift_bar, gz, gbz);
  HRT_LAUNCHED("ray_step_adjoint_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// kappa power-spectrum adjoint weights: spec *= W(k) = 2 c lambda_b / count_b for the bin b of the mode
// (lambda = dL/dP per bin, c = dtheta^4 / Theta^2); modes outside the bins get 0.  The caller then inverts.
// ---------------------------------------------------------------------------------------------------------
__global__ void power_adjoint_weight_kernel(float2* __restrict__ spec, int m, double theta_field, int nbins,
                                            double ln_lmin, double inv_ln_ratio, const double* __restrict__ wbin) {
  const int mzc = m / 2 + 1;
  const int64_t total = static_cast<int64_t>(m) * mzc;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int ix = static_cast<int>(e / mzc);
    const int iz = static_cast<int>(e - static_cast<int64_t>(ix) * mzc);
    const int nx = ix < m / 2 ? ix : ix - m;
    const double n2 = static_cast<double>(nx) * nx + static_cast<double>(iz) * iz;
    float w = 0.f;
    if (n2 > 0.0) {
      const double ell = 2.0 * M_PI * sqrt(n2) / theta_field;
      const double t = nbins * (log(ell) - ln_lmin) * inv_ln_ratio + 1e-9;
      if (t >= 0.0 && t < nbins) w = static_cast<float>(wbin[static_cast<int>(floor(t))]);
    }
    float2 v = spec[e];
    spec[e] = make_float2(w * v.x, w * v.y);
  }
}

hrt_status launch_power_adjoint_weight(void* spec, int64_t m, double dtheta, int nbins, double ell_min, double ell_max,
                                       const double* wbin_dev, cudaStream_t s) {
  const int64_t total = m * (m / 2 + 1);
  unsigned blocks = blocks_for(total, 256);
  if (blocks > 8 * 152) blocks = 8 * 152;
  power_adjoint_weight_kernel<<<blocks, 256, 0, s>>>(static_cast<float2*>(spec), static_cast<int>(m), m * dtheta, nbins,
                                                      std::log(ell_min), 1.0 / std::log(ell_max / ell_min), wbin_dev);
  HRT_LAUNCHED("power_adjoint_weight_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// Zel'dovich IC adjoint: out = sum_j -(i d_j T(n^2)) in_j  (T the FP64 host table incl. D1 and 1/n^3), and the
// table cotangent T_bar(n^2) += sum_j w_kz Re(conj(in_j) i d_j w_hat) for the omega_m chain.
// ---------------------------------------------------------------------------------------------------------
__global__ void ic_adjoint_kernel(const float2* __restrict__ in, const float2* __restrict__ w_hat, int n, int nzc,
                                  float kf, const float* __restrict__ table, int64_t elems, float2* __restrict__ out,
                                  double* __restrict__ table_bar) {
  const int iz = blockIdx.y * blockDim.x + threadIdx.x;
  const unsigned row = blockIdx.x * blockDim.y + threadIdx.y;
  if (iz >= nzc || row >= static_cast<unsigned>(n) * static_cast<unsigned>(n)) return;
  const int ix = static_cast<int>(row / static_cast<unsigned>(n));
  const int iy = static_cast<int>(row - static_cast<unsigned>(ix) * n);
  const int half = n >> 1;
  const int nx = ix < half ? ix : ix - n, ny = iy < half ? iy : iy - n;
  const int64_t e = static_cast<int64_t>(row) * nzc + iz;
  const int n2 = nx * nx + ny * ny + iz * iz;
  const float t = __ldg(table + n2);
  const float d[3] = {(nx == -half) ? 0.f : kf * nx, (ny == -half) ? 0.f : kf * ny, (iz == half) ? 0.f : kf * iz};
  const float2 wv = w_hat[e];
  float2 acc = make_float2(0.f, 0.f);
  double tb = 0.0;
  const double wkz = (iz == 0 || iz == half) ? 1.0 : 2.0;
  for (int j = 0; j < 3; ++j) {
    const float2 v = in[e + j * elems];
    const float cd = -t * d[j];  // -(i t d) v
    acc.x += -cd * v.y;
    acc.y += cd * v.x;
    // Re(conj(v) * i d w) = d (v.x * (-w.y) + v.y * w.x)
    tb += wkz * d[j] * (static_cast<double>(v.y) * wv.x - static_cast<double>(v.x) * wv.y);
  }
  out[e] = acc;
  if (table_bar != nullptr && tb != 0.0) atomicAdd(table_bar + n2, tb);
}

hrt_status launch_ic_adjoint(const void* in, const void* w_hat, int64_t n, double box, const float* table, void* out,
                             double* table_bar, cudaStream_t s) {
  const int64_t nzc = n / 2 + 1;
  dim3 block(64, 4);
  dim3 grid(static_cast<unsigned>((n * n + 3) / 4), static_cast<unsigned>((nzc + 63) / 64));
  ic_adjoint_kernel<<<grid, block, 0, s>>>(static_cast<const float2*>(in), static_cast<const float2*>(w_hat),
                                           static_cast<int>(n), static_cast<int>(nzc),
                                           static_cast<float>(2.0 * M_PI / box), table, n * n * nzc,
                                           static_cast<float2*>(out), table_bar);
  HRT_LAUNCHED("ic_adjoint_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// 2LPT adjoint pieces.  The forward (hrt_ic_2lpt) is, at unit growth, with w_hat = R2C(noise) and t = T / D1:
//   Psi1_j = C2R(i t d_j w_hat),  H_ab = C2R(t d_a d_b w_hat),  S = sum_{a<b} (H_aa H_bb - H_ab^2),
//   Psi2_j = C2R(-i d_j R2C(S) / (k^2 n^3)).
// Each C2R(M R2C(.)) with a Hermitian multiplier M has the transpose C2R(conj(M) R2C(.)).
// ---------------------------------------------------------------------------------------------------------

// out = sum_j (i d_j / (k^2 n^3)) in_j (the transpose of the Psi2 step, into the spectrum of S_bar).
__global__ void lpt2_kspace_adjoint_kernel(const float2* __restrict__ in, int n, int nzc, float kf, float inv_n3,
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
  const float d[3] = {(nx == -half) ? 0.f : kf * nx, (ny == -half) ? 0.f : kf * ny, (nz == half) ? 0.f : kf * nz};
  float2 acc = make_float2(0.f, 0.f);
  for (int j = 0; j < 3; ++j) {
    const float2 v = in[e + j * elems];
    const float cd = c * d[j];  // i cd v
    acc.x -= cd * v.y;
    acc.y += cd * v.x;
  }
  out[e] = acc;
}

hrt_status launch_lpt2_kspace_adjoint(const void* in, int64_t n, double box, void* out, cudaStream_t s) {
  const int64_t nzc = n / 2 + 1;
  dim3 block(64, 4);
  dim3 grid(static_cast<unsigned>((n * n + 3) / 4), static_cast<unsigned>((nzc + 63) / 64));
  lpt2_kspace_adjoint_kernel<<<grid, block, 0, s>>>(static_cast<const float2*>(in), static_cast<int>(n),
                                                    static_cast<int>(nzc), static_cast<float>(2.0 * M_PI / box),
                                                    static_cast<float>(1.0 / (static_cast<double>(n) * n * n)),
                                                    n * n * nzc, static_cast<float2*>(out));
  HRT_LAUNCHED("lpt2_kspace_adjoint_kernel");
  return HRT_OK;
}

// In place: h holds the six Hessian fields (xx, yy, zz, xy, xz, yz) and receives their cotangents for the
// source cotangent sb: d S / d H_aa = sum of the other two diagonal fields, d S / d H_ab = -2 H_ab.
__global__ void lpt2_source_adjoint_kernel(float* __restrict__ h, const float* __restrict__ sb, int64_t m) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= m) return;
  const float xx = h[i], yy = h[i + m], zz = h[i + 2 * m], xy = h[i + 3 * m], xz = h[i + 4 * m], yz = h[i + 5 * m];
  const float b = sb[i];
  h[i] = b * (yy + zz);
  h[i + m] = b * (xx + zz);
  h[i + 2 * m] = b * (xx + yy);
  h[i + 3 * m] = -2.f * b * xy;
  h[i + 4 * m] = -2.f * b * xz;
  h[i + 5 * m] = -2.f * b * yz;
}

hrt_status launch_lpt2_source_adjoint(float* h, const float* sb, int64_t m, cudaStream_t s) {
  lpt2_source_adjoint_kernel<<<blocks_for(m, 256), 256, 0, s>>>(h, sb, m);
  HRT_LAUNCHED("lpt2_source_adjoint_kernel");
  return HRT_OK;
}

// out += sum_j t f_j in_j for the Hessian set (0: xx, yy, zz; 1: xy, xz, yz) with f_j the product of the two
// derivative factors, and table_bar[|n|^2] += sum_j f_j Re(conj(in_j) w_hat) (half-spectrum weight 2 off the
// kz = 0 and Nyquist planes).
__global__ void ic_hessian_adjoint_kernel(const float2* __restrict__ in, const float2* __restrict__ w_hat, int n,
                                          int nzc, float kf, const float* __restrict__ table, int set, int64_t elems,
                                          float2* __restrict__ out, double* __restrict__ table_bar) {
  const int iz = blockIdx.y * blockDim.x + threadIdx.x;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.y + threadIdx.y;
  if (iz >= nzc || row >= static_cast<int64_t>(n) * n) return;
  const int ix = static_cast<int>(row / n);
  const int iy = static_cast<int>(row - static_cast<int64_t>(ix) * n);
  const int half = n >> 1;
  const int nx = ix < half ? ix : ix - n, ny = iy < half ? iy : iy - n, nz = iz;
  const int64_t e = row * nzc + iz;
  const int n2 = nx * nx + ny * ny + nz * nz;
  const float t = __ldg(table + n2);
  const float dx = (nx == -half) ? 0.f : kf * nx;
  const float dy = (ny == -half) ? 0.f : kf * ny;
  const float dz = (nz == half) ? 0.f : kf * nz;
  const float f[3] = {set == 0 ? dx * dx : dx * dy, set == 0 ? dy * dy : dx * dz, set == 0 ? dz * dz : dy * dz};
  const float2 wv = w_hat[e];
  float2 acc = out[e];
  double tb = 0.0;
  const double wkz = (iz == 0 || iz == half) ? 1.0 : 2.0;
  for (int j = 0; j < 3; ++j) {
    const float2 v = in[e + j * elems];
    acc.x += t * f[j] * v.x;
    acc.y += t * f[j] * v.y;
    tb += wkz * f[j] * (static_cast<double>(v.x) * wv.x + static_cast<double>(v.y) * wv.y);
  }
  out[e] = acc;
  if (table_bar != nullptr && tb != 0.0) atomicAdd(table_bar + n2, tb);
}

hrt_status launch_ic_hessian_adjoint(const void* in, const void* w_hat, int64_t n, double box, const float* table,
                                     int set, void* out, double* table_bar, cudaStream_t s) {
  const int64_t nzc = n / 2 + 1;
  dim3 block(64, 4);
  dim3 grid(static_cast<unsigned>((n * n + 3) / 4), static_cast<unsigned>((nzc + 63) / 64));
  ic_hessian_adjoint_kernel<<<grid, block, 0, s>>>(static_cast<const float2*>(in), static_cast<const float2*>(w_hat),
                                                   static_cast<int>(n), static_cast<int>(nzc),
                                                   static_cast<float>(2.0 * M_PI / box), table, set, n * n * nzc,
                                                   static_cast<float2*>(out), table_bar);
  HRT_LAUNCHED("ic_hessian_adjoint_kernel");
  return HRT_OK;
}

// ---------------------------------------------------------------------------------------------------------
// FP64 dot product of two float32 arrays (coefficient cotangents such as dL/dpref = <g_bar, g> / pref).
// ---------------------------------------------------------------------------------------------------------
__global__ void dot_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t m, double* __restrict__ out) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < m;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    s += static_cast<double>(a[i]) * b[i];
  block_add_double(s, out);
}

hrt_status launch_dot(const float* a, const float* b, int64_t m, double* out, cudaStream_t s) {
  unsigned blocks = blocks_for(m, 256);
  if (blocks > 4 * 152) blocks = 4 * 152;
  dot_kernel<<<blocks, 256, 0, s>>>(a, b, m, out);
  HRT_LAUNCHED("dot_kernel");
  return HRT_OK;
}

__global__ void axpy_kernel(const float* __restrict__ x, float* __restrict__ y, float alpha, int64_t m) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < m) y[i] += alpha * x[i];
}

hrt_status launch_axpy(const float* x, float* y, double alpha, int64_t m, cudaStream_t s) {
  if (m == 0) return HRT_OK;
  axpy_kernel<<<blocks_for(m, 256), 256, 0, s>>>(x, y, static_cast<float>(alpha), m);
  HRT_LAUNCHED("axpy_kernel");
  return HRT_OK;
}

}  // namespace hrt
