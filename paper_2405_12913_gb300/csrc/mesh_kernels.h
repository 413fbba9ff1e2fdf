// Launch wrappers of the mesh kernels (mesh_kernels.cu), the particle sort (sort_kernels.cu) and the ray kernels
// (ray_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.h"

namespace hrt {

// The same deposit with warp-aggregated atomics (n_side a power of two >= 32).
hrt_status launch_cic_scatter_warp(const float* disp, int64_t n_side, int64_t n, double box, float* rho,
                                   cudaStream_t s);
// order (or nullptr): particles stored in cell order, slot i holding lattice particle order[i]; rho_zeroed: rho
// is already zero (no memset before the deposit).
hrt_status launch_cic_scatter(const float* disp, int64_t n_side, int64_t n, double box, float* rho,
                              cudaStream_t s, const int32_t* order = nullptr, bool rho_zeroed = false);

// Bricks of the cell order: 8 x 8 x 32 cells, 64 sort keys (z-row segments) each.
constexpr int kBrickXY = 8;
constexpr int kBrickZ = 32;
constexpr int kBrickKeys = kBrickXY * kBrickXY;
// Mesh sides whose particles are sorted into bricks (a multiple of 32, at most 1024).
inline bool particle_bricks_ok(int64_t n) { return n >= kBrickZ && n <= 1024 && n % kBrickZ == 0; }

// Counting sort of the particles by z-row segments of 32 mesh cells, grouped into bricks if `bricks` and
// particle_bricks_ok(n), row-major otherwise: slot i of the output holds the particle that the key order puts
// there; disp, mom are [3][np] in slot order, order the slot -> lattice index map (nullptr: lattice order, read in
// the rows-of-sites order).  Writes disp_out, mom_out, order_out; counts (particle_sort_counts(n) ints) ends as
// the exclusive scan of the key counts (the first slot of every key); keys, ranks, src (np ints each) are
// scratch.
hrt_status launch_particle_sort(const float* disp, const float* mom, const int32_t* order, int64_t n_side, int64_t n,
                                double box, float* disp_out, float* mom_out, int32_t* order_out, int32_t* counts,
                                int32_t* keys, int32_t* ranks, int32_t* src, cudaStream_t s, bool bricks);
// Size (ints) of the counts scratch of launch_particle_sort for mesh side n.
int64_t particle_sort_counts(int64_t n);
// Slot order back to lattice order: out[:, order[i]] = in[:, i] for [3][np] arrays.
hrt_status launch_unsort(const float* in, const int32_t* order, int64_t np, float* out, cudaStream_t s);

void filter_tables(int64_t n, double box, const hrt_filter& f, std::vector<float>& wxy, std::vector<float>& wz);

// tab_* are device tables laid out [wxy (n) | wz (n/2+1)] for each filter set.
hrt_status launch_kspace(const void* rho_hat, int64_t n, double box, double pref, const float* tab_a,
                         const hrt_filter* fa, int n_a, void* out_a, const float* tab_b, const hrt_filter* fb,
                         int n_b, void* out_b, cudaStream_t s);

// With rho_out != nullptr the drifted particles are also CIC-deposited into rho_out (zeroed first).
struct KspaceCallbackInfo;
// Writes the caller info of the k-space load callback in stream order (kernel argument, no host wait).
hrt_status launch_set_callback_info(KspaceCallbackInfo* dst, const KspaceCallbackInfo& v, cudaStream_t s);

// rho_zeroed: rho_out is already zero (no memset before the deposit).
hrt_status launch_kick_drift(const float* grad, int64_t n, double box, int64_t n_side, float* disp, float* mom,
                             double kick, double drift, cudaStream_t s, float* rho_out = nullptr,
                             const int32_t* order = nullptr, bool rho_zeroed = false);
// The kick-drift-deposit on brick-sorted particles (particle_bricks_ok(n)): one block per brick, slots
// [key_start[64 b], key_start[64 b + 64]) (np after the last brick), with the brick's field tile and density tile
// in shared memory.  Any slot ranges give the same result; particles outside their block's tile take the
// global path.
// mode: kTilesTma (TMA boxes for tiles inside the mesh, row copies for the wrapping ones) or kTilesRows (row
// copies for all).  err (nullptr: a module-level word) receives kTileTimeout if a wait for a TMA box timed out.
constexpr int kTilesRows = 1;
constexpr int kTilesTma = 2;
constexpr int kTileTimeout = 2;
hrt_status launch_kick_drift_tiled(const float* grad, int64_t n, double box, int64_t n_side, float* disp, float* mom,
                                   double kick, double drift, float* rho_out, const int32_t* order,
                                   const int32_t* key_start, cudaStream_t s, int mode = kTilesTma,
                                   int* err = nullptr, bool rho_zeroed = false);

hrt_status launch_ic_kspace(const void* w_hat, int64_t n, double box, const float* table, void* out,
                            cudaStream_t s);

hrt_status launch_scale_copy(const float* in, float* out, double ratio, int64_t m, cudaStream_t s);

// Second-order Lagrangian ICs (2LPT): Hessian spectra of phi1 (set 0: xx, yy, zz; set 1: xy, xz, yz) from the
// unit-growth IC table, the real-space source, the spectra of Psi2 and the final combination.
hrt_status launch_ic_hessian(const void* w_hat, int64_t n, double box, const float* table, int set, void* out,
                             cudaStream_t s);
hrt_status launch_lpt2_source(const float* h, int64_t m, float* out, cudaStream_t s);
hrt_status launch_lpt2_kspace(const void* s_hat, int64_t n, double box, void* out, cudaStream_t s);
hrt_status launch_lpt_combine(const float* psi1, const float* psi2, int64_t m, double d1, double d2, double c1,
                              double c2, float* disp, float* mom, cudaStream_t s);

// ---- rays ----
constexpr int kMaxRayNodes = 1024;
constexpr int kMaxReplicas = 64;

struct RayStepParams {
  int n1, n2;            // nodes of the first and second half shell (after the force window)
  int n;                 // mesh cells per side
  int tile_w;            // > 0: rays form an image tile_w pixels wide, walked in 16 x 8 tiles
  int map_accumulate;    // readout: 0 writes the observables, 1 adds map_weight times them
  float map_weight;
  float drift;           // (chi_to - chi_from) / (c chi_mid^2), float32 copy for A
  double drift_d;        // the same in FP64 for theta
  double ref_r[2];       // reference radius of each half shell for the FP64 base position
  double obs_x, obs_y;   // observer transverse position
  double cell, box;
  float dr[kMaxRayNodes];   // (r_j - ref_r) / cell
  float cw[kMaxRayNodes];   // c_j
  float cwr[kMaxRayNodes];  // c_j r_j / cell
  int kz[kMaxRayNodes];     // lower node of the sample along the line-of-sight box axis (z without tiling)
  float fz[kMaxRayNodes];   // its fraction
  // light-cone tiling (tiled != 0): replica of each node, and per replica the box axis and sign of the sky
  // axes and the translation (cells) of the box axes that receive sky x and y
  int tiled;
  // precision ablation (0 in the method): 1 keeps the ray angle in FP32 (rounded after each drift) and forms the
  // interpolation position r theta in FP32 instead of the FP64 cell / fraction split
  int theta32;
  unsigned char rep[kMaxRayNodes];
  signed char rperm[kMaxReplicas][3];
  signed char rsign[kMaxReplicas][3];
  int rshift[kMaxReplicas][2];
};

// gz (the third gradient component) is read only when p.tiled.
hrt_status launch_ray_step(const hrt_rays& rays, const float* gx, const float* gy, const RayStepParams& p,
                           float* maps, cudaStream_t s, const float* gz = nullptr);
hrt_status launch_ray_drift_free(const hrt_rays& rays, double d, cudaStream_t s);
hrt_status launch_ray_readout(const hrt_rays& rays, float* maps, cudaStream_t s);
hrt_status launch_rays_init(const hrt_rays& rays, const double* theta0, cudaStream_t s);

// Power-spectrum binning of an m x (m/2+1) half spectrum into sums[3][nbins] (power, ell, count).
hrt_status launch_power_bin(const void* spec, int64_t m, double dtheta, int nbins, double ell_min, double ell_max,
                            double* sums, cudaStream_t s);

}  // namespace hrt
