/*
 * hrt.h -- C ABI of the GB300 (sm_103a) hot path of Hamiltonian ray tracing (HRT), after Zhou et al.,
 * "A Hamiltonian, post-Born, three-dimensional, on-the-fly ray tracing algorithm for gravitational lensing"
 * (arXiv 2405.12913).
 *
 * Units: lengths in Mpc/h, velocities in 100 km/s (H0 = 1), masses in Msun/h, angles in radians.  The speed
 * of light is c = 2997.92458 and G = 4.30091727e-13 in these units.
 *
 * Conventions shared by every call
 *   - Meshes are n^3 single-precision arrays indexed [ix][iy][iz] with iz fastest; node (ix, iy, iz) sits at
 *     (ix, iy, iz) * box / n and the mesh is periodic.  Half spectra are interleaved complex64 arrays
 *     [ix][iy][kz], kz = 0..n/2 (the layout of an out-of-place real-to-complex FFT).
 *   - Particles are on an n_side^3 Lagrangian lattice q = (i, j, k) * box / n_side with particle index
 *     (i * n_side + j) * n_side + k; positions are stored as float32 displacements from q, momenta as
 *     p = a^2 dx/dt, both structure-of-arrays [3][n_side^3].  n (mesh) must be a multiple of n_side.
 *   - Ray state, ray-major: theta [R][2] float64, eta [R][2] float32, A [R][4] and B [R][4] float32
 *     (row-major 2x2: A11, A12, A21, A22).
 *   - Pointer arguments are device pointers unless a name ends in _host.  They are borrowed for the call
 *     only; work is enqueued on the caller's CUDA stream (a cudaStream_t passed as void*, NULL = legacy
 *     default stream) and the caller keeps the buffers alive until that stream has reached the work.
 *     Calls documented as "synchronises" wait for the stream before returning.
 *   - Every call returns an hrt_status; nothing is thrown across the ABI.  After HRT_ERR_CUDA a context is
 *     poisoned: every later call on it returns HRT_ERR_STATE except hrt_destroy.
 */
#ifndef HRT_H
#define HRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hrt_status {
  HRT_OK = 0,
  HRT_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range; nothing was enqueued       */
  HRT_ERR_OOM = 2,         /* a device or host allocation failed; the context stays destroyable       */
  HRT_ERR_CUDA = 3,        /* a CUDA runtime or cuFFT call failed                                     */
  HRT_ERR_STATE = 4,       /* calls out of order (e.g. a step before particles exist), or poisoned    */
  HRT_ERR_NONFINITE = 5,   /* a NaN or infinity was found in an output that the call checks          */
  HRT_ERR_TIMEOUT = 6      /* a host wait for the stream exceeded its limit                           */
} hrt_status;

/* Human-readable name of a status code (static string). */
const char* hrt_status_string(hrt_status s);

/* Last error message of the calling thread (static thread-local buffer, empty if none). */
const char* hrt_last_error(void);

/* ------------------------------------------------------------------------------------------------------
 * FP64 host cosmology (flat LCDM without radiation), Sec. 2 (Poisson equation, r = chi) and Sec. 3.2
 * (growth time correction of Eq. "kick").  Host-only, no GPU needed.
 * ---------------------------------------------------------------------------------------------------- */

/* out[0] = E(a) = H/H0, out[1] = chi(a) (comoving distance of the light front at a from the observer at
 * a = 1), out[2] = D1(a) (linear growth, D1(1) = 1), out[3] = f(a) = dlnD1/dlna. */
hrt_status hrt_cosmo_eval(double omega_m, double a, double out_host[4]);

/* Signed particle time integrals: out[0] = K(a->b) = int_a^b da/(a E), out[1] = Dr(a->b) = int da/(a^3 E);
 * the leapfrog kick is p -= grad(phi) K and the drift x += p Dr (momentum p = a^2 dx/dt). */
hrt_status hrt_cosmo_time_integrals(double omega_m, double a, double b, double out_host[2]);

/* Scale factor of the light front at comoving distance chi (inverse of chi(a)). */
hrt_status hrt_cosmo_a_of_chi(double omega_m, double chi, double* a_host);

/* Amplitude A of P(k) = A k^n_s T_BBKS(k / (omega_m h))^2 with sigma(8 Mpc/h) = sigma8 at a = 1. */
hrt_status hrt_cosmo_power_amplitude(double omega_m, double h, double n_s, double sigma8, double* amp_host);

/* ------------------------------------------------------------------------------------------------------
 * Mesh kernels (stateless; the PM object below owns FFT plans and tables)
 * ---------------------------------------------------------------------------------------------------- */

/* CIC (cloud-in-cell) mass assignment, the density step of the PM force ("the most computationally
 * expensive operation", Sec. 5.1).  Overwrites rho[n^3] with rho/rho_mean = 1 + delta: each of the
 * n_side^3 particles carries n^3 / n_side^3 and gives weight (1-f) to node floor(u), f to floor(u)+1 per
 * axis, u = (q + disp) / cell, periodic.  disp is [3][n_side^3].  Accumulation order is not fixed (float32
 * atomics), so results are reproducible to rounding only.  n_side >= 1, n % n_side == 0, n >= 2. */
hrt_status hrt_cic_scatter(const float* disp, int64_t n_side, int64_t n, double box, float* rho,
                           void* stream);

/* hrt_cic_scatter with warp-aggregated atomics: lanes of a warp whose targets coincide combine their weights
 * (__match_any_sync) and one of them adds the sum.  The same result up to rounding; kept as the measured
 * alternative to the plain reductions (lattice-ordered particles rarely share a target within a warp).  Needs
 * n_side a power of two >= 32 (HRT_ERR_INVALID_ARG otherwise). */
hrt_status hrt_cic_scatter_warp_aggregated(const float* disp, int64_t n_side, int64_t n, double box, float* rho,
                                           void* stream);

/* Fused particle update of the leapfrog (nbody_reverse_step of Alg. 1): CIC-interpolate the three gradient
 * fields grad[3][n^3] (d_x phi, d_y phi, d_z phi) at q + disp, then p -= grad phi * kick and
 * disp += p * drift.  kick and drift are the signed FP64 time integrals (K, Dr above; drift = 0 for a
 * kick-only synchronisation), rounded to float32 for the arithmetic. */
hrt_status hrt_particle_kick_drift(const float* grad, int64_t n, double box, int64_t n_side, float* disp,
                                   float* mom, double kick, double drift, void* stream);

/* hrt_particle_kick_drift followed by the CIC mass assignment of the drifted particles into rho[n^3]
 * (overwritten with rho/rho_mean as in hrt_cic_scatter), in one pass over the particles: the density of the
 * next PM force comes out of the particle update without re-reading the positions. */
hrt_status hrt_particle_kick_drift_deposit(const float* grad, int64_t n, double box, int64_t n_side, float* disp,
                                           float* mom, double kick, double drift, float* rho, void* stream);

/* hrt_particle_kick_drift_deposit on particles stored in brick order (the context's sort, hrt_set_particle_sort),
 * with shared-memory field and density tiles: n a multiple of 32 up to 1024; slot i of disp, mom ([3][n_side^3])
 * holds lattice particle order[i] (device int32 [n_side^3]); key_start (device int32 [n^3 / 32]) gives the first
 * slot of every sort key, key = brick * 64 + 8 (ix mod 8) + (iy mod 8) for bricks of 8 x 8 x 32 cells numbered
 * ((iz / 32) (n / 8) + ix / 8) (n / 8) + iy / 8.  Brick b's block takes slots [key_start[64 b], key_start[64 b +
 * 64]) (to n_side^3 for the last brick; offsets are clamped into range).  The update of every particle is the
 * same bit for bit whatever the offsets: a particle outside its block's tile takes the per-particle path; only
 * the order of the density's float additions differs.  A slot outside every range is not updated. */
hrt_status hrt_particle_kick_drift_deposit_bricks(const float* grad, int64_t n, double box, int64_t n_side,
                                                  float* disp, float* mom, const int32_t* order,
                                                  const int32_t* key_start, double kick, double drift, float* rho,
                                                  void* stream);

/* k-space filter of the gradient fields (Sec. 5.2 kick operator taken on the 3D mesh):
 *   prod_i sinc(k_i cell/2)^-deconv_p  *  exp(-k^2 smooth^2 / 2)  *  g(|k|)
 * with g the optional learned correction table: g_table[nk] (device, float32) sampled uniformly on
 * |k| in [0, g_kmax], linearly interpolated, 1 beyond g_kmax; NULL means g = 1. */
typedef struct hrt_filter {
  double deconv_p;      /* power p of the per-axis sinc deconvolution (0 = none)                   */
  double smooth;        /* Gaussian smoothing length in Mpc/h (0 = none)                           */
  const float* g_table; /* learned multiplicative correction, or NULL                              */
  int32_t g_nk;         /* entries of g_table (>= 2 when given)                                    */
  double g_kmax;        /* |k| of the last entry, h/Mpc                                            */
} hrt_filter;

/* Fused k-space kernel of the Poisson solve (Sec. 2 Poisson equation, Sec. 5.2 deconvolution):
 * from rho_hat (half spectrum of rho, any k = 0 value) write n_out gradient spectra
 *   out_j = i k_j * (-pref / k^2) * F(k) * rho_hat / n^3,   j = 0..n_out-1 (x, y[, z])
 * with out = 0 at k = 0 and on the j-Nyquist plane, k_i = 2 pi n_i / box, n_i in [-n/2, n/2).  The 1/n^3
 * makes an unnormalised complex-to-real inverse FFT return d_j phi.  pref = (3/2) Omega_m / a for the
 * expanding universe or 4 pi G rho_mean for a static lens.  out holds n_out spectra back to back.
 * If second != NULL, n_second (0..3) more spectra with the filter *f2 are written to second (the ray
 * fields when they differ from the particle fields); the density spectrum is read once. */
hrt_status hrt_kspace_gradient(const void* rho_hat, int64_t n, double box, double pref, const hrt_filter* f,
                               int32_t n_out, void* out, const hrt_filter* f2, int32_t n_second,
                               void* second, void* stream);

/* Same computation and arguments as hrt_kspace_gradient, but allocating nothing on the device.  The paper
 * has no counterpart: this exists for callers that manage all device memory themselves (a host application
 * with its own memory pool that forbids allocations once running, or a time-stepping loop that must not
 * allocate mid-step).  The per-axis filter tables live in one fixed array in device global memory
 * (2 * (2048 + 1025) floats, about 24 KB), held by every GPU that loads the library until the process exits,
 * so the mesh side n may not exceed 2048 (larger sizes return HRT_ERR_INVALID_ARG).  The first call on each
 * device looks up that array's device address (cudaGetSymbolAddress) with the device current; make that first
 * call before any stream capture.  Each call overwrites the whole array with its own tables before its kernel
 * reads them, so nothing has to start at zero; but every call shares the array, so calls whose work overlaps
 * on the GPU (different streams, or several host threads) race and may read each other's tables: serialise
 * them, e.g. on one stream.  No cudaMalloc, cudaFree or allocating library routine is called.  The tables are
 * staged from a host buffer during the call, so a call made while its stream is being captured into a CUDA
 * graph returns HRT_ERR_STATE and enqueues nothing.  Invalid arguments (the checks of hrt_kspace_gradient)
 * return HRT_ERR_INVALID_ARG. */
hrt_status hrt_kspace_gradient_noalloc(const void* rho_hat, int64_t n, double box, double pref,
                                       const hrt_filter* f, int32_t n_out, void* out, const hrt_filter* f2,
                                       int32_t n_second, void* second, void* stream);

/* ------------------------------------------------------------------------------------------------------
 * PM solver object: cuFFT plans and buffers for one mesh size, rho -> grad phi (R2C, k-space, C2R).
 * ---------------------------------------------------------------------------------------------------- */
typedef struct hrt_pm hrt_pm;

/* Creates plans for an n^3 mesh on `stream`, with device buffers for rho_hat and the gradient spectra.
 * n_ray_fields (0 or 2) adds two separately filtered ray gradient fields. */
hrt_status hrt_pm_create(int64_t n, double box, int32_t n_ray_fields, void* stream, hrt_pm** out);
hrt_status hrt_pm_destroy(hrt_pm* pm); /* NULL is fine; synchronises the stream */

/* on = 1 builds (once) batched complex-to-real plans with the k-space step linked into cuFFT's load stage (an
 * LTO load callback, JIT-linked at plan creation; mesh side a power of two up to 1024), so the gradient
 * spectra are never written to memory, and uses them in hrt_pm_solve; on = 0 returns to the separate k-space
 * kernel (same results).  Off by default: on a GB300 the callback plans are slower than plain plans plus the
 * k-space kernel.  Returns HRT_ERR_CUDA if cuFFT refuses the callback. */
hrt_status hrt_pm_set_fused(hrt_pm* pm, int32_t on);

/* Split path of hrt_pm_solve (on by default for n = 256, 512, 1024): batched 2D (y, z) cuFFT plans over the
 * x-planes and one x-pass kernel between them that does the forward FFT along x, the k-space step of
 * hrt_kspace_gradient and the inverse FFTs along x, so that no 3D spectrum is written or read twice.  Same
 * results as the 3D path (FP32 rounding of a different FFT order).  on = 0 returns to 3D cuFFT plans and the
 * separate k-space kernel.  HRT_ERR_INVALID_ARG for other mesh sides. */
hrt_status hrt_pm_set_split(hrt_pm* pm, int32_t on);

/* grad[3][n^3] <- gradient of phi from rho[n^3] (rho is overwritten as FFT scratch);
 * ray_grad[2][n^3] (only if the object has ray fields; else pass NULL) with the ray filter. */
hrt_status hrt_pm_solve(hrt_pm* pm, float* rho, double pref, const hrt_filter* f, float* grad,
                        const hrt_filter* f_ray, float* ray_grad);

/* ------------------------------------------------------------------------------------------------------
 * Rays
 * ---------------------------------------------------------------------------------------------------- */

/* Device ray state (caller-owned), n_rays rays, layouts as in the header comment. */
typedef struct hrt_rays {
  double* theta;
  float* eta;
  float* A;
  float* B;
  int64_t n_rays;
} hrt_rays;

/* theta = theta0[n][2], eta = 0, A = I, B = 0 (initial conditions of Sec. 2 and Sec. 4). */
hrt_status hrt_rays_init(const hrt_rays* rays, const double* theta0, void* stream);

/* Geometry of a ray step: box, mesh, observer and the line-of-sight quadrature density. */
typedef struct hrt_ray_geom {
  int64_t n;                 /* mesh cells per side                                                  */
  double box;                /* box side, Mpc/h                                                      */
  double observer[3];        /* observer position; line of sight along +z                            */
  double samples_per_cell;   /* s: each half shell uses max(1, ceil(s |half shell| / cell)) nodes    */
  double window_lo;          /* only nodes with window_lo <= chi < window_hi kick (static lens box)   */
  double window_hi;
  int64_t image_width;       /* > 0: ray r is pixel (r % W, r / W) of an image W pixels wide; the kernel
                                then walks the rays in 16 x 8 pixel tiles (thread order only, same results) */
  /* Light-cone tiling (hrt_ray_step_tiled; 0 replicas: none).  Replica k is the slab observer_z + chi in
   * [k box, (k+1) box); with u = X mod box, sky axis a maps to box axis replica_perm[k][a] at
   * replica_sign[k][a] u_a + replica_shift[k][replica_perm[k][a]] cells (mod box), i.e. the snapshot is rotated
   * by multiples of 90 degrees and translated by whole cells (host arrays, read during the call, at most 64
   * replicas). */
  int32_t n_replicas;
  const int32_t* replica_perm;   /* [n_replicas][3], a permutation of 0, 1, 2 */
  const int32_t* replica_sign;   /* [n_replicas][3], +1 or -1 */
  const int32_t* replica_shift;  /* [n_replicas][3], cells in [0, n) */
} hrt_ray_geom;

/* One KDK step of every ray through the shell [chi_from, chi_to] with the A/B recursion, Alg. 1 order
 * (Eqs. "symp_1".."symp_3", "obsv_recurse1".."obsv_recurse3"):
 *   eta += K(theta) over [chi_from, chi_mid];  B += (dK/dtheta) A;
 *   theta += eta d;  A += d B,  d = (chi_to - chi_from) / (c chi_mid^2)       (Eq. "drift", midpoint r);
 *   eta += K(theta) over [chi_mid, chi_to];    B += (dK/dtheta) A.
 * K = sum_j c_j (d_x phi, d_y phi)(X_j) with X_j = observer + (chi_j theta, chi_j), midpoint nodes chi_j and
 * c_j = -(2/c) h chi_j g(chi_j) (Eq. "kick"), g = D1(a(chi)) a_ref / (D1(a_ref) a(chi)) when a_ref > 0 and
 * g = 1 when a_ref == 0 (static potential); dK/dtheta = sum_j c_j chi_j T_j, T the transverse derivative of
 * the trilinear interpolant.  grad_x, grad_y are the n^3 gradient fields.  If maps != NULL the readout of
 * Eqs. "obs_first_set"/"obs_second_set" is written after the step: maps[4][n_rays] = kappa, gamma1,
 * gamma2, omega.  At most 1024 nodes per step (else HRT_ERR_INVALID_ARG). */
hrt_status hrt_ray_step(const hrt_rays* rays, const float* grad_x, const float* grad_y,
                        const hrt_ray_geom* geom, double chi_from, double chi_to, double a_ref,
                        double omega_m, float* maps, void* stream);

/* hrt_ray_step through a light cone tiled by rotated and translated box replicas (geom->n_replicas >= 1; see
 * hrt_ray_geom and the tiling of Sec. 6.2): grad_x, grad_y, grad_z are the three gradient fields of the box, of
 * which each node reads the two that its replica turns into the sky x and y directions.
 * HRT_ERR_INVALID_ARG if a line-of-sight node falls outside the replicas or a replica is malformed.  Its
 * adjoint is hrt_ray_step_tiled_adjoint. */
hrt_status hrt_ray_step_tiled(const hrt_rays* rays, const float* grad_x, const float* grad_y, const float* grad_z,
                              const hrt_ray_geom* geom, double chi_from, double chi_to, double a_ref, double omega_m,
                              float* maps, void* stream);

/* Exact drift with no force over [chi_from, chi_to] (chi_from > 0): theta += eta (1/chi_from -
 * 1/chi_to)/c, A += B (1/chi_from - 1/chi_to)/c.  Used where the potential is known to vanish. */
hrt_status hrt_ray_drift_free(const hrt_rays* rays, double chi_from, double chi_to, void* stream);

/* Readout only: maps[4][n_rays] = kappa, gamma1, gamma2, omega from A (Eqs. "obs_first_set"); maps may be NULL
 * when there are no rays. */
hrt_status hrt_ray_readout(const hrt_rays* rays, float* maps, void* stream);

/* ------------------------------------------------------------------------------------------------------
 * Ray-mesh kick operator (Sec. 5.2 "kick on a 2D ray mesh", Sec. 5.3 "adaptive ray mesh", App. C): the
 * paper's own way of evaluating the kick of Eq. "kick", an alternative to the direct line-of-sight gather of
 * hrt_ray_step.  For a half shell [chi_a, chi_b) (either orientation):
 *   lambda_lim = max(2 cell / (|chi_a| + |chi_b|), mu)              (Eq. "reslim")
 *   x2d = iota lambda_lim, N = smallest power of two >= ceil(m_pix mu / x2d + p_min / iota)   (App. C);
 * the ray mesh holds N x N nodes at the angles ((i - N/2) x2d, (j - N/2) x2d).  Every 3D node of a plane
 * z = kz cell with min(chi_a, chi_b) <= chi = z - O_z < max(chi_a, chi_b), chi > 0 (and inside the geometry's
 * window), with its transverse periodic images, is projected to the angle (X_xy - O_xy) / chi and carries
 * -(2/c) chi g(chi) (d_x phi, d_y phi) times its line-of-sight extent (+cell, or -cell for a shell walked
 * towards the observer) and its solid angle over the ray-mesh cell's, cell^2 / (chi^2 x2d^2).  These values
 * are CIC-deposited; the mesh is then multiplied in 2D Fourier space by
 * sinc(k_x x2d / 2)^-4 sinc(k_y x2d / 2)^-4 exp(-(k_x^2 + k_y^2) lambda_lim^2 / 2) (the deconvolution of
 * both CIC steps and the Gaussian smoothing of Sec. 5.2), and the kick at a ray is the bilinear interpolation
 * of the mesh at its angle (zero outside the mesh), with dK/dtheta the derivative of that interpolant.
 * g(chi) is the growth correction of Eq. "kick" with a_ref (a_ref <= 0: g = 1).  The line of sight is the z
 * axis of the periodically replicated box, or, through the _tiled calls, of a light cone tiled by rotated and
 * translated replicas (hrt_ray_geom): the plane z = kz cell lies in replica floor(kz / n), and its node (i, j)
 * reads the box node that the replica's map gives for sky node (i, j, kz mod n), with the sky components
 * sign_a grad_{perm a} there.  samples_per_cell and image_width of the geometry are not used.  Computed in
 * float32: the 3D-to-mesh positions start from an FP64 base per 8 x 32 block of mesh nodes; the ray angles
 * stay FP64.
 * ------------------------------------------------------------------------------------------------------ */
typedef struct hrt_raymesh_config {
  double iota;      /* accuracy parameter, 0 < iota <= 1 (smaller: finer ray mesh)                      */
  double p_min;     /* minimum padding width in units of lambda_lim, >= 0                                */
  double mu;        /* pixel size of the ray image, rad, > 0                                             */
  int64_t m_pix;    /* pixels across the image, >= 1                                                     */
  int64_t n2d_max;  /* largest ray-mesh side accepted (0: 8192, at most 32768); a shell that needs a
                       larger mesh gives HRT_ERR_INVALID_ARG                                              */
} hrt_raymesh_config;

/* Workspace of the ray-mesh kick: cuFFT plans by mesh side and two device meshes (one per half shell),
 * grown on demand.  Not thread-safe; one stream at a time. */
typedef struct hrt_raymesh hrt_raymesh;

/* lambda_lim, x2d and N of the half shell [chi_a, chi_b) on a mesh of cell size cell (host only). */
hrt_status hrt_raymesh_geometry(const hrt_raymesh_config* cfg, double chi_a, double chi_b, double cell,
                                double* lambda_lim_host, double* x2d_host, int64_t* n2d_host);
hrt_status hrt_raymesh_create(const hrt_raymesh_config* cfg, hrt_raymesh** out);
hrt_status hrt_raymesh_destroy(hrt_raymesh* rm);  /* NULL is fine; synchronises the device */

/* The filtered ray mesh of one half shell into mesh (device, caller-owned, N x N x 2 float32 with
 * mesh[(i N + j) 2 + c] the component c at node (i, j); N from hrt_raymesh_geometry).  grad_x, grad_y: the
 * transverse gradient fields [n][n][n] (x, y, z; z fastest), device float32.  HRT_ERR_INVALID_ARG for a bad
 * geometry or configuration, more than 512 planes in the shell, or a ray-mesh cell wider than 64 mesh cells. */
hrt_status hrt_raymesh_kick(hrt_raymesh* rm, const float* grad_x, const float* grad_y, const hrt_ray_geom* geom,
                            double chi_a, double chi_b, double a_ref, double omega_m, float* mesh, void* stream);
/* hrt_raymesh_kick through a tiled light cone (geom->n_replicas >= 1): grad_z is the third gradient field.
 * HRT_ERR_INVALID_ARG also if a plane falls outside the replicas or a replica is malformed.  The untiled calls
 * refuse a geometry with replicas. */
hrt_status hrt_raymesh_kick_tiled(hrt_raymesh* rm, const float* grad_x, const float* grad_y, const float* grad_z,
                                  const hrt_ray_geom* geom, double chi_a, double chi_b, double a_ref, double omega_m,
                                  float* mesh, void* stream);

/* One KDK ray step over [chi_from, chi_to] in the order of Alg. 1 (as hrt_ray_step) whose half kicks over
 * [chi_from, chi_mid) and [chi_mid, chi_to) come from their ray meshes; the drift is that of hrt_ray_step.
 * maps (device float32 [4][n_rays], or NULL) receives kappa, gamma1, gamma2, omega.  Errors as
 * hrt_raymesh_kick. */
hrt_status hrt_raymesh_ray_step(hrt_raymesh* rm, const hrt_rays* rays, const float* grad_x, const float* grad_y,
                                const hrt_ray_geom* geom, double chi_from, double chi_to, double a_ref,
                                double omega_m, float* maps, void* stream);
hrt_status hrt_raymesh_ray_step_tiled(hrt_raymesh* rm, const hrt_rays* rays, const float* grad_x, const float* grad_y,
                                      const float* grad_z, const hrt_ray_geom* geom, double chi_from, double chi_to,
                                      double a_ref, double omega_m, float* maps, void* stream);

/* ------------------------------------------------------------------------------------------------------
 * Convergence power spectrum: P(ell) = <|FFT2(kappa) dtheta^2|^2>_bin / (m dtheta)^2 over nbins log bins
 * in [ell_min, ell_max) (bin b = floor(nbins ln(ell/ell_min)/ln(ell_max/ell_min) + 1e-9), the 1e-9 placing
 * exact edges in the upper bin), ell = 2 pi |n| / (m dtheta).  Outputs the mean ell, mean power and mode
 * count per bin to host arrays of nbins.  kappa is m x m float32 (m even, 2 <= m <= 16384,
 * 1 <= nbins <= 256).  Synchronises the stream: it first waits for the work already queued on the stream
 * within the host wait limit (hrt_set_host_wait_limit) and returns HRT_ERR_TIMEOUT, having enqueued nothing,
 * when that expires; then its own transform and binning run and are waited for.
 * ---------------------------------------------------------------------------------------------------- */
hrt_status hrt_kappa_power(const float* kappa, int64_t m, double dtheta, int32_t nbins, double ell_min,
                           double ell_max, double* ell_host, double* p_host, int64_t* count_host,
                           void* stream);

/* ------------------------------------------------------------------------------------------------------
 * Zel'dovich initial conditions (particle lattice, a_init): delta_k = w_k sqrt(P(k)/V_cell) from white
 * noise w[n_side^3] (float32), Psi_k = i k delta_k / k^2 (0 at k = 0 and on Nyquist planes),
 * disp = D1(a) Psi, mom = a^2 E(a) f(a) D1(a) Psi.  disp, mom are [3][n_side^3].
 * ---------------------------------------------------------------------------------------------------- */
typedef struct hrt_cosmology {
  double omega_m, h, n_s, sigma8;
} hrt_cosmology;

hrt_status hrt_ic_zeldovich(const float* noise, int64_t n_side, double box, const hrt_cosmology* cosmo,
                            double a_init, float* disp, float* mom, void* stream);

/* Second-order Lagrangian ICs (the paper's IC scheme, Sec. 6.2): from the same white noise and linear density
 * as hrt_ic_zeldovich, x = q + D1 Psi1 + D2 Psi2 and p = a^2 E (f1 D1 Psi1 + f2 D2 Psi2), where Psi1 is the
 * Zel'dovich displacement at unit growth, Psi2 = grad phi2 with lap phi2 = sum_{i<j} (phi1_ii phi1_jj -
 * phi1_ij^2) (spectral derivatives, zero on Nyquist planes), D2 = -(3/7) D1^2 Omega_m(a)^(-1/143) and
 * f2 = 2 Omega_m(a)^(6/11).  Same layouts as hrt_ic_zeldovich; allocates 6 n_side^3 floats of scratch for the
 * call. */
hrt_status hrt_ic_2lpt(const float* noise, int64_t n_side, double box, const hrt_cosmology* cosmo, double a_init,
                       float* disp, float* mom, void* stream);

/* ------------------------------------------------------------------------------------------------------
 * Adjoints (reverse mode).  Each call is the vector-Jacobian product of the forward call of the same name:
 * given cotangents of the outputs it returns (or accumulates, where stated) the cotangents of the inputs and
 * of the host coefficients, so that a caller can run the forward path backwards with checkpointing.  Paper:
 * the adjoint method is named as future work (Sec. 7); these are the transposes of the operations above.
 * Coefficient cotangents are FP64 device accumulators that the calls add to.
 * ---------------------------------------------------------------------------------------------------- */

/* disp_bar[3][n_side^3] += d(sum rho_bar * rho)/d disp for rho = hrt_cic_scatter(disp). */
hrt_status hrt_cic_scatter_adjoint(const float* rho_bar, const float* disp, int64_t n_side, int64_t n, double box,
                                   float* disp_bar, void* stream);

/* Transpose of hrt_particle_kick_drift (and of hrt_particle_kick_drift_deposit when rho_bar != NULL) taken at
 * the PRE-step state disp, mom: on entry disp_bar, mom_bar hold the cotangents of the updated state, on return
 * those of (disp, mom); grad_bar[3][n^3] accumulates the cotangent of the gradient fields; coef_bar[0] and
 * coef_bar[1] accumulate dL/dkick and dL/ddrift. */
hrt_status hrt_particle_kick_drift_adjoint(const float* grad, int64_t n, double box, int64_t n_side, const float* disp,
                                           const float* mom, double kick, double drift, const float* rho_bar,
                                           float* disp_bar, float* mom_bar, float* grad_bar, double* coef_bar,
                                           void* stream);

/* Transpose of hrt_pm_solve: rho_bar[n^3] <- d(<grad_bar, grad> + <ray_grad_bar, ray_grad>)/d rho (the same
 * FFT pipeline with the conjugate transfer function).  grad_bar (and ray_grad_bar) are used as FFT input and
 * destroyed.  ray_grad_bar may be NULL. */
hrt_status hrt_pm_solve_adjoint(hrt_pm* pm, float* grad_bar, double pref, const hrt_filter* f, float* ray_grad_bar,
                                const hrt_filter* f_ray, float* rho_bar);

/* Transpose of hrt_ray_step at the PRE-step ray state `rays` (not modified): on entry bar holds the
 * cotangents of the state after the step (its maps readout must already be folded into bar->A), on return
 * those of the state before it; gx_bar, gy_bar accumulate the field cotangents; node_bar[3][1024]
 * accumulates, per line-of-sight node j of the step's node table, dL/dc_j, dL/d(c_j r_j / cell) and dL/dchi_j;
 * drift_bar[0] accumulates dL/dd for the drift coefficient d. */
hrt_status hrt_ray_step_adjoint(const hrt_rays* rays, const float* grad_x, const float* grad_y, const hrt_ray_geom* geom,
                                double chi_from, double chi_to, double a_ref, double omega_m, const hrt_rays* bar,
                                float* gx_bar, float* gy_bar, double* node_bar, double* drift_bar, void* stream);

/* hrt_ray_step_adjoint through a tiled light cone (geom->n_replicas >= 1, as hrt_ray_step_tiled): grad_z is the
 * third gradient field and gz_bar its cotangent; each node's cotangents go to the two box fields its replica
 * turns into the sky x and y directions. */
hrt_status hrt_ray_step_tiled_adjoint(const hrt_rays* rays, const float* grad_x, const float* grad_y,
                                      const float* grad_z, const hrt_ray_geom* geom, double chi_from, double chi_to,
                                      double a_ref, double omega_m, const hrt_rays* bar, float* gx_bar, float* gy_bar,
                                      float* gz_bar, double* node_bar, double* drift_bar, void* stream);

/* FP64 node table of a ray step as the kernels use it (host): counts of the two half shells and, per kept
 * node, c_j, c_j r_j / cell and chi_j, plus the drift coefficient.  Arrays hold at least 1024 entries. */
hrt_status hrt_ray_step_coefficients(const hrt_ray_geom* geom, double chi_from, double chi_to, double a_ref,
                                     double omega_m, int32_t* n1_host, int32_t* n2_host, double* cw_host,
                                     double* cwr_host, double* chi_host, double* drift_host);

/* kappa_bar[m^2] <- dL/dkappa for L a function of the binned power (hrt_kappa_power) with dL/dP_b given per bin
 * (host array of nbins).  Synchronises the stream. */
hrt_status hrt_kappa_power_adjoint(const float* kappa, int64_t m, double dtheta, int32_t nbins, double ell_min,
                                   double ell_max, const double* dl_dp_host, float* kappa_bar, void* stream);

/* FP64 host table of the Zel'dovich IC transfer T(|n|^2) = D1 sqrt(P(k)/V_cell) / k^2 / n_side^3 (size
 * 3 (n_side/2)^2 + 1) and the momentum ratio a^2 E f. */
hrt_status hrt_ic_table(int64_t n_side, double box, const hrt_cosmology* cosmo, double a_init, double* table_host,
                        double* ratio_host);

/* Transpose of hrt_ic_zeldovich: noise_bar[n_side^3] <- dL/dnoise given disp_bar, mom_bar (cotangents of its
 * outputs) and disp (its displacement output); table_bar_host (size as hrt_ic_table, may be NULL) receives
 * dL/dT(|n|^2) and ratio_bar_host dL/d(a^2 E f).  Synchronises the stream. */
hrt_status hrt_ic_zeldovich_adjoint(const float* noise, int64_t n_side, double box, const hrt_cosmology* cosmo,
                                    double a_init, const float* disp_bar, const float* mom_bar, const float* disp,
                                    float* noise_bar, double* table_bar_host, double* ratio_bar_host, void* stream);

/* Transpose of hrt_ic_2lpt (R21: x = q + D1 Psi1 + D2 Psi2, p = c1 Psi1 + c2 Psi2 with c1 = a^2 E f1 D1 and
 * c2 = a^2 E f2 D2): noise_bar[n_side^3] <- dL/dnoise given disp_bar, mom_bar, the cotangents of its outputs.
 * table_bar_host (size as hrt_ic_table, or NULL) receives dL/dt for the unit-growth transfer t(|n|^2) =
 * T(|n|^2) / D1(a_init), and coef_bar_host (4 doubles, or NULL) dL/d(D1, D2, c1, c2) of the combine; both
 * depend on Omega_m (hrt_ic_table, hrt_ic_2lpt_coefficients).  Recomputes the forward fields (device memory:
 * about 60 B per particle plus 2 spectra).  Synchronises the stream. */
hrt_status hrt_ic_2lpt_adjoint(const float* noise, int64_t n_side, double box, const hrt_cosmology* cosmo,
                               double a_init, const float* disp_bar, const float* mom_bar, float* noise_bar,
                               double* table_bar_host, double* coef_bar_host, void* stream);
/* (D1, D2, c1, c2) of hrt_ic_2lpt's combine at a_init (host). */
hrt_status hrt_ic_2lpt_coefficients(const hrt_cosmology* cosmo, double a_init, double* out_host);

/* out_host = sum_i a[i] b[i] in FP64 over m float32 elements (synchronises). */
hrt_status hrt_dot(const float* a, const float* b, int64_t m, double* out_host, void* stream);

/* ------------------------------------------------------------------------------------------------------
 * Learned force correction (the analogue of the force-sharpening factor g of Sec. 6.2, k/k^2 -> (k/k^2) g,
 * here applied to the ray gradient fields of a coarse mesh): g = 1 + MLP(|k| cell, a, ln N_mesh), a 3-64-64-
 * 64-1 perceptron with SiLU activations.  Parameters: HRT_MLP_PARAMS floats in the order W1 [64][16] (input
 * columns 3..15 zero), b1 [64], W2 [64][64], b2 [64], W3 [64][64], b3 [64], W4 [64], b4 [1]; a BF16 copy of the
 * same layout (2 bytes per entry) feeds the tensor-core forward; biases are read from the FP32 master.
 * ---------------------------------------------------------------------------------------------------- */
#define HRT_MLP_PARAMS 9473

/* g[rows] = 1 + MLP(x[rows][3]): BF16 weights and activations, FP32 accumulation (tensor cores). */
hrt_status hrt_mlp_forward(const float* x, int32_t rows, const void* w_bf16, const float* w_f32, float* g,
                           void* stream);

/* grad[HRT_MLP_PARAMS] += d(sum_r g_bar[r] g[r]) / d parameters (FP32, with the BF16-rounded weights). */
hrt_status hrt_mlp_backward(const float* x, int32_t rows, const void* w_bf16, const float* w_f32,
                            const float* g_bar, float* grad, void* stream);

/* One Adam step (bias-corrected, step >= 1) on the FP32 master, then the BF16 copy. */
hrt_status hrt_mlp_adam(float* w_f32, void* w_bf16, const float* grad, float* m, float* v, double lr, double beta1,
                        double beta2, double eps, int32_t step, void* stream);

/* BF16 copy of the FP32 master (padding columns zeroed). */
hrt_status hrt_mlp_to_bf16(const float* w_f32, void* w_bf16, void* stream);

/* Cotangent of the learned table: table_bar[g_nk] += dL/dg_i for gradient fields made by hrt_kspace_gradient
 * with filter *f (whose g_table has g_nk entries over [0, g_kmax]) from rho_hat, given gbar_hat = the real-to-
 * complex FFT of the cotangents of those n_comp fields (x, y[, z]). */
hrt_status hrt_kspace_table_adjoint(const void* gbar_hat, int32_t n_comp, const void* rho_hat, int64_t n, double box,
                                    double pref, const hrt_filter* f, float* table_bar, void* stream);

/* Copies the density half spectrum of the last hrt_pm_solve into out (complex64 [n][n][n/2+1]); HRT_ERR_STATE
 * if that solve took the split path (see hrt_pm_set_split), which never forms the 3D spectrum. */
hrt_status hrt_pm_density_spectrum(hrt_pm* pm, void* out);

/* fields[n_out][n^3] <- gradient fields from a stored density half spectrum rho_hat (not modified): the k-space
 * kernel with filter *f, then n_out complex-to-real FFTs (the second half of hrt_pm_solve). */
hrt_status hrt_pm_gradient_from_spectrum(hrt_pm* pm, const void* rho_hat, double pref, const hrt_filter* f,
                                         int32_t n_out, float* fields);

/* out (complex64 half spectrum) <- real-to-complex FFT of real[n^3] with the object's plan. */
hrt_status hrt_pm_forward_fft(hrt_pm* pm, const float* real, void* out);

/* ------------------------------------------------------------------------------------------------------
 * Simulation context: particles + mesh + rays co-evolved as in Alg. 1 (one PM force per step).
 * ---------------------------------------------------------------------------------------------------- */
typedef struct hrt_config {
  int64_t n_mesh;           /* mesh cells per side                                                  */
  double box;               /* Mpc/h                                                                */
  int64_t n_side;           /* particles per side (n_mesh % n_side == 0)                            */
  hrt_cosmology cosmo;      /* ignored in static mode except omega_m                                */
  double deconv_p;          /* k-space filter of the gradient fields (see hrt_filter)               */
  double smooth_cells;      /* Gaussian smoothing length in mesh cells                              */
  double samples_per_cell;  /* ray line-of-sight samples per mesh cell                              */
  double observer[3];
  int32_t static_mode;      /* 1: flat static space, a = 1, Poisson prefactor static_pref           */
  double static_pref;       /* 4 pi G rho_mean for the static lens                                  */
  double window_lo, window_hi; /* chi range in which rays feel the force (static lens box)         */
  int32_t n_sources;        /* number of source planes (maps)                                       */
  int32_t ray_fields;       /* 0: rays use the particle fields; 2: separately filtered ray fields   */
  double ray_deconv_p, ray_smooth_cells; /* ray filter when ray_fields == 2                          */
} hrt_config;

typedef struct hrt_ctx hrt_ctx;

hrt_status hrt_create(const hrt_config* cfg, void* stream, hrt_ctx** out);
hrt_status hrt_destroy(hrt_ctx* ctx);  /* NULL is fine; synchronises the context's stream */

/* Device bytes a context of this configuration allocates (plans and buffers, with the buffers of the default
 * particle sort), for capacity planning; the ray mesh and a recorded run for hrt_adjoint come on top. */
hrt_status hrt_workspace_bytes(const hrt_config* cfg, int64_t n_rays, size_t* bytes_host);

/* Particles from Zel'dovich ICs (noise[n_side^3] device float32) at a_init, then the PM force at a_init. */
hrt_status hrt_init_particles_zeldovich(hrt_ctx* ctx, const float* noise, double a_init);

/* Particles from second-order Lagrangian (2LPT) ICs (noise as for hrt_init_particles_zeldovich; see
 * hrt_ic_2lpt), then the PM force at a_init. */
hrt_status hrt_init_particles_2lpt(hrt_ctx* ctx, const float* noise, double a_init);

/* Particles from caller state (copied) at scale factor a (momentum synchronised at a), then the force.  disp and
 * mom may be device or host memory (stream-ordered copies; pinned host memory keeps the call asynchronous). */
hrt_status hrt_init_particles(hrt_ctx* ctx, const float* disp, const float* mom, double a);

/* Rays at the observer (copied): theta0[n_rays][2], in device or host memory. */
hrt_status hrt_init_rays(hrt_ctx* ctx, const double* theta0, int64_t n_rays);

/* One co-evolution step from the current a to a_next (Alg. 1): if rays exist and a_next < a they are
 * traced through [chi(a), chi(a_next)] with the current force (and read out to map `source` if
 * source >= 0); then particles kick from their momentum time to (a + a_next)/2 and drift to a_next; then
 * the PM force is recomputed at a_next.  Forward steps (a_next > a) move particles only. */
hrt_status hrt_step(hrt_ctx* ctx, double a_next, int32_t source);

/* Learned correction of the ray force (the analogue of the trained force-sharpening factor g of Sec. 6.2):
 * params (device float32, HRT_MLP_PARAMS values in the hrt_mlp_forward layout) are copied into the
 * context, rounded to BF16, and from then on every force evaluation at scale factor a first evaluates
 * g(|k|) = hrt_mlp_forward((|k| cell, a, ln n_mesh)) on 512 points over |k| in [0, 1.0001 sqrt(3) pi / cell]
 * and multiplies the Green's function of the ray fields by it (linear interpolation in |k|).  The
 * particle force stays plain.  Needs ray_fields == 2 (HRT_ERR_STATE otherwise).  params == NULL
 * restores the plain ray kernel.  Takes effect at the next force evaluation (the next hrt_step). */
hrt_status hrt_set_ray_correction(hrt_ctx* ctx, const float* params);

/* Learned correction of the particle force (off by default; params = NULL returns to the plain kernel): the same
 * network form as hrt_set_ray_correction, g(|k| cell, a, ln N_mesh) = 1 + MLP, evaluated on the tensor cores at
 * each force evaluation's scale factor and multiplying the Green's function of the particle gradient fields
 * (k/k^2 -> (k/k^2) g, the force sharpening of Sec. 6.2).  The rays read the corrected fields unless the context
 * has ray fields of its own (ray_fields == 2).  params: device float32 [hrt_mlp_params] (copied).  The plain
 * kernel stays the fallback and the yardstick; a run with it is not recorded for hrt_adjoint. */
hrt_status hrt_set_particle_correction(hrt_ctx* ctx, const float* params);

/* Light-cone tiling of the context's rays (see hrt_ray_geom): n replicas with their [n][3] axis, sign and
 * shift tables (host, copied); n = 0 removes it.  Needs ray_fields == 0 (HRT_ERR_STATE otherwise). */
hrt_status hrt_set_replicas(hrt_ctx* ctx, int32_t n, const int32_t* perm, const int32_t* sign, const int32_t* shift);

/* Adjoints of the ray-mesh kick (the kick operator of Sec. 5.2 and App. C, differentiated as the adjoint
 * method that Sec. 7 names as future work).  The mesh geometry (lambda_lim, x2d, N, the plane set) is
 * held fixed: derivatives are taken with respect to the fields, the ray state and the plane weights
 * w_p = -(2/c) chi_p g(chi_p) (+-cell) cell^2 / (chi_p^2 x2d^2), not with respect to the discretisation.
 *
 * hrt_raymesh_kick_adjoint: transpose of hrt_raymesh_kick.  mesh_bar (device, N x N x 2 float32, layout of
 * hrt_raymesh_kick's output) is dL/dK of the filtered mesh; gx_bar, gy_bar (device [n^3] float32) accumulate
 * dL/d(grad_x), dL/d(grad_y); plane_bar_host (host, >= 512 doubles, or NULL) accumulates dL/dw_p for the
 * shell's planes in the order of hrt_raymesh_step_planes.  grad_x, grad_y are the forward's fields (for dL/dw_p).
 * Synchronises the stream. */
hrt_status hrt_raymesh_kick_adjoint(hrt_raymesh* rm, const float* grad_x, const float* grad_y, const float* mesh_bar,
                                    const hrt_ray_geom* geom, double chi_a, double chi_b, double a_ref, double omega_m,
                                    float* gx_bar, float* gy_bar, double* plane_bar_host, void* stream);

/* hrt_raymesh_ray_step_adjoint: transpose of hrt_raymesh_ray_step (without the readout).  rays hold the state
 * before the step (unchanged); bar holds on entry the cotangents of the state after it and on return those of
 * the state before it; gx_bar, gy_bar accumulate the field cotangents; plane_bar_host ([2][512] doubles, or NULL)
 * accumulates dL/dw_p of the two half shells' planes; drift_bar_host[0] (or NULL) accumulates dL/dd for the drift
 * coefficient d = (chi_to - chi_from) / (c chi_mid^2).  Synchronises the stream. */
hrt_status hrt_raymesh_ray_step_adjoint(hrt_raymesh* rm, const hrt_rays* rays, const float* grad_x, const float* grad_y,
                                        const hrt_ray_geom* geom, double chi_from, double chi_to, double a_ref,
                                        double omega_m, const hrt_rays* bar, float* gx_bar, float* gy_bar,
                                        double* plane_bar_host, double* drift_bar_host, void* stream);

/* The same two transposes through a light cone tiled by box replicas (Sec. 6.2; geom with n_replicas >= 1;
 * the forwards are hrt_raymesh_kick_tiled and hrt_raymesh_ray_step_tiled).  A node of a plane in replica k was
 * read from box field perm[k][a] with sign sign[k][a] for sky component a, at the replica's shifted box node, so
 * its cotangent goes there: gx_bar, gy_bar and gz_bar (device [n^3] float32, all three required) accumulate the
 * cotangents of the three box fields.  Other arguments and outputs as in the untiled calls. */
hrt_status hrt_raymesh_kick_tiled_adjoint(hrt_raymesh* rm, const float* grad_x, const float* grad_y,
                                          const float* grad_z, const float* mesh_bar, const hrt_ray_geom* geom,
                                          double chi_a, double chi_b, double a_ref, double omega_m, float* gx_bar,
                                          float* gy_bar, float* gz_bar, double* plane_bar_host, void* stream);
hrt_status hrt_raymesh_ray_step_tiled_adjoint(hrt_raymesh* rm, const hrt_rays* rays, const float* grad_x,
                                              const float* grad_y, const float* grad_z, const hrt_ray_geom* geom,
                                              double chi_from, double chi_to, double a_ref, double omega_m,
                                              const hrt_rays* bar, float* gx_bar, float* gy_bar, float* gz_bar,
                                              double* plane_bar_host, double* drift_bar_host, void* stream);

/* Host: the planes of a ray-mesh step, per half shell h the count n_h, chi_host[h * 512 + q] and the FP64
 * weight w_host[h * 512 + q], and the drift coefficient. */
hrt_status hrt_raymesh_step_planes(const hrt_raymesh_config* cfg, const hrt_ray_geom* geom, double chi_from,
                                   double chi_to, double a_ref, double omega_m, int32_t* n1_host, int32_t* n2_host,
                                   double* chi_host, double* w_host, double* drift_host);

/* Storage order of the context's particles: every `every` particle steps (hrt_step, hrt_step_accumulate) the
 * context re-sorts its particles by mesh cell (a counting sort by z-row segments of 32 cells in row-major order,
 * grouped into bricks of 8 x 8 x 32 cells while the tiled deposit of hrt_set_tiled_deposit is selected) before
 * the kick-drift-deposit, so that neighbouring threads gather from and deposit into neighbouring cells also
 * after clustering has spread lattice neighbours apart; 0 keeps lattice order (the default after hrt_create is
 * 8).  Particles given by hrt_init_particles or hrt_load_state are sorted before their first force (inside
 * the call); initial conditions, still in cell order, wait for the interval.  Only the storage order changes: every read-out
 * (hrt_read_particles, hrt_save_state) is in lattice order.  Extra device memory once sorting starts: 44 B per
 * particle and 4 B per 32 mesh cells. */
hrt_status hrt_set_particle_sort(hrt_ctx* ctx, int32_t every);

/* Kick-drift-deposit of the context (the particle update of Algorithm 1 with the CIC assignment of Sec. 2.2).
 * mode 0 (the default): one thread per particle, gathers and vector reductions in global memory, particles
 * sorted by z-row segments.  mode 2: the sort groups its keys into bricks of 8 x 8 x 32 cells (mesh sides that
 * are multiples of 32 up to 1024), and one block per brick copies the brick's field tile into shared memory (TMA
 * boxes for tiles inside the mesh, 16-byte row copies for tiles that wrap around it), gathers from it, deposits
 * into a shared density tile and adds that to the mesh; particles whose stencil left the tile take the
 * per-particle path.  mode 1: the same with row copies for every tile.  Momenta and displacements come out the
 * same bit for bit in every mode; the density differs only in the order of its float additions.  The tiled
 * modes are slower on a GB300 (a measured alternative) and apply from the next sort on.  A wait for a TMA box
 * that gives up (after about a second) makes the block take the per-particle path and the step return
 * HRT_ERR_TIMEOUT when the non-finite check is on. */
hrt_status hrt_set_tiled_deposit(hrt_ctx* ctx, int32_t mode);

/* Reverse mode of a whole run (the adjoint method named as future work in Sec. 7).  hrt_set_checkpointing(ctx,
 * k) with k >= 1 makes the context record the run that starts at the next hrt_init_particles_zeldovich: the
 * noise, the steps (hrt_step, hrt_step_accumulate, hrt_sync_particles), the initial ray angles
 * (hrt_init_rays) and, every k steps, a checkpoint of the particles and rays (device memory: 24 B per particle
 * + 48 B per ray per checkpoint, freed by the next call or hrt_destroy); k = 0 stops recording and frees it.
 * hrt_adjoint then returns the gradient of a loss L with respect to the white noise and Omega_m, given
 * kappa_bar (device float32 [n_sources][n_rays], dL/dkappa of the maps as they are at the end of the run, or
 * NULL) and theta_bar (device FP64 [n_rays][2], dL/dtheta of the final ray angles, or NULL): noise_bar (device
 * float32 [n_side^3]) receives dL/dnoise and *omega_bar_host (or NULL) dL/dOmega_m.  It recomputes each
 * segment of k steps from its checkpoint (transient device memory: k pre-step states of particles, rays and
 * the three fields) and runs the adjoint calls above in reverse.  Supported: Zel'dovich or 2LPT ICs, ray steps
 * on the particle fields (ray_fields == 0) with the direct gather or the ray mesh, untiled or through a tiled
 * light cone; given initial particles, loaded states, static-lens steps, free drifts, ray fields and replicas
 * changed during the run make the record unusable
 * (HRT_ERR_STATE with the reason).  Synchronises the context's stream. */
hrt_status hrt_set_checkpointing(hrt_ctx* ctx, int32_t every);
hrt_status hrt_adjoint(hrt_ctx* ctx, const float* kappa_bar, const double* theta_bar, float* noise_bar,
                       double* omega_bar_host);

/* Kick operator of the context's rays: cfg != NULL switches to the ray-mesh kick of hrt_raymesh_ray_step
 * (configuration copied; the context owns its workspace), cfg == NULL back to the direct line-of-sight
 * gather.  The ray mesh reads the same 3D fields as the direct gather (the ray fields when ray_fields == 2; all
 * three particle fields through a tiled light cone, hrt_set_replicas).  HRT_ERR_INVALID_ARG for a bad
 * configuration.  Takes effect at the next ray step. */
hrt_status hrt_set_ray_mesh(hrt_ctx* ctx, const hrt_raymesh_config* cfg);

/* Fixed learned correction of the ray force: g_table[nk] (device float32, copied) sampled uniformly on
 * |k| in [0, kmax], multiplying the Green's function of the ray fields (linear interpolation, 1 beyond kmax),
 * the same at every step; the a-independent form of hrt_set_ray_correction, which it replaces (and vice
 * versa).  Needs ray_fields == 2 (HRT_ERR_STATE otherwise).  g_table == NULL removes it.  Takes effect at the
 * next force evaluation. */
hrt_status hrt_set_ray_kernel_table(hrt_ctx* ctx, const float* g_table, int32_t nk, double kmax);

/* Checkpoint and resume of a context.  hrt_state_bytes gives the size of the state of the context as it is
 * now (particles, rays, maps); hrt_save_state writes it into caller device memory buf (a header, then the
 * displacements and momenta, the ray angles, momenta, A and B, and the maps) and synchronises the stream;
 * HRT_ERR_INVALID_ARG if bytes is too small, HRT_ERR_STATE without particles.  hrt_load_state restores such a
 * state into a context of the same particle and mesh sides (HRT_ERR_INVALID_ARG otherwise), reallocating its
 * rays, and recomputes the PM force at the saved scale factor from the particles, so that stepping on gives
 * the run that was saved (up to the rounding order of the deposit).  The learned correction and the profiling
 * state are not part of it. */
hrt_status hrt_state_bytes(hrt_ctx* ctx, size_t* bytes);
hrt_status hrt_save_state(hrt_ctx* ctx, void* buf, size_t bytes);
hrt_status hrt_load_state(hrt_ctx* ctx, const void* buf, size_t bytes);

/* One co-evolution step as hrt_step, with the rays' readout accumulated instead of written: map `source` (>= 0)
 * += weight * (kappa, gamma1, gamma2, omega) of the rays at the end of the step.  Called at every reverse step
 * with weight = n_g(chi_n), it builds the observable O = sum_n n_g(chi_n) O_n of a source distribution n_g
 * (Eq. obs_accum); the weights are the caller's, normalised as it chooses.  Maps start at zero after
 * hrt_init_rays.  HRT_ERR_INVALID_ARG for source < 0 or a non-finite weight. */
hrt_status hrt_step_accumulate(hrt_ctx* ctx, double a_next, int32_t source, double weight);

/* Kick the momenta from their time to the current a with the current force (synchronise). */
hrt_status hrt_sync_particles(hrt_ctx* ctx);

/* Static mode: trace rays through [chi_from, chi_to] in the fixed potential (a = 1, no growth), readout
 * to map `source` if >= 0.  Particles do not move. */
hrt_status hrt_step_static(hrt_ctx* ctx, double chi_from, double chi_to, int32_t source);

/* Exact force-free drift of the rays (see hrt_ray_drift_free). */
hrt_status hrt_drift_free(hrt_ctx* ctx, double chi_from, double chi_to);

/* Copies of the context state into caller buffers (any pointer may be NULL), stream-ordered on the context's
 * stream.  hrt_read_rays and hrt_read_maps accept device or host memory (a pinned host buffer is filled
 * asynchronously: synchronise the stream before reading it); hrt_read_particles and hrt_read_grad write
 * device memory only. */
hrt_status hrt_read_rays(hrt_ctx* ctx, double* theta, float* eta, float* A, float* B);
hrt_status hrt_read_maps(hrt_ctx* ctx, int32_t source, float* kappa, float* gamma1, float* gamma2,
                         float* omega);
hrt_status hrt_read_particles(hrt_ctx* ctx, float* disp, float* mom, double* a_host, double* a_mom_host);
hrt_status hrt_read_grad(hrt_ctx* ctx, float* grad /* [3][n^3] */);

/* Asynchronous read-outs of the results of Algorithm 1 that a caller takes every step: the ray angles theta
 * (FP64 [n_rays][2], advanced by Eq. "drift"; their difference from the initial angles is the deflection) and
 * the convergence map kappa of source plane `source` (float32 [n_rays], the readout of Eqs. "obs_first_set").
 * Each call snapshots the data into a device staging buffer on the context's stream, in order after the work
 * queued so far, and copies it to host_dst on a separate copy stream, so that the copy runs beside the
 * context's next steps; the call itself returns at once.  host_dst is host memory (pinned, for the copy to
 * overlap) that stays valid until hrt_read_wait has returned HRT_OK, and holds the data from then on; copies
 * into the same buffer land in the order of the calls.  hrt_read_wait blocks until every asynchronous copy so
 * far has landed (bounded by hrt_set_host_wait_limit: HRT_ERR_TIMEOUT).  Device memory: 20 B per ray for the
 * staging buffer, allocated on first use.  Errors: HRT_ERR_STATE without rays (or maps), HRT_ERR_INVALID_ARG
 * for a NULL destination or a source out of range. */
hrt_status hrt_read_rays_async(hrt_ctx* ctx, double* theta_host);
hrt_status hrt_read_kappa_async(hrt_ctx* ctx, int32_t source, float* kappa_host);
hrt_status hrt_read_wait(hrt_ctx* ctx);

/* Opt-in checks for NaN and infinity (off by default).  With on = 1, hrt_init_particles and hrt_init_rays
 * scan the state they copied in and return HRT_ERR_NONFINITE before using it (the context then has no
 * particles, or no rays), and hrt_step / hrt_step_accumulate scan the particle state, the ray state and the
 * maps after the step and return HRT_ERR_NONFINITE if any value is not finite.  Each check waits for the
 * context's stream (within the host wait limit), so it costs a synchronisation and a pass over the state.
 * A kernel that gave up waiting for its own copies is reported here as HRT_ERR_TIMEOUT.  Neither status
 * poisons the context. */
hrt_status hrt_set_nonfinite_check(hrt_ctx* ctx, int32_t on);

/* Poisson prefactor of a static lens of total mass `mass` (Msun/h) in a periodic box of side `box` (Mpc/h):
 * 4 pi G M / box^3 in the library's units ((100 km/s)^2 per (Mpc/h)^2), the value hrt_config.static_pref takes
 * for the point-mass test (Sec. 6.1; the FFT solve then sees delta = rho / rho_mean - 1).  HRT_ERR_INVALID_ARG
 * for a non-positive or non-finite mass or box. */
hrt_status hrt_static_prefactor(double mass, double box, double* pref);

/* Precision ablation of the direct line-of-sight kick: bits = 64 (the default, the method as built) keeps the
 * ray angles in FP64 and forms each interpolation position from an FP64 cell / fraction split (Alg. 1 ray
 * state, Sec. 3.1); bits = 32 keeps the angles in FP32 (rounded after every drift) and forms the positions in
 * FP32, which is what a single-precision build would do.  For measuring what the FP64 parts buy; a recorded run
 * for hrt_adjoint is invalidated by bits = 32.  HRT_ERR_INVALID_ARG for other values. */
hrt_status hrt_set_ray_theta_bits(hrt_ctx* ctx, int32_t bits);

/* Host-side fault injection for tests of the error paths: the k-th device allocation of the library from now
 * (1-based) reports HRT_ERR_OOM as if the device were out of memory; k = 0 turns it off.  The environment
 * variable HRT_FAIL_ALLOC_AT=k does the same from process start.  Process-wide; HRT_ERR_INVALID_ARG for k < 0. */
hrt_status hrt_inject_alloc_failure(int64_t k);

/* Process-wide limit, in seconds, of the library's host waits for a stream (hrt_kappa_power and
 * hrt_ctx_kappa_power waiting for the work already queued, the checks above); seconds <= 0 removes it (the
 * default).  When a wait exceeds it the call returns HRT_ERR_TIMEOUT; the queued work keeps running and the
 * call may be repeated.  HRT_ERR_INVALID_ARG for NaN. */
hrt_status hrt_set_host_wait_limit(double seconds);

/* Power spectrum of the kappa map of `source` (the rays must form an m x m image, m^2 = n_rays). */
hrt_status hrt_ctx_kappa_power(hrt_ctx* ctx, int32_t source, int64_t m, double dtheta, int32_t nbins,
                               double ell_min, double ell_max, double* ell_host, double* p_host,
                               int64_t* count_host);

/* Phase timing with CUDA events recorded on the context's stream around each part of a step.  Phases:
 * 0 ray step, 1 particle kick-drift (in hrt_step fused with the CIC deposit of the next density, and with
 * its memset), 2 stand-alone CIC scatter (initial force only), 3 R2C FFT, 4 k-space kernel,
 * 5 C2R FFTs (all fields), 6 whole hrt_step.  hrt_ctx_phase_times synchronises, returns the summed
 * milliseconds and launch counts since the last call (arrays of 8), and resets them. */
hrt_status hrt_ctx_set_profiling(hrt_ctx* ctx, int32_t on);
hrt_status hrt_ctx_phase_times(hrt_ctx* ctx, double* ms_host, int64_t* counts_host);

/* Device pointers of the context's ray state (for callers that launch the ray kernels directly). */
hrt_status hrt_ctx_rays(hrt_ctx* ctx, hrt_rays* out_host);

#ifdef __cplusplus
}
#endif

#endif /* HRT_H */
