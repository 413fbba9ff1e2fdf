// Internal: the context object behind hrt_ctx (api.cu) and the record of a run that its adjoint replays
// (tape.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <utility>
#include <vector>

#include "common.h"

namespace hrt {

// One recorded step of a context: 'F' particles only, 'S' the synchronising kick, 'R' rays and particles.
struct TapeStep {
  char kind;
  double a_x, a_next, a_p;  // position time before and after, momentum time before
  int slot;                 // map written after a ray step (-1: none)
  double weight;            // readout weight when accumulating
  bool accumulate;
  bool mesh;                // the rays were kicked on the ray mesh ...
  hrt_raymesh_config mesh_cfg;  // ... of this configuration
  bool tiled;               // through the light cone tiled by the tape's replicas
};

// State before a step, kept every `every` steps.
struct TapeCheckpoint {
  float* disp = nullptr;
  float* mom = nullptr;
  hrt_rays rays{};  // theta == nullptr: no rays yet
};

struct Tape {
  int every = 0;
  bool valid = false;           // a run from Zel'dovich ICs is being recorded
  const char* invalid_why = "no initial conditions from white noise recorded";
  double a_init = 0.0;
  bool lpt2 = false;            // 2LPT (else Zel'dovich) initial conditions
  float* noise = nullptr;       // copy of the white noise
  float* disp0 = nullptr;       // displacements of the ICs
  double* theta0 = nullptr;     // initial ray angles
  int64_t n_rays = 0;
  int rays_start = -1;          // index of the first step with rays
  std::vector<TapeStep> steps;
  std::map<int, TapeCheckpoint> checkpoints;
  std::vector<int32_t> rep_perm, rep_sign, rep_shift;  // replicas of the tiled steps
};

void device_free(void* p, cudaStream_t s);

}  // namespace hrt

struct hrt_ctx {
  hrt_config cfg{};
  cudaStream_t stream = nullptr;
  bool poisoned = false;
  hrt_pm* pm = nullptr;
  float* disp = nullptr;
  float* mom = nullptr;
  float* rho = nullptr;
  float* grad = nullptr;
  float* ray_grad = nullptr;
  bool have_particles = false;
  bool force_valid = false;  // grad (and ray_grad) hold the force of the current particles
  double a = 1.0, a_mom = 1.0;
  hrt_rays rays{};
  float* maps = nullptr;
  int64_t maps_rays = 0;
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> phases[8];
  // second stream for the ray step, which overlaps the particle update of the same step (both only read
  // the force fields); ev_fields: fields ready, ev_rays: ray step done (the next C2R waits for it)
  cudaStream_t ray_stream = nullptr;
  cudaEvent_t ev_fields = nullptr, ev_rays = nullptr;
  bool rays_pending = false;
  // asynchronous read-outs (hrt_read_rays_async, hrt_read_kappa_async): results are staged in a device buffer on
  // the context stream and copied to the host on copy_stream, beside the next steps; region 0 holds the ray angles
  // (16 B per ray), region 1 one convergence map (4 B per ray); ev_copied[i]: the last copy out of region i
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_staged = nullptr, ev_copied[2] = {nullptr, nullptr};
  bool copy_pending[2] = {false, false};
  char* stage = nullptr;
  size_t stage_bytes = 0;   // allocated
  size_t stage_layout = 0;  // bytes of the layout in use (20 B per ray of the current rays)
  // learned ray-force correction (NULL: plain)
  float* corr_w = nullptr;
  void* corr_wb = nullptr;
  float* corr_x = nullptr;
  float* corr_table = nullptr;
  // learned correction of the particle force (NULL: plain), the same network form evaluated per force at a
  float* pcorr_w = nullptr;
  void* pcorr_wb = nullptr;
  float* pcorr_x = nullptr;
  float* pcorr_table = nullptr;
  // light-cone tiling (empty: none): [n][3] perm, sign, shift
  std::vector<int32_t> rep_perm, rep_sign, rep_shift;
  // ray-mesh kick operator of Sec. 5.2 (NULL: the direct line-of-sight gather)
  hrt_raymesh* raymesh = nullptr;
  // record of the run for hrt_adjoint (NULL: not recording)
  hrt::Tape* tape = nullptr;
  // particles stored in cell order, re-sorted every sort_every particle steps (0: never): slot i of disp and mom
  // holds lattice particle order_buf[order_cur][i] (order_cur < 0: lattice order)
  int32_t* order_buf[2] = {nullptr, nullptr};
  int order_cur = -1;
  float* disp_alt = nullptr;
  float* mom_alt = nullptr;
  int32_t* sort_scratch = nullptr;
  int32_t sort_every = 0;
  int32_t steps_since_sort = 0;
  // rho was set to zero by the last solve (split path): the next deposit needs no memset
  bool rho_clear = false;
  // the sort of the current order used brick keys; particles given by the caller are sorted before their first
  // force whatever the interval
  bool sort_bricks = false;
  bool sort_first = false;
  // kick-drift-deposit with shared-memory field and density tiles on brick-sorted particles: 0 off (the
  // default, z-row keys), 1 tiles copied by rows, 2 TMA boxes for the tiles inside the mesh
  int tiled_deposit = 0;
  // fixed learned table of the ray fields (NULL: none); exclusive with the network above
  float* ray_table = nullptr;
  int32_t ray_table_nk = 0;
  double ray_table_kmax = 0.0;
  // opt-in checks for NaN and infinity (hrt_set_nonfinite_check): device flag of the scans
  bool theta32 = false;  // FP32 ray-angle ablation of the direct kick (hrt_set_ray_theta_bits)
  bool check_finite = false;
  int* finite_flag = nullptr;
};

namespace hrt {

hrt_filter ctx_filter(const hrt_config& c, bool ray);
// The slot -> lattice index map of the context's particles (nullptr: lattice order).
const int32_t* ctx_order(const hrt_ctx* ctx);
// The context's particles in lattice order into disp_out, mom_out ([3][np] device, either may be NULL).
hrt_status ctx_particles_lattice(hrt_ctx* ctx, float* disp_out, float* mom_out);
hrt_ray_geom ctx_geom(const hrt_config& c, const hrt_ctx* ctx);

// Recording hooks (tape.cu); each is a no-op without a tape.
hrt_status tape_on_ics(hrt_ctx* ctx, const float* noise, double a_init, bool lpt2);
hrt_status tape_on_rays(hrt_ctx* ctx, const double* theta0, int64_t n_rays);
hrt_status tape_on_step(hrt_ctx* ctx, char kind, double a_next, int slot, double weight, bool accumulate);
void tape_invalidate(hrt_ctx* ctx, const char* why);
void tape_free(hrt_ctx* ctx);
// Gradients of a recorded run (hrt_adjoint).
hrt_status tape_adjoint(hrt_ctx* ctx, const float* kappa_bar, const double* theta_bar, float* noise_bar,
                        double* omega_bar);

}  // namespace hrt
