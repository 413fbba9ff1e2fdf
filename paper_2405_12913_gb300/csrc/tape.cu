// Reverse mode of a whole context run (hrt_adjoint): the context records its run (tape_on_* hooks) with a
// checkpoint of the particle and ray state every `every` steps; the adjoint walks the checkpoint segments
// backwards, recomputes each segment forward from its checkpoint (keeping the pre-step states), and applies the
// adjoint calls of the library step by step in reverse.  Omega_m enters only through host FP64 coefficients
// (IC table and momentum ratio, particle kick and drift integrals, Poisson prefactors, the ray steps' node or
// plane weights and drift coefficients); the kernels return their cotangents and the host chains them with
// FP64 central differences of the coefficient builders.  The adjoint method is named as future work in Sec. 7.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "common.h"
#include "context.h"
#include "cosmo.h"
#include "mesh_kernels.h"
#include "raymesh.h"

namespace hrt {

namespace {

constexpr double kEpsOmega = 1e-5;

// Device buffers freed together when the scope ends.
struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (void* p : ptrs) device_free(p, s);
  }
  template <typename T>
  hrt_status get(T** p, size_t count, const char* what) {
    HRT_TRY(device_alloc(reinterpret_cast<void**>(p), count * sizeof(T), s, what));
    ptrs.push_back(*p);
    return HRT_OK;
  }
};

void free_rays(hrt_rays& r, cudaStream_t s) {
  device_free(r.theta, s);
  device_free(r.eta, s);
  device_free(r.A, s);
  device_free(r.B, s);
  r = hrt_rays{};
}

hrt_status alloc_rays(hrt_rays& r, int64_t n, cudaStream_t s) {
  r = hrt_rays{};
  r.n_rays = n;
  hrt_status st = device_alloc(reinterpret_cast<void**>(&r.theta), 2 * n * sizeof(double), s, "tape theta");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&r.eta), 2 * n * sizeof(float), s, "tape eta");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&r.A), 4 * n * sizeof(float), s, "tape A");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&r.B), 4 * n * sizeof(float), s, "tape B");
  if (st != HRT_OK) free_rays(r, s);
  return st;
}

hrt_status copy_rays(const hrt_rays& dst, const hrt_rays& src, cudaStream_t s) {
  const int64_t n = src.n_rays;
  HRT_CUDA(cudaMemcpyAsync(dst.theta, src.theta, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  HRT_CUDA(cudaMemcpyAsync(dst.eta, src.eta, 2 * n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  HRT_CUDA(cudaMemcpyAsync(dst.A, src.A, 4 * n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  HRT_CUDA(cudaMemcpyAsync(dst.B, src.B, 4 * n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return HRT_OK;
}

hrt_status copy_floats(float* dst, const float* src, int64_t count, cudaStream_t s) {
  return cuda_status(cudaMemcpyAsync(dst, src, count * sizeof(float), cudaMemcpyDeviceToDevice, s), "tape copy");
}

void tape_clear(Tape& t, cudaStream_t s) {
  device_free(t.noise, s);
  device_free(t.disp0, s);
  device_free(t.theta0, s);
  t.noise = t.disp0 = nullptr;
  t.theta0 = nullptr;
  for (auto& kv : t.checkpoints) {
    device_free(kv.second.disp, s);
    device_free(kv.second.mom, s);
    free_rays(kv.second.rays, s);
  }
  t.checkpoints.clear();
  t.steps.clear();
  t.rep_perm.clear();
  t.rep_sign.clear();
  t.rep_shift.clear();
  t.valid = false;
  t.invalid_why = "no initial conditions from white noise recorded";
  t.n_rays = 0;
  t.rays_start = -1;
}

// A_bar[:, 0] and A_bar[:, 3] -= c kappa_bar (kappa = 1 - (A11 + A22) / 2 read out with weight w: c = w / 2).
__global__ void kappa_inject_kernel(float4* __restrict__ A_bar, const float* __restrict__ kb, float c, int64_t n) {
  const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (r >= n) return;
  float4 a = A_bar[r];
  const float v = c * kb[r];
  a.x -= v;
  a.w -= v;
  A_bar[r] = a;
}

// The state the step recursion carries.
struct State {
  float* d;
  float* m;
  hrt_rays rays;
  bool has_rays;
  float* g;
};

}  // namespace

void tape_free(hrt_ctx* ctx) {
  if (!ctx->tape) return;
  tape_clear(*ctx->tape, ctx->stream);
  delete ctx->tape;
  ctx->tape = nullptr;
}

void tape_invalidate(hrt_ctx* ctx, const char* why) {
  if (ctx->tape && ctx->tape->valid) {
    ctx->tape->valid = false;
    ctx->tape->invalid_why = why;
  }
}

hrt_status tape_on_ics(hrt_ctx* ctx, const float* noise, double a_init, bool lpt2) {
  if (!ctx->tape) return HRT_OK;
  Tape& t = *ctx->tape;
  cudaStream_t s = ctx->stream;
  tape_clear(t, s);
  const int64_t np = ctx->cfg.n_side * ctx->cfg.n_side * ctx->cfg.n_side;
  HRT_TRY(device_alloc(reinterpret_cast<void**>(&t.noise), np * sizeof(float), s, "tape noise"));
  HRT_TRY(device_alloc(reinterpret_cast<void**>(&t.disp0), 3 * np * sizeof(float), s, "tape ICs"));
  HRT_TRY(copy_floats(t.noise, noise, np, s));
  HRT_TRY(copy_floats(t.disp0, ctx->disp, 3 * np, s));
  t.a_init = a_init;
  t.lpt2 = lpt2;
  t.valid = true;
  if (ctx->pcorr_w) tape_invalidate(ctx, "a learned particle force is not differentiated");
  return HRT_OK;
}

hrt_status tape_on_rays(hrt_ctx* ctx, const double* theta0, int64_t n_rays) {
  if (!ctx->tape || !ctx->tape->valid) return HRT_OK;
  Tape& t = *ctx->tape;
  if (t.rays_start >= 0) {
    tape_invalidate(ctx, "the rays were initialised twice in the recorded run");
    return HRT_OK;
  }
  HRT_TRY(device_alloc(reinterpret_cast<void**>(&t.theta0), 2 * n_rays * sizeof(double), ctx->stream, "tape rays"));
  HRT_CUDA(cudaMemcpyAsync(t.theta0, theta0, 2 * n_rays * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  t.n_rays = n_rays;
  t.rays_start = static_cast<int>(t.steps.size());
  return HRT_OK;
}

hrt_status tape_on_step(hrt_ctx* ctx, char kind, double a_next, int slot, double weight, bool accumulate) {
  if (!ctx->tape || !ctx->tape->valid) return HRT_OK;
  Tape& t = *ctx->tape;
  if (ctx->pcorr_w) {
    tape_invalidate(ctx, "a learned particle force is not differentiated");
    return HRT_OK;
  }
  if (kind == 'R' && t.rays_start < 0) {
    tape_invalidate(ctx, "a ray step ran with rays not initialised after the recorded ICs");
    return HRT_OK;
  }
  const bool tiled = kind == 'R' && !ctx->rep_perm.empty();
  if (kind == 'R' && ctx->cfg.ray_fields != 0) {
    tape_invalidate(ctx, "the adjoint supports ray steps on the particle fields only");
    return HRT_OK;
  }
  if (tiled) {
    if (t.rep_perm.empty()) {
      t.rep_perm = ctx->rep_perm;
      t.rep_sign = ctx->rep_sign;
      t.rep_shift = ctx->rep_shift;
    } else if (t.rep_perm != ctx->rep_perm || t.rep_sign != ctx->rep_sign || t.rep_shift != ctx->rep_shift) {
      tape_invalidate(ctx, "the light-cone replicas changed during the recorded run");
      return HRT_OK;
    }
  }
  const int idx = static_cast<int>(t.steps.size());
  if (idx % t.every == 0) {
    cudaStream_t s = ctx->stream;
    const int64_t np3 = 3 * ctx->cfg.n_side * ctx->cfg.n_side * ctx->cfg.n_side;
    TapeCheckpoint c;
    hrt_status st = device_alloc(reinterpret_cast<void**>(&c.disp), np3 * sizeof(float), s, "checkpoint");
    if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&c.mom), np3 * sizeof(float), s, "checkpoint");
    if (st == HRT_OK) st = ctx_particles_lattice(ctx, c.disp, c.mom);
    if (st == HRT_OK && t.rays_start >= 0 && idx >= t.rays_start) {
      st = alloc_rays(c.rays, t.n_rays, s);
      if (st == HRT_OK) st = copy_rays(c.rays, ctx->rays, s);
    }
    if (st != HRT_OK) {
      device_free(c.disp, s);
      device_free(c.mom, s);
      free_rays(c.rays, s);
      return st;
    }
    t.checkpoints[idx] = c;
  }
  TapeStep st{kind, ctx->a, a_next, ctx->a_mom, slot, weight, accumulate, ctx->raymesh != nullptr, {}, tiled};
  if (ctx->raymesh) st.mesh_cfg = raymesh_config_of(ctx->raymesh);
  t.steps.push_back(st);
  return HRT_OK;
}

namespace {

// Kick and drift integrals of a particle step (as the context's step uses them).
void step_coefficients(const TapeStep& st, double om, double& K, double& D) {
  Cosmo c(om);
  if (st.kind == 'S') {
    K = c.kick(st.a_p, st.a_x);
    D = 0.0;
    return;
  }
  const double a_half = 0.5 * (st.a_x + st.a_next);
  K = c.kick(st.a_p, a_half);
  D = c.drift(st.a_x, st.a_next);
}

struct MeshSet {
  std::vector<std::pair<hrt_raymesh_config, hrt_raymesh*>> list;
  ~MeshSet() {
    for (auto& e : list) hrt_raymesh_destroy(e.second);
  }
  hrt_status get(const hrt_raymesh_config& c, hrt_raymesh** out) {
    for (auto& e : list)
      if (std::memcmp(&e.first, &c, sizeof(c)) == 0) {
        *out = e.second;
        return HRT_OK;
      }
    HRT_TRY(hrt_raymesh_create(&c, out));
    list.emplace_back(c, *out);
    return HRT_OK;
  }
};

}  // namespace

hrt_status tape_adjoint(hrt_ctx* ctx, const float* kappa_bar, const double* theta_bar, float* noise_bar,
                        double* omega_bar) {
  if (!ctx->tape) return fail(HRT_ERR_STATE, "the run was not recorded (hrt_set_checkpointing)");
  Tape& t = *ctx->tape;
  if (!t.valid) return fail(HRT_ERR_STATE, "the recorded run cannot be differentiated: %s", t.invalid_why);
  if (t.steps.empty()) return fail(HRT_ERR_STATE, "no steps recorded");
  if (!noise_bar) return fail(HRT_ERR_INVALID_ARG, "noise_bar is NULL");
  const hrt_config& cfg = ctx->cfg;
  cudaStream_t s = ctx->stream;
  const double om = cfg.cosmo.omega_m;
  const int64_t n = cfg.n_mesh, np = cfg.n_side * cfg.n_side * cfg.n_side, m = n * n * n, R = t.n_rays;
  const int n_steps = static_cast<int>(t.steps.size()), k = t.every;
  const hrt_filter f = ctx_filter(cfg, false);
  const hrt_ray_geom geom = ctx_geom(cfg, nullptr);
  hrt_ray_geom geom_tiled = geom;
  if (!t.rep_perm.empty()) {
    geom_tiled.n_replicas = static_cast<int32_t>(t.rep_perm.size() / 3);
    geom_tiled.replica_perm = t.rep_perm.data();
    geom_tiled.replica_sign = t.rep_sign.data();
    geom_tiled.replica_shift = t.rep_shift.data();
  }
  Cosmo cosmo(om);
  auto pref = [&](double a) { return 1.5 * om / a; };

  Scratch sc(s);
  MeshSet meshes;
  State st{};
  std::vector<State> pre(k);
  HRT_TRY(sc.get(&st.d, 3 * np, "adjoint state"));
  HRT_TRY(sc.get(&st.m, 3 * np, "adjoint state"));
  HRT_TRY(sc.get(&st.g, 3 * m, "adjoint fields"));
  for (auto& p : pre) {
    HRT_TRY(sc.get(&p.d, 3 * np, "segment state"));
    HRT_TRY(sc.get(&p.m, 3 * np, "segment state"));
    HRT_TRY(sc.get(&p.g, 3 * m, "segment fields"));
  }
  float *d_bar, *m_bar, *rho_bar, *g_bar, *rho;
  HRT_TRY(sc.get(&d_bar, 3 * np, "disp cotangent"));
  HRT_TRY(sc.get(&m_bar, 3 * np, "mom cotangent"));
  HRT_TRY(sc.get(&rho_bar, m, "density cotangent"));
  HRT_TRY(sc.get(&g_bar, 3 * m, "field cotangent"));
  HRT_TRY(sc.get(&rho, m, "density"));
  hrt_rays r_bar{};
  if (R > 0) {
    for (hrt_rays* r : {&st.rays, &r_bar}) {
      r->n_rays = R;
      HRT_TRY(sc.get(&r->theta, 2 * R, "rays"));
      HRT_TRY(sc.get(&r->eta, 2 * R, "rays"));
      HRT_TRY(sc.get(&r->A, 4 * R, "rays"));
      HRT_TRY(sc.get(&r->B, 4 * R, "rays"));
    }
    for (auto& p : pre) {
      p.rays.n_rays = R;
      HRT_TRY(sc.get(&p.rays.theta, 2 * R, "segment rays"));
      HRT_TRY(sc.get(&p.rays.eta, 2 * R, "segment rays"));
      HRT_TRY(sc.get(&p.rays.A, 4 * R, "segment rays"));
      HRT_TRY(sc.get(&p.rays.B, 4 * R, "segment rays"));
    }
    HRT_CUDA(cudaMemsetAsync(r_bar.theta, 0, 2 * R * sizeof(double), s));
    HRT_CUDA(cudaMemsetAsync(r_bar.eta, 0, 2 * R * sizeof(float), s));
    HRT_CUDA(cudaMemsetAsync(r_bar.A, 0, 4 * R * sizeof(float), s));
    HRT_CUDA(cudaMemsetAsync(r_bar.B, 0, 4 * R * sizeof(float), s));
    if (theta_bar) HRT_CUDA(cudaMemcpyAsync(r_bar.theta, theta_bar, 2 * R * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  double *coef_bar, *node_bar, *drift_bar;
  HRT_TRY(sc.get(&coef_bar, 2 * static_cast<size_t>(n_steps), "coefficient cotangents"));
  HRT_TRY(sc.get(&node_bar, 3 * static_cast<size_t>(kMaxRayNodes) * n_steps, "node cotangents"));
  HRT_TRY(sc.get(&drift_bar, static_cast<size_t>(n_steps), "drift cotangents"));
  HRT_CUDA(cudaMemsetAsync(coef_bar, 0, 2 * n_steps * sizeof(double), s));
  HRT_CUDA(cudaMemsetAsync(node_bar, 0, 3 * kMaxRayNodes * n_steps * sizeof(double), s));
  HRT_CUDA(cudaMemsetAsync(drift_bar, 0, n_steps * sizeof(double), s));
  HRT_CUDA(cudaMemsetAsync(d_bar, 0, 3 * np * sizeof(float), s));
  HRT_CUDA(cudaMemsetAsync(m_bar, 0, 3 * np * sizeof(float), s));
  HRT_CUDA(cudaMemsetAsync(rho_bar, 0, m * sizeof(float), s));
  std::vector<double> pref_bar(n_steps, 0.0), plane_bar(static_cast<size_t>(n_steps) * 1024, 0.0),
      mesh_drift_bar(n_steps, 0.0);
  std::vector<char> seen(std::max<int>(cfg.n_sources, 1), 0);

  // one step of the context's recursion on st (as ctx_step and hrt_sync_particles compute it)
  auto forward = [&](const TapeStep& step) -> hrt_status {
    double K, D;
    step_coefficients(step, om, K, D);
    if (step.kind == 'S') return hrt_particle_kick_drift(st.g, n, cfg.box, cfg.n_side, st.d, st.m, K, 0.0, s);
    if (step.kind == 'R') {
      const double chi0 = cosmo.chi(step.a_x), chi1 = cosmo.chi(step.a_next);
      if (step.mesh) {
        hrt_raymesh* rm;
        HRT_TRY(meshes.get(step.mesh_cfg, &rm));
        if (step.tiled)
          HRT_TRY(hrt_raymesh_ray_step_tiled(rm, &st.rays, st.g, st.g + m, st.g + 2 * m, &geom_tiled, chi0, chi1,
                                             step.a_x, om, nullptr, s));
        else
          HRT_TRY(hrt_raymesh_ray_step(rm, &st.rays, st.g, st.g + m, &geom, chi0, chi1, step.a_x, om, nullptr, s));
      } else if (step.tiled) {
        HRT_TRY(hrt_ray_step_tiled(&st.rays, st.g, st.g + m, st.g + 2 * m, &geom_tiled, chi0, chi1, step.a_x, om,
                                   nullptr, s));
      } else {
        HRT_TRY(hrt_ray_step(&st.rays, st.g, st.g + m, &geom, chi0, chi1, step.a_x, om, nullptr, s));
      }
    }
    HRT_TRY(hrt_particle_kick_drift_deposit(st.g, n, cfg.box, cfg.n_side, st.d, st.m, K, D, rho, s));
    return hrt_pm_solve(ctx->pm, rho, pref(step.a_next), &f, st.g, nullptr, nullptr);
  };

  std::vector<int> starts;
  for (auto& kv : t.checkpoints) starts.push_back(kv.first);
  for (int ci = static_cast<int>(starts.size()) - 1; ci >= 0; --ci) {
    const int s0 = starts[ci], s1 = std::min(s0 + k, n_steps);
    const TapeCheckpoint& cp = t.checkpoints.at(s0);
    HRT_TRY(copy_floats(st.d, cp.disp, 3 * np, s));
    HRT_TRY(copy_floats(st.m, cp.mom, 3 * np, s));
    st.has_rays = cp.rays.theta != nullptr;
    if (st.has_rays) HRT_TRY(copy_rays(st.rays, cp.rays, s));
    // the fields at the checkpoint: the force of its positions at its position time
    HRT_TRY(hrt_cic_scatter(st.d, cfg.n_side, n, cfg.box, rho, s));
    HRT_TRY(hrt_pm_solve(ctx->pm, rho, pref(t.steps[s0].a_x), &f, st.g, nullptr, nullptr));
    for (int i = s0; i < s1; ++i) {
      if (i == t.rays_start) {
        HRT_TRY(hrt_rays_init(&st.rays, t.theta0, s));
        st.has_rays = true;
      }
      State& p = pre[i - s0];
      HRT_TRY(copy_floats(p.d, st.d, 3 * np, s));
      HRT_TRY(copy_floats(p.m, st.m, 3 * np, s));
      HRT_TRY(copy_floats(p.g, st.g, 3 * m, s));
      p.has_rays = st.has_rays;
      if (st.has_rays) HRT_TRY(copy_rays(p.rays, st.rays, s));
      HRT_TRY(forward(t.steps[i]));
    }
    for (int i = s1 - 1; i >= s0; --i) {
      const TapeStep& step = t.steps[i];
      State& p = pre[i - s0];
      double K, D;
      step_coefficients(step, om, K, D);
      if (step.kind == 'R' && step.slot >= 0 && kappa_bar && !seen[step.slot]) {
        // the readout after the step (a later overwrite of the same map hides it)
        const float c = static_cast<float>(0.5 * (step.accumulate ? step.weight : 1.0));
        kappa_inject_kernel<<<blocks_for(R, 256), 256, 0, s>>>(reinterpret_cast<float4*>(r_bar.A),
                                                                 kappa_bar + static_cast<int64_t>(step.slot) * R, c, R);
        HRT_LAUNCHED("kappa_inject_kernel");
      }
      if (step.kind == 'R' && step.slot >= 0 && !step.accumulate) seen[step.slot] = 1;
      HRT_CUDA(cudaMemsetAsync(g_bar, 0, 3 * m * sizeof(float), s));
      if (step.kind == 'S') {
        // the density of these fields was deposited at these positions by the step before
        HRT_TRY(hrt_cic_scatter_adjoint(rho_bar, p.d, cfg.n_side, n, cfg.box, d_bar, s));
        HRT_TRY(hrt_particle_kick_drift_adjoint(p.g, n, cfg.box, cfg.n_side, p.d, p.m, K, 0.0, nullptr, d_bar, m_bar,
                                                g_bar, coef_bar + 2 * i, s));
      } else {
        HRT_TRY(hrt_particle_kick_drift_adjoint(p.g, n, cfg.box, cfg.n_side, p.d, p.m, K, D, rho_bar, d_bar, m_bar,
                                                g_bar, coef_bar + 2 * i, s));
      }
      if (step.kind == 'R') {
        const double chi0 = cosmo.chi(step.a_x), chi1 = cosmo.chi(step.a_next);
        if (step.mesh) {
          hrt_raymesh* rm;
          HRT_TRY(meshes.get(step.mesh_cfg, &rm));
          double* pb = plane_bar.data() + 1024 * static_cast<size_t>(i);
          if (step.tiled)
            HRT_TRY(hrt_raymesh_ray_step_tiled_adjoint(rm, &p.rays, p.g, p.g + m, p.g + 2 * m, &geom_tiled, chi0, chi1,
                                                       step.a_x, om, &r_bar, g_bar, g_bar + m, g_bar + 2 * m, pb,
                                                       &mesh_drift_bar[i], s));
          else
            HRT_TRY(hrt_raymesh_ray_step_adjoint(rm, &p.rays, p.g, p.g + m, &geom, chi0, chi1, step.a_x, om, &r_bar,
                                                 g_bar, g_bar + m, pb, &mesh_drift_bar[i], s));
        } else if (step.tiled) {
          HRT_TRY(hrt_ray_step_tiled_adjoint(&p.rays, p.g, p.g + m, p.g + 2 * m, &geom_tiled, chi0, chi1, step.a_x,
                                             om, &r_bar, g_bar, g_bar + m, g_bar + 2 * m,
                                             node_bar + 3 * kMaxRayNodes * static_cast<size_t>(i), drift_bar + i, s));
        } else {
          HRT_TRY(hrt_ray_step_adjoint(&p.rays, p.g, p.g + m, &geom, chi0, chi1, step.a_x, om, &r_bar, g_bar,
                                       g_bar + m, node_bar + 3 * kMaxRayNodes * static_cast<size_t>(i),
                                       drift_bar + i, s));
        }
      }
      const double pf = pref(step.a_x);
      double dot = 0.0;
      HRT_TRY(hrt_dot(g_bar, p.g, 3 * m, &dot, s));
      pref_bar[i] = dot / pf;
      HRT_TRY(hrt_pm_solve_adjoint(ctx->pm, g_bar, pf, &f, nullptr, nullptr, rho_bar));
    }
  }
  // the initial density from the IC positions, then the ICs
  HRT_TRY(hrt_cic_scatter_adjoint(rho_bar, t.disp0, cfg.n_side, n, cfg.box, d_bar, s));
  const int64_t ntab = 3 * (cfg.n_side / 2) * (cfg.n_side / 2) + 1;
  std::vector<double> table_bar(ntab, 0.0);
  double ratio_bar = 0.0, lpt_bar[4] = {0.0, 0.0, 0.0, 0.0};
  if (t.lpt2)
    HRT_TRY(hrt_ic_2lpt_adjoint(t.noise, cfg.n_side, cfg.box, &cfg.cosmo, t.a_init, d_bar, m_bar, noise_bar,
                                table_bar.data(), lpt_bar, s));
  else
    HRT_TRY(hrt_ic_zeldovich_adjoint(t.noise, cfg.n_side, cfg.box, &cfg.cosmo, t.a_init, d_bar, m_bar, t.disp0,
                                     noise_bar, table_bar.data(), &ratio_bar, s));
  if (!omega_bar) return HRT_OK;

  // Omega_m: FP64 central differences of the host coefficients, weighted by their cotangents
  std::vector<double> coef(2 * n_steps), nodes(3 * kMaxRayNodes * static_cast<size_t>(n_steps)), drift(n_steps);
  HRT_CUDA(cudaMemcpyAsync(coef.data(), coef_bar, coef.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  HRT_CUDA(cudaMemcpyAsync(nodes.data(), node_bar, nodes.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  HRT_CUDA(cudaMemcpyAsync(drift.data(), drift_bar, drift.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  HRT_CUDA(cudaStreamSynchronize(s));
  const double e = kEpsOmega;
  double total = 0.0;
  for (int i = 0; i < n_steps; ++i) {
    const TapeStep& step = t.steps[i];
    double Kp, Dp, Km, Dm;
    step_coefficients(step, om + e, Kp, Dp);
    step_coefficients(step, om - e, Km, Dm);
    total += coef[2 * i] * (Kp - Km) / (2 * e) + coef[2 * i + 1] * (Dp - Dm) / (2 * e);
    total += pref_bar[i] * 1.5 / step.a_x;
    if (step.kind != 'R') continue;
    const double oms[2] = {om + e, om - e};
    if (step.mesh) {
      // plane weights at this run's ray-mesh geometry: w is proportional to g(chi_p) / x2d^2, x2d held fixed
      auto x2d_at = [&](double o, double x[2]) -> hrt_status {
        Cosmo c(o);
        const double c0 = c.chi(step.a_x), c1 = c.chi(step.a_next), mid = 0.5 * (c0 + c1);
        double lam;
        int64_t nn;
        HRT_TRY(hrt_raymesh_geometry(&step.mesh_cfg, c0, mid, cfg.box / n, &lam, &x[0], &nn));
        return hrt_raymesh_geometry(&step.mesh_cfg, mid, c1, cfg.box / n, &lam, &x[1], &nn);
      };
      double x0[2];
      HRT_TRY(x2d_at(om, x0));
      std::vector<double> w[2] = {std::vector<double>(1024, 0.0), std::vector<double>(1024, 0.0)};
      std::vector<double> chi_p(1024);
      int32_t cnt[2][2];
      double dd[2];
      for (int sg = 0; sg < 2; ++sg) {
        Cosmo c(oms[sg]);
        HRT_TRY(hrt_raymesh_step_planes(&step.mesh_cfg, &geom, c.chi(step.a_x), c.chi(step.a_next), step.a_x, oms[sg],
                                        &cnt[sg][0], &cnt[sg][1], chi_p.data(), w[sg].data(), &dd[sg]));
        double xs[2];
        HRT_TRY(x2d_at(oms[sg], xs));
        for (int h = 0; h < 2; ++h)
          for (int q = 0; q < cnt[sg][h]; ++q) w[sg][h * 512 + q] *= (xs[h] / x0[h]) * (xs[h] / x0[h]);
      }
      for (int h = 0; h < 2; ++h) {
        if (cnt[0][h] != cnt[1][h])
          return fail(HRT_ERR_STATE, "a ray-mesh plane changes half shell within the Omega_m difference step");
        for (int q = 0; q < cnt[0][h]; ++q)
          total += plane_bar[1024 * static_cast<size_t>(i) + h * 512 + q] * (w[0][h * 512 + q] - w[1][h * 512 + q]) /
                   (2 * e);
      }
      total += mesh_drift_bar[i] * (dd[0] - dd[1]) / (2 * e);
    } else {
      std::vector<double> cw[2], cwr[2], chi[2];
      double dd[2];
      int32_t n1[2], n2[2];
      for (int sgn = 0; sgn < 2; ++sgn) {
        Cosmo c(oms[sgn]);
        cw[sgn].assign(kMaxRayNodes, 0.0);
        cwr[sgn].assign(kMaxRayNodes, 0.0);
        chi[sgn].assign(kMaxRayNodes, 0.0);
        HRT_TRY(hrt_ray_step_coefficients(step.tiled ? &geom_tiled : &geom, c.chi(step.a_x), c.chi(step.a_next), step.a_x, oms[sgn], &n1[sgn],
                                          &n2[sgn], cw[sgn].data(), cwr[sgn].data(), chi[sgn].data(), &dd[sgn]));
      }
      if (n1[0] + n2[0] != n1[1] + n2[1])
        return fail(HRT_ERR_STATE, "line-of-sight node count changes within the Omega_m difference step");
      const double* nb = nodes.data() + 3 * kMaxRayNodes * static_cast<size_t>(i);
      for (int j = 0; j < n1[0] + n2[0]; ++j)
        total += (nb[j] * (cw[0][j] - cw[1][j]) + nb[kMaxRayNodes + j] * (cwr[0][j] - cwr[1][j]) +
                  nb[2 * kMaxRayNodes + j] * (chi[0][j] - chi[1][j])) / (2 * e);
      total += drift[i] * (dd[0] - dd[1]) / (2 * e);
    }
  }
  std::vector<double> tp(ntab), tm(ntab);
  double rp, rm;
  hrt_cosmology cp = cfg.cosmo, cm = cfg.cosmo;
  cp.omega_m = om + e;
  cm.omega_m = om - e;
  HRT_TRY(hrt_ic_table(cfg.n_side, cfg.box, &cp, t.a_init, tp.data(), &rp));
  HRT_TRY(hrt_ic_table(cfg.n_side, cfg.box, &cm, t.a_init, tm.data(), &rm));
  if (t.lpt2) {
    // the 2LPT transfer is the table at unit growth, and the combine has its own growth coefficients
    double gp[4], gm[4];
    HRT_TRY(hrt_ic_2lpt_coefficients(&cp, t.a_init, gp));
    HRT_TRY(hrt_ic_2lpt_coefficients(&cm, t.a_init, gm));
    for (int64_t j = 0; j < ntab; ++j) total += table_bar[j] * (tp[j] / gp[0] - tm[j] / gm[0]) / (2 * e);
    for (int k = 0; k < 4; ++k) total += lpt_bar[k] * (gp[k] - gm[k]) / (2 * e);
  } else {
    for (int64_t j = 0; j < ntab; ++j) total += table_bar[j] * (tp[j] - tm[j]) / (2 * e);
    total += ratio_bar * (rp - rm) / (2 * e);
  }
  *omega_bar = total;
  return HRT_OK;
}

}  // namespace hrt
