// C ABI of the HRT library (include/hrt.h): argument checks, FP64 host tables, cuFFT plans and the
// simulation context that sequences the kernels of one co-evolution step (Alg. 1).
#include <cuda_runtime.h>
#include <cufft.h>
#include <cufftXt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <new>
#include <thread>
#include <vector>

#include "adjoint.h"
#include "common.h"
#include "context.h"
#include "cosmo.h"
#include "kspace_callback.h"
#include "mesh_kernels.h"
#include "mlp.h"
#include "raymesh.h"
#include "xpass.h"

extern "C" const unsigned char hrt_kspace_callback_fatbin[];
extern "C" const size_t hrt_kspace_callback_fatbin_size;

namespace hrt {

static thread_local char g_err[512];

hrt_status fail(hrt_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

hrt_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HRT_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(HRT_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  }
  return fail(HRT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static hrt_status cufft_status(cufftResult r, const char* what) {
  if (r == CUFFT_SUCCESS) return HRT_OK;
  if (r == CUFFT_ALLOC_FAILED) return fail(HRT_ERR_OOM, "%s: cuFFT allocation failed", what);
  return fail(HRT_ERR_CUDA, "%s: cuFFT error %d", what, static_cast<int>(r));
}
#define HRT_CUFFT(expr) HRT_TRY(::hrt::cufft_status((expr), #expr))

// Host-side allocation-failure injection: the target-th device allocation counted from the last reset reports
// out-of-memory (0: off).  The environment variable HRT_FAIL_ALLOC_AT sets the first target of the process.
static std::atomic<long> g_fail_target{-1};
static std::atomic<long> g_alloc_count{0};

void set_alloc_failure(int64_t k) {
  g_alloc_count.store(0);
  g_fail_target.store(static_cast<long>(k));
}

bool inject_alloc_failure() {
  long target = g_fail_target.load();
  if (target < 0) {
    const char* v = std::getenv("HRT_FAIL_ALLOC_AT");
    long t = v ? std::atol(v) : 0L;
    long expected = -1;
    g_fail_target.compare_exchange_strong(expected, t < 0 ? 0 : t);
    target = g_fail_target.load();
  }
  if (target <= 0) return false;
  return g_alloc_count.fetch_add(1) + 1 == target;
}

hrt_status device_alloc(void** p, size_t bytes, cudaStream_t stream, const char* what) {
  *p = nullptr;
  if (bytes == 0) return HRT_OK;
  if (inject_alloc_failure()) return fail(HRT_ERR_OOM, "%s: injected allocation failure", what);
  return cuda_status(cudaMallocAsync(p, bytes, stream), what);
}

void device_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

static std::atomic<double> g_wait_limit{0.0};

hrt_status wait_stream(cudaStream_t s, const char* what) {
  const double limit = g_wait_limit.load();
  if (!(limit > 0.0)) return cuda_status(cudaStreamSynchronize(s), what);
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) return HRT_OK;
    if (e != cudaErrorNotReady) return cuda_status(e, what);
    const double waited = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (waited > limit)
      return fail(HRT_ERR_TIMEOUT, "%s: the queued work did not finish within the host wait limit of %g s", what,
                  limit);
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

// Uploads host floats to a fresh stream-ordered device buffer (the host copy is consumed before return).
static hrt_status upload(const std::vector<float>& h, float** d, cudaStream_t s, const char* what) {
  HRT_TRY(device_alloc(reinterpret_cast<void**>(d), h.size() * sizeof(float), s, what));
  return cuda_status(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, s), what);
}

static hrt_status check_mesh(int64_t n, double box) {
  if (n < 2 || n % 2 != 0 || n > 2048) return fail(HRT_ERR_INVALID_ARG, "mesh size %lld must be even, 2..2048", (long long)n);
  if (!(box > 0.0) || !std::isfinite(box)) return fail(HRT_ERR_INVALID_ARG, "box must be positive");
  return HRT_OK;
}

static hrt_status check_particles(int64_t n_side, int64_t n) {
  if (n_side < 1 || n % n_side != 0) return fail(HRT_ERR_INVALID_ARG, "n_side %lld must divide the mesh %lld", (long long)n_side, (long long)n);
  return HRT_OK;
}

static hrt_status check_filter(const hrt_filter* f) {
  if (!f) return fail(HRT_ERR_INVALID_ARG, "filter is NULL");
  if (!std::isfinite(f->deconv_p) || !(f->smooth >= 0.0)) return fail(HRT_ERR_INVALID_ARG, "bad filter");
  if (f->g_table && (f->g_nk < 2 || !(f->g_kmax > 0.0))) return fail(HRT_ERR_INVALID_ARG, "bad learned table");
  return HRT_OK;
}

static hrt_status filter_upload(int64_t n, double box, const hrt_filter& f, float** d, cudaStream_t s) {
  std::vector<float> wxy, wz;
  filter_tables(n, box, f, wxy, wz);
  wxy.insert(wxy.end(), wz.begin(), wz.end());
  return upload(wxy, d, s, "filter table");
}

// ---------------------------------------------------------------------------------------------------------
// Ray step parameters: FP64 node table of the half shells (Eq. "kick" with the growth correction).
// ---------------------------------------------------------------------------------------------------------
static hrt_status build_ray_params(const hrt_ray_geom& g, double chi_from, double chi_to, double a_ref,
                                   double omega_m, RayStepParams& p, double* cw64 = nullptr,
                                   double* cwr64 = nullptr, double* chi64 = nullptr) {
  if (!(g.samples_per_cell > 0.0)) return fail(HRT_ERR_INVALID_ARG, "samples_per_cell must be > 0");
  HRT_TRY(check_mesh(g.n, g.box));
  const double cell = g.box / g.n;
  const double chi_mid = 0.5 * (chi_from + chi_to);
  if (!(chi_mid > 0.0)) return fail(HRT_ERR_INVALID_ARG, "shell midpoint must be at chi > 0");
  Cosmo cosmo(omega_m);
  const double d1_ref = a_ref > 0.0 ? cosmo.D1(a_ref) : 1.0;
  p.n = static_cast<int>(g.n);
  p.tile_w = 0;
  p.map_accumulate = 0;
  p.map_weight = 1.f;
  p.theta32 = 0;
  p.tiled = g.n_replicas > 0 ? 1 : 0;
  if (p.tiled) {
    if (g.n_replicas > kMaxReplicas || !g.replica_perm || !g.replica_sign || !g.replica_shift)
      return fail(HRT_ERR_INVALID_ARG, "tiling needs 1..%d replicas with their perm, sign and shift tables", kMaxReplicas);
    for (int k = 0; k < g.n_replicas; ++k) {
      int seen = 0;
      for (int a = 0; a < 3; ++a) {
        const int ax = g.replica_perm[3 * k + a], sg = g.replica_sign[3 * k + a], sh = g.replica_shift[3 * k + a];
        if (ax < 0 || ax > 2 || (sg != 1 && sg != -1) || sh < 0 || sh >= g.n)
          return fail(HRT_ERR_INVALID_ARG, "replica %d: bad axis, sign or shift", k);
        seen |= 1 << ax;
        p.rperm[k][a] = static_cast<signed char>(ax);
        p.rsign[k][a] = static_cast<signed char>(sg);
      }
      if (seen != 7) return fail(HRT_ERR_INVALID_ARG, "replica %d: the axes are not a permutation", k);
      p.rshift[k][0] = g.replica_shift[3 * k + g.replica_perm[3 * k]];
      p.rshift[k][1] = g.replica_shift[3 * k + g.replica_perm[3 * k + 1]];
    }
  }
  p.cell = cell;
  p.box = g.box;
  p.obs_x = g.observer[0];
  p.obs_y = g.observer[1];
  p.drift_d = (chi_to - chi_from) / (kCLight * chi_mid * chi_mid);
  p.drift = static_cast<float>(p.drift_d);
  int total = 0;
  const double lo[2] = {chi_from, chi_mid}, hi[2] = {chi_mid, chi_to};
  for (int h = 0; h < 2; ++h) {
    int cnt = half_shell_count(lo[h], hi[h], g.samples_per_cell, cell);
    double hh = (hi[h] - lo[h]) / cnt;
    p.ref_r[h] = lo[h] + 0.5 * hh;
    int kept = 0;
    for (int j = 0; j < cnt; ++j) {
      double chi = lo[h] + (j + 0.5) * hh;
      if (!(g.window_lo <= chi && chi < g.window_hi)) continue;
      if (total >= kMaxRayNodes) return fail(HRT_ERR_INVALID_ARG, "more than %d line-of-sight nodes in one step", kMaxRayNodes);
      double gw = 1.0;
      if (a_ref > 0.0) {
        double a = cosmo.a_of_chi(chi);
        gw = cosmo.D1(a) / d1_ref * a_ref / a;
      }
      double r = chi;
      double c = -(2.0 / kCLight) * hh * r * gw;
      p.dr[total] = static_cast<float>((r - p.ref_r[h]) / cell);
      p.cw[total] = static_cast<float>(c);
      p.cwr[total] = static_cast<float>(c * r / cell);
      if (cw64) cw64[total] = c;
      if (cwr64) cwr64[total] = c * r / cell;
      if (chi64) chi64[total] = chi;
      double uz = (g.observer[2] + chi) / cell;
      if (p.tiled) {
        // replica of the node and its line-of-sight coordinate on the replica's box axis
        const double zu = g.observer[2] + chi;
        const int k = static_cast<int>(std::floor(zu / g.box));
        if (k < 0 || k >= g.n_replicas)
          return fail(HRT_ERR_INVALID_ARG, "line-of-sight node at chi = %g is outside the %d replicas", chi, g.n_replicas);
        const int ax = g.replica_perm[3 * k + 2];
        uz = (g.replica_sign[3 * k + 2] * (zu - k * g.box)) / cell + g.replica_shift[3 * k + ax];
        p.rep[total] = static_cast<unsigned char>(k);
      }
      uz -= g.n * std::floor(uz / g.n);
      double fl = std::floor(uz);
      int kz = static_cast<int>(fl);
      float fz = static_cast<float>(uz - fl);
      if (kz >= g.n) kz -= static_cast<int>(g.n);
      p.kz[total] = kz;
      p.fz[total] = fz;
      ++total;
      ++kept;
    }
    if (h == 0) p.n1 = kept; else p.n2 = kept;
  }
  return HRT_OK;
}

// 2D tiles when the rays form a W-wide image with W % 16 == 0 and a height that is a multiple of 8 (and the
// 128-thread blocks then cover the rays exactly).
static void set_tiles(const hrt_ray_geom& g, int64_t n_rays, RayStepParams& p) {
  const int64_t w = g.image_width;
  if (w > 0 && w % 16 == 0 && n_rays % w == 0 && (n_rays / w) % 8 == 0 && w < (int64_t{1} << 30)) p.tile_w = static_cast<int>(w);
}

static hrt_status check_rays(const hrt_rays* r) {
  if (!r) return fail(HRT_ERR_INVALID_ARG, "rays is NULL");
  if (r->n_rays < 0) return fail(HRT_ERR_INVALID_ARG, "negative ray count");
  if (r->n_rays > 0 && (!r->theta || !r->eta || !r->A || !r->B)) return fail(HRT_ERR_INVALID_ARG, "ray state pointer is NULL");
  return HRT_OK;
}

}  // namespace hrt

// ---------------------------------------------------------------------------------------------------------
// Context (the struct is in context.h)
// ---------------------------------------------------------------------------------------------------------

namespace hrt {

// Records a CUDA event pair around a phase of a step when profiling is on.
struct PhaseScope {
  hrt_ctx* ctx;
  int phase;
  cudaEvent_t end = nullptr;
  PhaseScope(hrt_ctx* c, int p) : ctx(c), phase(p) {
    if (!ctx->profiling) return;
    cudaEvent_t start;
    if (cudaEventCreate(&start) != cudaSuccess) return;
    if (cudaEventCreate(&end) != cudaSuccess) {
      cudaEventDestroy(start);
      end = nullptr;
      return;
    }
    cudaEventRecord(start, ctx->stream);
    ctx->phases[phase].emplace_back(start, end);
  }
  ~PhaseScope() {
    if (end) cudaEventRecord(end, ctx->stream);
  }
};

}  // namespace hrt

// ---------------------------------------------------------------------------------------------------------
// PM object
// ---------------------------------------------------------------------------------------------------------

struct hrt_pm {
  int64_t n = 0;
  double box = 0.0;
  int32_t n_ray = 0;
  cudaStream_t stream = nullptr;
  cufftHandle r2c = 0, c2r = 0;
  bool have_r2c = false, have_c2r = false;
  void* work = nullptr;
  void* rho_hat = nullptr;
  void* grad_hat = nullptr;     // 3 + n_ray spectra
  float* tab_a = nullptr;       // filter tables (particles)
  float* tab_b = nullptr;       // filter tables (rays)
  hrt_filter key_a{}, key_b{};  // filters the tables were built for
  // fused path: batched C2R plans whose load callback evaluates the k-space kernel (no spectra written)
  bool fused = false;
  cufftHandle c2r_cb3 = 0, c2r_cb2 = 0;
  bool have_cb3 = false, have_cb2 = false;
  hrt::KspaceCallbackInfo* cb_info = nullptr;  // device: [0] particle fields, [1] ray fields
  size_t work_bytes = 0;
  // split path (the default where supported): batched 2D (y, z) plans over the x-planes, and the
  // x-pass kernel between them (forward x-FFT, k-space step, inverse x-FFTs)
  bool split = false;
  cufftHandle r2c2d = 0, c2r2d = 0;
  bool have_r2c2d = false, have_c2r2d = false;
  float2* xtw = nullptr;    // x-FFT twiddles
  int* xerr = nullptr;      // device error word of the kernels that wait for TMA copies (x-pass, tiled deposit)
  bool last_split = false;  // rho_hat holds the (y, z)-transformed density of the split path
};

namespace hrt {

static size_t spectrum_bytes(int64_t n) { return static_cast<size_t>(n) * n * (n / 2 + 1) * sizeof(float2); }
// Bytes of one spectrum buffer: the half spectrum, or the padded split layout where the split path exists.
static size_t spectrum_alloc(int64_t n) {
  return xpass_supported(n) ? static_cast<size_t>(n) * n * xpass_row(n) * sizeof(float2) : spectrum_bytes(n);
}

static bool fusable(int64_t n) { return n >= 8 && n <= 1024 && (n & (n - 1)) == 0; }

// Batched C2R plan with the k-space load callback linked in (LTO, JIT at plan time).
static hrt_status make_callback_plan(hrt_pm* pm, cufftHandle* plan, bool* have, int batch,
                                     hrt::KspaceCallbackInfo* info, size_t* work) {
  long long dims[3] = {pm->n, pm->n, pm->n};
  HRT_CUFFT(cufftCreate(plan));
  *have = true;
  void* info_ptr = info;
  HRT_CUFFT(cufftXtSetJITCallback(*plan, "hrt_kspace_load", hrt_kspace_callback_fatbin,
                                  hrt_kspace_callback_fatbin_size, CUFFT_CB_LD_COMPLEX, &info_ptr));
  HRT_CUFFT(cufftSetAutoAllocation(*plan, 0));
  HRT_CUFFT(cufftMakePlanMany64(*plan, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, batch, work));
  return HRT_OK;
}

static void pm_set_work(hrt_pm* pm) {
  for (cufftHandle p : {pm->r2c, pm->c2r}) {
    cufftSetWorkArea(p, pm->work);
    cufftSetStream(p, pm->stream);
  }
  if (pm->have_cb3) {
    cufftSetWorkArea(pm->c2r_cb3, pm->work);
    cufftSetStream(pm->c2r_cb3, pm->stream);
  }
  if (pm->have_cb2) {
    cufftSetWorkArea(pm->c2r_cb2, pm->work);
    cufftSetStream(pm->c2r_cb2, pm->stream);
  }
  for (int i = 0; i < 2; ++i) {
    if (!(i == 0 ? pm->have_r2c2d : pm->have_c2r2d)) continue;
    cufftHandle p = i == 0 ? pm->r2c2d : pm->c2r2d;
    cufftSetWorkArea(p, pm->work);
    cufftSetStream(p, pm->stream);
  }
}

// Batched 2D (y, z) plans over the n x-planes, spectra rows padded to xpass_row(n), and the x-FFT twiddles.
static hrt_status pm_make_split(hrt_pm* pm, size_t* work) {
  const long long n = pm->n, nzp = xpass_row(pm->n);
  long long dims[2] = {n, n}, real_embed[2] = {n, n}, spec_embed[2] = {n, nzp};
  size_t w1 = 0, w2 = 0;
  HRT_CUFFT(cufftCreate(&pm->r2c2d));
  pm->have_r2c2d = true;
  HRT_CUFFT(cufftSetAutoAllocation(pm->r2c2d, 0));
  HRT_CUFFT(cufftMakePlanMany64(pm->r2c2d, 2, dims, real_embed, 1, n * n, spec_embed, 1, n * nzp, CUFFT_R2C, n, &w1));
  HRT_CUFFT(cufftCreate(&pm->c2r2d));
  pm->have_c2r2d = true;
  HRT_CUFFT(cufftSetAutoAllocation(pm->c2r2d, 0));
  HRT_CUFFT(cufftMakePlanMany64(pm->c2r2d, 2, dims, spec_embed, 1, n * nzp, real_embed, 1, n * n, CUFFT_C2R, n, &w2));
  *work = std::max(w1, w2);
  std::vector<float2> tw;
  xpass_twiddles(pm->n, tw);
  HRT_TRY(device_alloc(reinterpret_cast<void**>(&pm->xerr), sizeof(int), pm->stream, "x-pass error word"));
  HRT_CUDA(cudaMemsetAsync(pm->xerr, 0, sizeof(int), pm->stream));
  HRT_TRY(device_alloc(reinterpret_cast<void**>(&pm->xtw), tw.size() * sizeof(float2), pm->stream, "twiddles"));
  HRT_CUDA(cudaMemcpyAsync(pm->xtw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, pm->stream));
  // the host vector must outlive the copy
  HRT_CUDA(cudaStreamSynchronize(pm->stream));
  return HRT_OK;
}

static hrt_status pm_make(int64_t n, double box, int32_t n_ray, cudaStream_t s, hrt_pm* pm) {
  pm->n = n;
  pm->box = box;
  pm->n_ray = n_ray;
  pm->stream = s;
  long long dims[3] = {n, n, n};
  size_t w1 = 0, w2 = 0;
  HRT_CUFFT(cufftCreate(&pm->r2c));
  pm->have_r2c = true;
  HRT_CUFFT(cufftSetAutoAllocation(pm->r2c, 0));
  HRT_CUFFT(cufftMakePlanMany64(pm->r2c, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 1, &w1));
  HRT_CUFFT(cufftCreate(&pm->c2r));
  pm->have_c2r = true;
  HRT_CUFFT(cufftSetAutoAllocation(pm->c2r, 0));
  HRT_CUFFT(cufftMakePlanMany64(pm->c2r, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 1, &w2));
  pm->work_bytes = std::max(w1, w2);
  if (xpass_supported(n)) {
    size_t w3 = 0;
    HRT_TRY(pm_make_split(pm, &w3));
    pm->work_bytes = std::max(pm->work_bytes, w3);
    pm->split = true;
  }
  HRT_TRY(device_alloc(&pm->work, pm->work_bytes, s, "cuFFT work area"));
  pm_set_work(pm);
  HRT_TRY(device_alloc(&pm->rho_hat, spectrum_alloc(n), s, "rho_hat"));
  HRT_TRY(device_alloc(&pm->grad_hat, spectrum_alloc(n) * (3 + n_ray), s, "gradient spectra"));
  return HRT_OK;
}

// Builds the batched C2R plans with the k-space load callback (on request only: on a GB300 with cuFFT 12.0 the
// callback plans run the three inverse transforms in 36-40 ms at 1024^3, against 21 ms for three plain C2R
// plus the separate k-space kernel, so the context does not use them).
static hrt_status pm_build_fused(hrt_pm* pm) {
  if (pm->have_cb3) return HRT_OK;
  if (!fusable(pm->n)) return fail(HRT_ERR_INVALID_ARG, "fused plans need a power-of-two mesh side <= 1024");
  size_t w3 = 0, w4 = 0;
  if (!pm->cb_info)
    HRT_TRY(device_alloc(reinterpret_cast<void**>(&pm->cb_info), 2 * sizeof(KspaceCallbackInfo), pm->stream,
                         "callback info"));
  hrt_status cs = make_callback_plan(pm, &pm->c2r_cb3, &pm->have_cb3, 3, pm->cb_info, &w3);
  if (cs == HRT_OK && pm->n_ray > 0)
    cs = make_callback_plan(pm, &pm->c2r_cb2, &pm->have_cb2, pm->n_ray, pm->cb_info + 1, &w4);
  if (cs != HRT_OK) {
    if (pm->have_cb3) cufftDestroy(pm->c2r_cb3);
    if (pm->have_cb2) cufftDestroy(pm->c2r_cb2);
    pm->have_cb3 = pm->have_cb2 = false;
    return cs;
  }
  const size_t need = std::max(w3, w4);
  if (need > pm->work_bytes) {
    device_free(pm->work, pm->stream);
    pm->work = nullptr;
    HRT_TRY(device_alloc(&pm->work, need, pm->stream, "cuFFT work area"));
    pm->work_bytes = need;
  }
  pm_set_work(pm);
  return HRT_OK;
}

static void pm_release(hrt_pm* pm) {
  if (!pm) return;
  cudaStreamSynchronize(pm->stream);
  if (pm->have_r2c) cufftDestroy(pm->r2c);
  if (pm->have_c2r) cufftDestroy(pm->c2r);
  if (pm->have_cb3) cufftDestroy(pm->c2r_cb3);
  if (pm->have_cb2) cufftDestroy(pm->c2r_cb2);
  if (pm->have_r2c2d) cufftDestroy(pm->r2c2d);
  if (pm->have_c2r2d) cufftDestroy(pm->c2r2d);
  device_free(pm->xtw, pm->stream);
  device_free(pm->xerr, pm->stream);
  device_free(pm->work, pm->stream);
  device_free(pm->rho_hat, pm->stream);
  device_free(pm->grad_hat, pm->stream);
  device_free(pm->tab_a, pm->stream);
  device_free(pm->tab_b, pm->stream);
  device_free(pm->cb_info, pm->stream);
  cudaStreamSynchronize(pm->stream);
}

static bool same_filter(const hrt_filter& a, const hrt_filter& b) {
  return a.deconv_p == b.deconv_p && a.smooth == b.smooth;
}

static hrt_status pm_tables(hrt_pm* pm, const hrt_filter& f, float** tab, hrt_filter* key) {
  if (*tab && same_filter(f, *key)) return HRT_OK;
  device_free(*tab, pm->stream);
  *tab = nullptr;
  HRT_TRY(filter_upload(pm->n, pm->box, f, tab, pm->stream));
  *key = f;
  return HRT_OK;
}

static KspaceCallbackInfo callback_info(const hrt_pm* pm, const float* tab, const hrt_filter& f, double pref,
                                         int n_comp) {
  KspaceCallbackInfo ci{};
  const int64_t n = pm->n;
  ci.rho_hat = pm->rho_hat;
  ci.wx = tab;
  ci.wy = tab;
  ci.wz = tab + n;
  ci.g = f.g_table;
  ci.g_nk = f.g_nk;
  ci.g_inv_dk = f.g_table ? static_cast<float>((f.g_nk - 1) / f.g_kmax) : 0.f;
  ci.n = static_cast<int>(n);
  ci.nzc = static_cast<int>(n / 2 + 1);
  int l = 0;
  while ((int64_t{1} << l) < n) ++l;
  ci.log2n = l;
  ci.n_comp = n_comp;
  ci.elems = static_cast<unsigned>(n * n * (n / 2 + 1));
  ci.magic = ((1ull << 42) + static_cast<unsigned long long>(ci.nzc) - 1) / static_cast<unsigned long long>(ci.nzc);
  ci.kf = static_cast<float>(2.0 * M_PI / pm->box);
  ci.scale = static_cast<float>(-pref / (static_cast<double>(n) * n * n));
  return ci;
}

// before_fields (optional): an event the stream waits for before the C2Rs overwrite grad / ray_grad (work on
// another stream that still reads the previous fields).  clear_rho: on the split path the x-pass sets rho to
// zero once the 2D R2C has consumed it (*cleared tells whether it did), which spares the next deposit its memset.
static hrt_status pm_solve(hrt_pm* pm, float* rho, double pref, const hrt_filter* f, float* grad,
                           const hrt_filter* fr, float* ray_grad, hrt_ctx* prof = nullptr,
                           cudaEvent_t before_fields = nullptr, bool* cleared = nullptr) {
  if (cleared) *cleared = false;
  static hrt_ctx no_profiling;
  hrt_ctx* pc = prof ? prof : &no_profiling;
  HRT_TRY(check_filter(f));
  const bool rays = pm->n_ray > 0 && ray_grad != nullptr;
  if (rays) HRT_TRY(check_filter(fr));
  HRT_TRY(pm_tables(pm, *f, &pm->tab_a, &pm->key_a));
  if (rays) HRT_TRY(pm_tables(pm, *fr, &pm->tab_b, &pm->key_b));
  pm->last_split = pm->split && !pm->fused;
  if (pm->last_split) {
    const int64_t n = pm->n;
    const size_t sp = spectrum_alloc(n);
    char* gh = static_cast<char*>(pm->grad_hat);
    {
      PhaseScope ps(pc, 3);
      HRT_CUFFT(cufftExecR2C(pm->r2c2d, rho, static_cast<cufftComplex*>(pm->rho_hat)));
    }
    auto set = [&](const float* tab, const hrt_filter& flt, int n_out, char* out) {
      XpassSet x{};
      x.wxy = tab;
      x.wz = tab + n;
      x.g = flt.g_table;
      x.g_nk = flt.g_nk;
      x.g_inv_dk = flt.g_table ? static_cast<float>((flt.g_nk - 1) / flt.g_kmax) : 0.f;
      x.n_out = n_out;
      x.out = reinterpret_cast<float2*>(out);
      return x;
    };
    const XpassSet xa = set(pm->tab_a, *f, 3, gh);
    const XpassSet xb = rays ? set(pm->tab_b, *fr, pm->n_ray, gh + 3 * sp) : XpassSet{};
    {
      PhaseScope ps(pc, 4);
      HRT_TRY(launch_xpass(pm->rho_hat, n, pm->box, pref, pm->xtw, xa, xb, pm->xerr, pm->stream,
                           cleared ? rho : nullptr, cleared ? n * n * n : 0));
      if (cleared) *cleared = true;
    }
    if (before_fields) HRT_CUDA(cudaStreamWaitEvent(pm->stream, before_fields, 0));
    PhaseScope ps(pc, 5);
    const size_t mb = static_cast<size_t>(n) * n * n;
    for (int j = 0; j < 3; ++j)
      HRT_CUFFT(cufftExecC2R(pm->c2r2d, reinterpret_cast<cufftComplex*>(gh + j * sp), grad + j * mb));
    if (rays)
      for (int j = 0; j < pm->n_ray; ++j)
        HRT_CUFFT(cufftExecC2R(pm->c2r2d, reinterpret_cast<cufftComplex*>(gh + (3 + j) * sp), ray_grad + j * mb));
    return HRT_OK;
  }
  {
    PhaseScope ps(pc, 3);
    HRT_CUFFT(cufftExecR2C(pm->r2c, rho, static_cast<cufftComplex*>(pm->rho_hat)));
  }
  const size_t sb = spectrum_bytes(pm->n);
  char* gh = static_cast<char*>(pm->grad_hat);
  const size_t mb = static_cast<size_t>(pm->n) * pm->n * pm->n;
  if (pm->fused) {
    // k-space step inside the batched C2R: the callback reads rho_hat; grad_hat is cuFFT's scratch input
    HRT_TRY(launch_set_callback_info(pm->cb_info, callback_info(pm, pm->tab_a, *f, pref, 3), pm->stream));
    if (rays) HRT_TRY(launch_set_callback_info(pm->cb_info + 1, callback_info(pm, pm->tab_b, *fr, pref, pm->n_ray),
                                               pm->stream));
    if (before_fields) HRT_CUDA(cudaStreamWaitEvent(pm->stream, before_fields, 0));
    PhaseScope ps(pc, 5);
    HRT_CUFFT(cufftExecC2R(pm->c2r_cb3, reinterpret_cast<cufftComplex*>(gh), grad));
    if (rays) HRT_CUFFT(cufftExecC2R(pm->c2r_cb2, reinterpret_cast<cufftComplex*>(gh + 3 * sb), ray_grad));
    return HRT_OK;
  }
  {
    PhaseScope ps(pc, 4);
    HRT_TRY(launch_kspace(pm->rho_hat, pm->n, pm->box, pref, pm->tab_a, f, 3, gh, rays ? pm->tab_b : nullptr, fr,
                          rays ? pm->n_ray : 0, gh + 3 * sb, pm->stream));
  }
  if (before_fields) HRT_CUDA(cudaStreamWaitEvent(pm->stream, before_fields, 0));
  PhaseScope ps(pc, 5);
  for (int j = 0; j < 3; ++j)
    HRT_CUFFT(cufftExecC2R(pm->c2r, reinterpret_cast<cufftComplex*>(gh + j * sb), grad + j * mb));
  if (rays)
    for (int j = 0; j < pm->n_ray; ++j)
      HRT_CUFFT(cufftExecC2R(pm->c2r, reinterpret_cast<cufftComplex*>(gh + (3 + j) * sb), ray_grad + j * mb));
  return HRT_OK;
}

}  // namespace hrt


namespace hrt {

static hrt_status ctx_guard(hrt_ctx* ctx) {
  if (!ctx) return fail(HRT_ERR_INVALID_ARG, "context is NULL");
  if (ctx->poisoned) return fail(HRT_ERR_STATE, "context is poisoned by an earlier CUDA error");
  return HRT_OK;
}

static hrt_status ctx_mark(hrt_ctx* ctx, hrt_status s) {
  if (s == HRT_ERR_CUDA) ctx->poisoned = true;
  return s;
}

// The opt-in check for NaN and infinity: scans the given arrays on the context's stream (after everything queued
// so far), waits within the host wait limit and returns HRT_ERR_NONFINITE if any value is not finite.  Also
// reports a kernel that gave up waiting for its own copies (the x-pass error word) as HRT_ERR_TIMEOUT.
struct ScanItem {
  const void* p;
  int64_t n;
  bool dbl;
};

static hrt_status ctx_scan(hrt_ctx* ctx, std::initializer_list<ScanItem> items, const char* what) {
  if (!ctx->check_finite) return HRT_OK;
  cudaStream_t st = ctx->stream;
  HRT_CUDA(cudaMemsetAsync(ctx->finite_flag, 0, sizeof(int), st));
  for (const ScanItem& it : items) {
    if (!it.p) continue;
    if (it.dbl) HRT_TRY(launch_nonfinite_scan(static_cast<const double*>(it.p), it.n, ctx->finite_flag, st));
    else HRT_TRY(launch_nonfinite_scan(static_cast<const float*>(it.p), it.n, ctx->finite_flag, st));
  }
  HRT_TRY(wait_stream(st, what));
  int flag = 0, xerr = 0;
  HRT_CUDA(cudaMemcpy(&flag, ctx->finite_flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (ctx->pm && ctx->pm->xerr) HRT_CUDA(cudaMemcpy(&xerr, ctx->pm->xerr, sizeof(int), cudaMemcpyDeviceToHost));
  if (xerr) return fail(HRT_ERR_TIMEOUT, "%s: a kernel gave up waiting for a tile's copy", what);
  if (flag) return fail(HRT_ERR_NONFINITE, "%s: a NaN or an infinity was found", what);
  return HRT_OK;
}

static hrt_status ctx_scan_state(hrt_ctx* ctx, const char* what) {
  const int64_t np3 = 3 * ctx->cfg.n_side * ctx->cfg.n_side * ctx->cfg.n_side, r = ctx->rays.n_rays;
  return ctx_scan(ctx,
                  {{ctx->have_particles ? ctx->disp : nullptr, np3, false},
                   {ctx->have_particles ? ctx->mom : nullptr, np3, false},
                   {ctx->rays.theta, 2 * r, true},
                   {ctx->rays.eta, 2 * r, false},
                   {ctx->rays.A, 4 * r, false},
                   {ctx->rays.B, 4 * r, false},
                   {ctx->maps, 4 * r * ctx->cfg.n_sources, false}},
                  what);
}

const int32_t* ctx_order(const hrt_ctx* ctx) { return ctx->order_cur >= 0 ? ctx->order_buf[ctx->order_cur] : nullptr; }

hrt_status ctx_particles_lattice(hrt_ctx* ctx, float* disp_out, float* mom_out) {
  const int64_t np = ctx->cfg.n_side * ctx->cfg.n_side * ctx->cfg.n_side;
  const int32_t* order = ctx_order(ctx);
  if (order) {
    if (disp_out) HRT_TRY(launch_unsort(ctx->disp, order, np, disp_out, ctx->stream));
    if (mom_out) HRT_TRY(launch_unsort(ctx->mom, order, np, mom_out, ctx->stream));
    return HRT_OK;
  }
  const size_t bytes = 3 * static_cast<size_t>(np) * sizeof(float);
  if (disp_out) HRT_CUDA(cudaMemcpyAsync(disp_out, ctx->disp, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  if (mom_out) HRT_CUDA(cudaMemcpyAsync(mom_out, ctx->mom, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return HRT_OK;
}

// Buffers of the particle sort, allocated on first use.
static hrt_status ctx_sort_alloc(hrt_ctx* ctx) {
  const hrt_config& c = ctx->cfg;
  const int64_t np = c.n_side * c.n_side * c.n_side;
  cudaStream_t st = ctx->stream;
  if (!ctx->disp_alt) {
    // All five buffers or none: they are allocated into locals and handed to the context only together, so
    // a failed allocation (which leaves the context usable) never leaves a partial set that a later sort
    // would launch on.
    float *disp_alt = nullptr, *mom_alt = nullptr;
    int32_t *order0 = nullptr, *order1 = nullptr, *scratch = nullptr;
    hrt_status s = device_alloc(reinterpret_cast<void**>(&disp_alt), 3 * np * sizeof(float), st, "sorted particles");
    if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&mom_alt), 3 * np * sizeof(float), st, "sorted particles");
    if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&order0), np * sizeof(int32_t), st, "particle order");
    if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&order1), np * sizeof(int32_t), st, "particle order");
    if (s == HRT_OK)
      s = device_alloc(reinterpret_cast<void**>(&scratch), (particle_sort_counts(c.n_mesh) + 3 * np) * sizeof(int32_t),
                       st, "sort scratch");
    if (s != HRT_OK) {
      device_free(disp_alt, st);
      device_free(mom_alt, st);
      device_free(order0, st);
      device_free(order1, st);
      device_free(scratch, st);
      return s;
    }
    ctx->disp_alt = disp_alt;
    ctx->mom_alt = mom_alt;
    ctx->order_buf[0] = order0;
    ctx->order_buf[1] = order1;
    ctx->sort_scratch = scratch;
  }
  return HRT_OK;
}

// Re-sorts the particles by cell (counting sort by z-row segments): the storage order changes, the particles
// do not.
static hrt_status ctx_sort(hrt_ctx* ctx) {
  const hrt_config& c = ctx->cfg;
  const int64_t np = c.n_side * c.n_side * c.n_side;
  cudaStream_t st = ctx->stream;
  HRT_TRY(ctx_sort_alloc(ctx));
  if (!ctx->mom_alt || !ctx->order_buf[0] || !ctx->order_buf[1] || !ctx->sort_scratch)
    return fail(HRT_ERR_STATE, "particle sort buffers are incomplete");
  const int dst = ctx->order_cur == 0 ? 1 : 0;
  // brick keys only for the tiled kick-drift-deposit: the per-particle kernel is faster on z-row order
  const bool bricks = ctx->tiled_deposit != 0 && particle_bricks_ok(c.n_mesh);
  int32_t* counts = ctx->sort_scratch;
  int32_t* keys = counts + particle_sort_counts(c.n_mesh);
  HRT_TRY(launch_particle_sort(ctx->disp, ctx->mom, ctx_order(ctx), c.n_side, c.n_mesh, c.box, ctx->disp_alt,
                               ctx->mom_alt, ctx->order_buf[dst], counts, keys, keys + np, keys + 2 * np, st, bricks));
  std::swap(ctx->disp, ctx->disp_alt);
  std::swap(ctx->mom, ctx->mom_alt);
  ctx->order_cur = dst;
  ctx->sort_bricks = bricks;
  ctx->sort_first = false;
  return HRT_OK;
}

// Back to lattice order (new particles).  Initial conditions keep it until the regular sort (lattice order is
// cell order while the displacements are small); particles given by the caller or a saved state, which may be
// clustered, are sorted at their first step.
static void ctx_lattice_order(hrt_ctx* ctx, bool evolved = false) {
  ctx->order_cur = -1;
  ctx->steps_since_sort = 0;
  ctx->sort_first = evolved;
}

hrt_filter ctx_filter(const hrt_config& c, bool ray) {
  hrt_filter f{};
  const double cell = c.box / c.n_mesh;
  f.deconv_p = ray ? c.ray_deconv_p : c.deconv_p;
  f.smooth = (ray ? c.ray_smooth_cells : c.smooth_cells) * cell;
  return f;
}

static double ctx_pref(const hrt_ctx* ctx, double a) {
  return ctx->cfg.static_mode ? ctx->cfg.static_pref : 1.5 * ctx->cfg.cosmo.omega_m / a;
}

// Gradient fields at ctx->a from the density already deposited in ctx->rho (with the learned ray table
// evaluated at ctx->a first when a correction is set).
static hrt_status ctx_solve(hrt_ctx* ctx) {
  const hrt_config& c = ctx->cfg;
  ctx->force_valid = false;
  hrt_filter f = ctx_filter(c, false), fr = ctx_filter(c, true);
  if (ctx->corr_w) {
    const double cell = c.box / c.n_mesh;
    HRT_TRY(launch_correction_inputs(ctx->corr_x, kCorrectionRows, kCorrectionKmaxCell / (kCorrectionRows - 1),
                                     ctx->a, std::log(static_cast<double>(c.n_mesh)), ctx->stream));
    HRT_TRY(launch_mlp_forward(ctx->corr_x, kCorrectionRows, ctx->corr_wb, ctx->corr_w, ctx->corr_table,
                               ctx->stream));
    fr.g_table = ctx->corr_table;
    fr.g_nk = kCorrectionRows;
    fr.g_kmax = kCorrectionKmaxCell / cell;
  } else if (ctx->ray_table) {
    fr.g_table = ctx->ray_table;
    fr.g_nk = ctx->ray_table_nk;
    fr.g_kmax = ctx->ray_table_kmax;
  }
  if (ctx->pcorr_w) {
    // the learned factor of the particle force (read by the rays too when they have no fields of their own)
    const double cell = c.box / c.n_mesh;
    HRT_TRY(launch_correction_inputs(ctx->pcorr_x, kCorrectionRows, kCorrectionKmaxCell / (kCorrectionRows - 1),
                                     ctx->a, std::log(static_cast<double>(c.n_mesh)), ctx->stream));
    HRT_TRY(launch_mlp_forward(ctx->pcorr_x, kCorrectionRows, ctx->pcorr_wb, ctx->pcorr_w, ctx->pcorr_table,
                               ctx->stream));
    f.g_table = ctx->pcorr_table;
    f.g_nk = kCorrectionRows;
    f.g_kmax = kCorrectionKmaxCell / cell;
  }
  cudaEvent_t wait = ctx->rays_pending ? ctx->ev_rays : nullptr;
  ctx->rays_pending = false;
  ctx->force_valid = false;
  ctx->rho_clear = false;
  const hrt_status s = pm_solve(ctx->pm, ctx->rho, ctx_pref(ctx, ctx->a), &f, ctx->grad, &fr, ctx->ray_grad, ctx,
                                wait, &ctx->rho_clear);
  if (s != HRT_OK) {
    // a solve that failed before its C2Rs waited for the ray step still joins it, so that whatever comes next on
    // the context stream (reads of the rays, a new ray set freeing the old buffers) runs after the ray step
    if (wait) cudaStreamWaitEvent(ctx->stream, wait, 0);
    return s;
  }
  ctx->force_valid = true;
  return HRT_OK;
}

// CIC deposit of the current particles, then the gradient fields.  Particles given by the caller are sorted by
// cell first (when sorting is on), so that the deposit runs in cell order too.
static hrt_status ctx_force(hrt_ctx* ctx) {
  const hrt_config& c = ctx->cfg;
  ctx->force_valid = false;
  if (ctx->sort_first && ctx->sort_every > 0) {
    PhaseScope ps(ctx, 7);
    HRT_TRY(ctx_sort(ctx));
    ctx->steps_since_sort = 0;
  }
  {
    PhaseScope ps(ctx, 2);
    // the density is still zero if the last solve cleared it and nothing has been deposited since
    const bool zeroed = ctx->rho_clear;
    ctx->rho_clear = false;
    HRT_TRY(launch_cic_scatter(ctx->disp, c.n_side, c.n_mesh, c.box, ctx->rho, ctx->stream, ctx_order(ctx), zeroed));
  }
  return ctx_solve(ctx);
}


hrt_ray_geom ctx_geom(const hrt_config& c, const hrt_ctx* ctx) {
  hrt_ray_geom g{};
  if (ctx && !ctx->rep_perm.empty()) {
    g.n_replicas = static_cast<int32_t>(ctx->rep_perm.size() / 3);
    g.replica_perm = ctx->rep_perm.data();
    g.replica_sign = ctx->rep_sign.data();
    g.replica_shift = ctx->rep_shift.data();
  }
  g.n = c.n_mesh;
  g.box = c.box;
  std::memcpy(g.observer, c.observer, sizeof(g.observer));
  g.samples_per_cell = c.samples_per_cell;
  g.window_lo = c.window_lo;
  g.window_hi = c.window_hi;
  return g;
}

static hrt_status ctx_ray_step(hrt_ctx* ctx, double chi_from, double chi_to, double a_ref, int32_t source,
                               cudaStream_t stream, double weight = 1.0, bool accumulate = false) {
  const hrt_config& c = ctx->cfg;
  if (source >= c.n_sources) return fail(HRT_ERR_INVALID_ARG, "source %d out of range", source);
  static thread_local RayStepParams p;
  hrt_ray_geom g = ctx_geom(c, ctx);
  // rays that fill a square image are walked in tiles (a thread-order choice; any ray set is valid)
  const int64_t w = static_cast<int64_t>(std::llround(std::sqrt(static_cast<double>(ctx->rays.n_rays))));
  if (w * w == ctx->rays.n_rays) g.image_width = w;
  HRT_TRY(build_ray_params(g, chi_from, chi_to, a_ref, c.cosmo.omega_m, p));
  set_tiles(g, ctx->rays.n_rays, p);
  p.theta32 = ctx->theta32 ? 1 : 0;
  p.map_accumulate = accumulate ? 1 : 0;
  p.map_weight = static_cast<float>(weight);
  const int64_t m = c.n_mesh * c.n_mesh * c.n_mesh;
  const float* gx = ctx->ray_grad ? ctx->ray_grad : ctx->grad;
  float* maps = source >= 0 ? ctx->maps + static_cast<int64_t>(source) * 4 * ctx->rays.n_rays : nullptr;
  if (ctx->raymesh)
    return raymesh_step(ctx->raymesh, ctx->rays, gx, gx + m, p.tiled ? ctx->grad + 2 * m : nullptr, g, chi_from,
                        chi_to, a_ref, c.cosmo.omega_m, maps, accumulate ? 1 : 0, static_cast<float>(weight), stream);
  // a tiled light cone reads all three particle gradient fields (ray_fields == 0 is checked when it is set)
  return launch_ray_step(ctx->rays, gx, gx + m, p, maps, stream, p.tiled ? ctx->grad + 2 * m : nullptr);
}

}  // namespace hrt

using namespace hrt;

extern "C" {

const char* hrt_status_string(hrt_status s) {
  switch (s) {
    case HRT_OK: return "HRT_OK";
    case HRT_ERR_INVALID_ARG: return "HRT_ERR_INVALID_ARG";
    case HRT_ERR_OOM: return "HRT_ERR_OOM";
    case HRT_ERR_CUDA: return "HRT_ERR_CUDA";
    case HRT_ERR_STATE: return "HRT_ERR_STATE";
    case HRT_ERR_NONFINITE: return "HRT_ERR_NONFINITE";
    case HRT_ERR_TIMEOUT: return "HRT_ERR_TIMEOUT";
  }
  return "HRT_ERR_UNKNOWN";
}

const char* hrt_last_error(void) { return g_err; }

hrt_status hrt_cosmo_eval(double omega_m, double a, double out[4]) {
  if (!out || !(omega_m > 0.0 && omega_m <= 1.0) || !(a > 0.0 && a <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "bad cosmology arguments");
  Cosmo c(omega_m);
  out[0] = c.E(a);
  out[1] = c.chi(a);
  out[2] = c.D1(a);
  out[3] = c.f(a);
  return HRT_OK;
}

hrt_status hrt_cosmo_time_integrals(double omega_m, double a, double b, double out[2]) {
  if (!out || !(omega_m > 0.0 && omega_m <= 1.0) || !(a > 0.0) || !(b > 0.0)) return fail(HRT_ERR_INVALID_ARG, "bad arguments");
  Cosmo c(omega_m);
  out[0] = c.kick(a, b);
  out[1] = c.drift(a, b);
  return HRT_OK;
}

hrt_status hrt_cosmo_a_of_chi(double omega_m, double chi, double* a) {
  if (!a || !(omega_m > 0.0 && omega_m <= 1.0) || !(chi >= 0.0)) return fail(HRT_ERR_INVALID_ARG, "bad arguments");
  *a = Cosmo(omega_m).a_of_chi(chi);
  return HRT_OK;
}

hrt_status hrt_cosmo_power_amplitude(double omega_m, double h, double n_s, double sigma8, double* amp) {
  if (!amp || !(omega_m > 0.0) || !(h > 0.0) || !(sigma8 > 0.0)) return fail(HRT_ERR_INVALID_ARG, "bad arguments");
  *amp = power_amplitude(omega_m, h, n_s, sigma8);
  return HRT_OK;
}

hrt_status hrt_cic_scatter_warp_aggregated(const float* disp, int64_t n_side, int64_t n, double box, float* rho,
                                           void* stream) {
  HRT_TRY(check_mesh(n, box));
  HRT_TRY(check_particles(n_side, n));
  if (!disp || !rho) return fail(HRT_ERR_INVALID_ARG, "NULL buffer");
  return launch_cic_scatter_warp(disp, n_side, n, box, rho, as_stream(stream));
}

hrt_status hrt_cic_scatter(const float* disp, int64_t n_side, int64_t n, double box, float* rho, void* stream) {
  HRT_TRY(check_mesh(n, box));
  HRT_TRY(check_particles(n_side, n));
  if (!disp || !rho) return fail(HRT_ERR_INVALID_ARG, "NULL buffer");
  return launch_cic_scatter(disp, n_side, n, box, rho, as_stream(stream));
}

hrt_status hrt_particle_kick_drift(const float* grad, int64_t n, double box, int64_t n_side, float* disp,
                                   float* mom, double kick, double drift, void* stream) {
  HRT_TRY(check_mesh(n, box));
  HRT_TRY(check_particles(n_side, n));
  if (!grad || !disp || !mom) return fail(HRT_ERR_INVALID_ARG, "NULL buffer");
  if (!std::isfinite(kick) || !std::isfinite(drift)) return fail(HRT_ERR_INVALID_ARG, "non-finite coefficient");
  return launch_kick_drift(grad, n, box, n_side, disp, mom, kick, drift, as_stream(stream));
}

hrt_status hrt_particle_kick_drift_deposit(const float* grad, int64_t n, double box, int64_t n_side, float* disp,
                                           float* mom, double kick, double drift, float* rho, void* stream) {
  HRT_TRY(check_mesh(n, box));
  HRT_TRY(check_particles(n_side, n));
  if (!grad || !disp || !mom || !rho) return fail(HRT_ERR_INVALID_ARG, "NULL buffer");
  if (!std::isfinite(kick) || !std::isfinite(drift)) return fail(HRT_ERR_INVALID_ARG, "non-finite coefficient");
  return launch_kick_drift(grad, n, box, n_side, disp, mom, kick, drift, as_stream(stream), rho);
}

hrt_status hrt_particle_kick_drift_deposit_bricks(const float* grad, int64_t n, double box, int64_t n_side,
                                                  float* disp, float* mom, const int32_t* order,
                                                  const int32_t* key_start, double kick, double drift, float* rho,
                                                  void* stream) {
  HRT_TRY(check_mesh(n, box));
  HRT_TRY(check_particles(n_side, n));
  if (!particle_bricks_ok(n)) return fail(HRT_ERR_INVALID_ARG, "mesh side must be a multiple of 32 up to 1024");
  if (!grad || !disp || !mom || !rho || !order || !key_start) return fail(HRT_ERR_INVALID_ARG, "NULL buffer");
  if (!std::isfinite(kick) || !std::isfinite(drift)) return fail(HRT_ERR_INVALID_ARG, "non-finite coefficient");
  return launch_kick_drift_tiled(grad, n, box, n_side, disp, mom, kick, drift, rho, order, key_start,
                                 as_stream(stream));
}

hrt_status hrt_kspace_gradient(const void* rho_hat, int64_t n, double box, double pref, const hrt_filter* f,
                               int32_t n_out, void* out, const hrt_filter* f2, int32_t n_second, void* second,
                               void* stream) {
  HRT_TRY(check_mesh(n, box));
  HRT_TRY(check_filter(f));
  if (!rho_hat || !out || n_out < 1 || n_out > 3) return fail(HRT_ERR_INVALID_ARG, "bad primary output");
  if (second && (n_second < 1 || n_second > 3)) return fail(HRT_ERR_INVALID_ARG, "bad second output count");
  if (second) HRT_TRY(check_filter(f2));
  if (!std::isfinite(pref)) return fail(HRT_ERR_INVALID_ARG, "non-finite prefactor");
  cudaStream_t s = as_stream(stream);
  float* ta = nullptr;
  float* tb = nullptr;
  hrt_status st = filter_upload(n, box, *f, &ta, s);
  if (st == HRT_OK && second) st = filter_upload(n, box, *f2, &tb, s);
  if (st == HRT_OK)
    st = launch_kspace(rho_hat, n, box, pref, ta, f, n_out, out, tb, f2, second ? n_second : 0, second, s);
  device_free(ta, s);
  device_free(tb, s);
  return st;
}

hrt_status hrt_pm_create(int64_t n, double box, int32_t n_ray_fields, void* stream, hrt_pm** out) {
  if (!out) return fail(HRT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  HRT_TRY(check_mesh(n, box));
  if (n_ray_fields != 0 && n_ray_fields != 2) return fail(HRT_ERR_INVALID_ARG, "n_ray_fields must be 0 or 2");
  hrt_pm* pm = new (std::nothrow) hrt_pm();
  if (!pm) return fail(HRT_ERR_OOM, "host allocation");
  hrt_status s = pm_make(n, box, n_ray_fields, as_stream(stream), pm);
  if (s != HRT_OK) {
    pm_release(pm);
    delete pm;
    return s;
  }
  *out = pm;
  return HRT_OK;
}

hrt_status hrt_pm_destroy(hrt_pm* pm) {
  if (!pm) return HRT_OK;
  pm_release(pm);
  delete pm;
  return HRT_OK;
}

hrt_status hrt_pm_set_fused(hrt_pm* pm, int32_t on) {
  if (!pm) return fail(HRT_ERR_INVALID_ARG, "pm is NULL");
  if (on) HRT_TRY(pm_build_fused(pm));
  pm->fused = on != 0;
  return HRT_OK;
}

hrt_status hrt_pm_set_split(hrt_pm* pm, int32_t on) {
  if (!pm) return fail(HRT_ERR_INVALID_ARG, "pm is NULL");
  if (on && !pm->have_r2c2d) return fail(HRT_ERR_INVALID_ARG, "the split path needs a mesh side of 256, 512 or 1024");
  pm->split = on != 0;
  return HRT_OK;
}

hrt_status hrt_pm_solve(hrt_pm* pm, float* rho, double pref, const hrt_filter* f, float* grad,
                        const hrt_filter* f_ray, float* ray_grad) {
  if (!pm || !rho || !grad) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (ray_grad && pm->n_ray == 0) return fail(HRT_ERR_INVALID_ARG, "PM object has no ray fields");
  return pm_solve(pm, rho, pref, f, grad, f_ray, ray_grad);
}

hrt_status hrt_rays_init(const hrt_rays* rays, const double* theta0, void* stream) {
  HRT_TRY(check_rays(rays));
  if (rays->n_rays > 0 && !theta0) return fail(HRT_ERR_INVALID_ARG, "theta0 is NULL");
  return launch_rays_init(*rays, theta0, as_stream(stream));
}

hrt_status hrt_ray_step(const hrt_rays* rays, const float* grad_x, const float* grad_y, const hrt_ray_geom* geom,
                        double chi_from, double chi_to, double a_ref, double omega_m, float* maps, void* stream) {
  HRT_TRY(check_rays(rays));
  if (!geom || !grad_x || !grad_y) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (!std::isfinite(chi_from) || !std::isfinite(chi_to) || !(a_ref >= 0.0) || a_ref > 1.0)
    return fail(HRT_ERR_INVALID_ARG, "bad step range");
  if (a_ref > 0.0 && !(omega_m > 0.0 && omega_m <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "bad omega_m");
  if (geom->n_replicas > 0)
    return fail(HRT_ERR_INVALID_ARG, "a tiled light cone needs all three gradient components: hrt_ray_step_tiled");
  static thread_local RayStepParams p;
  HRT_TRY(build_ray_params(*geom, chi_from, chi_to, a_ref, omega_m, p));
  set_tiles(*geom, rays->n_rays, p);
  return launch_ray_step(*rays, grad_x, grad_y, p, maps, as_stream(stream));
}

hrt_status hrt_ray_step_tiled(const hrt_rays* rays, const float* grad_x, const float* grad_y, const float* grad_z,
                              const hrt_ray_geom* geom, double chi_from, double chi_to, double a_ref, double omega_m,
                              float* maps, void* stream) {
  HRT_TRY(check_rays(rays));
  if (!geom || !grad_x || !grad_y || !grad_z) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (geom->n_replicas < 1) return fail(HRT_ERR_INVALID_ARG, "tiling needs at least one replica");
  if (!std::isfinite(chi_from) || !std::isfinite(chi_to) || !(a_ref >= 0.0) || a_ref > 1.0)
    return fail(HRT_ERR_INVALID_ARG, "bad step range");
  if (a_ref > 0.0 && !(omega_m > 0.0 && omega_m <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "bad omega_m");
  static thread_local RayStepParams p;
  HRT_TRY(build_ray_params(*geom, chi_from, chi_to, a_ref, omega_m, p));
  set_tiles(*geom, rays->n_rays, p);
  return launch_ray_step(*rays, grad_x, grad_y, p, maps, as_stream(stream), grad_z);
}

hrt_status hrt_ray_drift_free(const hrt_rays* rays, double chi_from, double chi_to, void* stream) {
  HRT_TRY(check_rays(rays));
  if (!(chi_from > 0.0) || !(chi_to > 0.0)) return fail(HRT_ERR_INVALID_ARG, "free drift needs chi > 0");
  return launch_ray_drift_free(*rays, (1.0 / chi_from - 1.0 / chi_to) / kCLight, as_stream(stream));
}

hrt_status hrt_ray_readout(const hrt_rays* rays, float* maps, void* stream) {
  HRT_TRY(check_rays(rays));
  if (!maps && rays->n_rays > 0) return fail(HRT_ERR_INVALID_ARG, "maps is NULL");
  return launch_ray_readout(*rays, maps, as_stream(stream));
}

hrt_status hrt_kappa_power(const float* kappa, int64_t m, double dtheta, int32_t nbins, double ell_min,
                           double ell_max, double* ell_host, double* p_host, int64_t* count_host, void* stream) {
  if (!kappa || !ell_host || !p_host || !count_host) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (m < 2 || m % 2 || m > 16384 || nbins < 1 || nbins > 256 || !(dtheta > 0.0) || !(ell_min > 0.0) ||
      !(ell_max > ell_min))
    return fail(HRT_ERR_INVALID_ARG, "bad power-spectrum arguments");
  cudaStream_t s = as_stream(stream);
  // first the work already queued on the stream (e.g. the steps that wrote the map), within the host wait limit;
  // on expiry nothing has been enqueued and the call can be repeated
  HRT_TRY(wait_stream(s, "hrt_kappa_power"));
  cufftHandle plan;
  HRT_CUFFT(cufftPlan2d(&plan, static_cast<int>(m), static_cast<int>(m), CUFFT_R2C));
  void* spec = nullptr;
  double* sums = nullptr;
  hrt_status st = cufft_status(cufftSetStream(plan, s), "cufftSetStream");
  if (st == HRT_OK) st = device_alloc(&spec, static_cast<size_t>(m) * (m / 2 + 1) * sizeof(float2), s, "kappa spectrum");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&sums), 3 * nbins * sizeof(double), s, "power bins");
  if (st == HRT_OK)
    st = cufft_status(cufftExecR2C(plan, const_cast<float*>(kappa), static_cast<cufftComplex*>(spec)), "cufftExecR2C");
  if (st == HRT_OK) st = launch_power_bin(spec, m, dtheta, nbins, ell_min, ell_max, sums, s);
  std::vector<double> h(3 * nbins);
  if (st == HRT_OK) st = cuda_status(cudaMemcpyAsync(h.data(), sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "power bins copy");
  if (st == HRT_OK) st = cuda_status(cudaStreamSynchronize(s), "power bins sync");
  device_free(spec, s);
  device_free(sums, s);
  cudaStreamSynchronize(s);
  cufftDestroy(plan);
  if (st != HRT_OK) return st;
  for (int b = 0; b < nbins; ++b) {
    double cnt = h[2 * nbins + b];
    count_host[b] = static_cast<int64_t>(std::llround(cnt));
    p_host[b] = cnt > 0 ? h[b] / cnt : 0.0;
    ell_host[b] = cnt > 0 ? h[nbins + b] / cnt : 0.0;
  }
  return HRT_OK;
}

static std::vector<double> ic_table64(int64_t n, double box, const hrt_cosmology* cosmo, double a_init,
                                      double* ratio) {
  Cosmo c(cosmo->omega_m);
  const double amp = power_amplitude(cosmo->omega_m, cosmo->h, cosmo->n_s, cosmo->sigma8);
  const double d1 = c.D1(a_init);
  if (ratio) *ratio = a_init * a_init * c.E(a_init) * c.f(a_init);
  const double kf = 2.0 * M_PI / box, v_cell = std::pow(box / n, 3);
  const int64_t max_n2 = 3 * (n / 2) * (n / 2);
  std::vector<double> table(max_n2 + 1, 0.0);
  for (int64_t i = 1; i <= max_n2; ++i) {
    double k = kf * std::sqrt(static_cast<double>(i));
    double pk = amp * std::pow(k, cosmo->n_s) * std::pow(bbks_transfer(k / (cosmo->omega_m * cosmo->h)), 2);
    table[i] = d1 * std::sqrt(pk / v_cell) / (k * k) / (static_cast<double>(n) * n * n);
  }
  return table;
}

hrt_status hrt_ic_zeldovich(const float* noise, int64_t n_side, double box, const hrt_cosmology* cosmo,
                            double a_init, float* disp, float* mom, void* stream) {
  HRT_TRY(check_mesh(n_side, box));
  if (!noise || !cosmo || !disp || !mom) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (!(a_init > 0.0 && a_init <= 1.0) || !(cosmo->omega_m > 0.0 && cosmo->omega_m <= 1.0))
    return fail(HRT_ERR_INVALID_ARG, "bad cosmology");
  cudaStream_t s = as_stream(stream);
  const int64_t n = n_side;
  double ratio = 0.0;
  const std::vector<double> t64 = ic_table64(n, box, cosmo, a_init, &ratio);
  std::vector<float> table(t64.begin(), t64.end());
  hrt_pm tmp;
  hrt_status st = pm_make(n, box, 0, s, &tmp);
  float* tab = nullptr;
  if (st == HRT_OK) st = upload(table, &tab, s, "IC table");
  if (st == HRT_OK)
    st = cufft_status(cufftExecR2C(tmp.r2c, const_cast<float*>(noise), static_cast<cufftComplex*>(tmp.rho_hat)), "IC R2C");
  if (st == HRT_OK) st = launch_ic_kspace(tmp.rho_hat, n, box, tab, tmp.grad_hat, s);
  const size_t sb = spectrum_bytes(n);
  const int64_t np = n * n * n;
  for (int j = 0; j < 3 && st == HRT_OK; ++j)
    st = cufft_status(cufftExecC2R(tmp.c2r, reinterpret_cast<cufftComplex*>(static_cast<char*>(tmp.grad_hat) + j * sb),
                                   disp + j * np), "IC C2R");
  if (st == HRT_OK) st = launch_scale_copy(disp, mom, ratio, 3 * np, s);
  device_free(tab, s);
  pm_release(&tmp);
  return st;
}

hrt_status hrt_ic_2lpt(const float* noise, int64_t n_side, double box, const hrt_cosmology* cosmo, double a_init,
                       float* disp, float* mom, void* stream) {
  HRT_TRY(check_mesh(n_side, box));
  if (!noise || !cosmo || !disp || !mom) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (!(a_init > 0.0 && a_init <= 1.0) || !(cosmo->omega_m > 0.0 && cosmo->omega_m <= 1.0))
    return fail(HRT_ERR_INVALID_ARG, "bad cosmology");
  cudaStream_t s = as_stream(stream);
  const int64_t n = n_side, np = n * n * n;
  // growth factors: first order from the host cosmology, second order by the fits exact for Omega_m = 1
  Cosmo c(cosmo->omega_m);
  const double d1 = c.D1(a_init), f1 = c.f(a_init), e = c.E(a_init);
  const double om_a = cosmo->omega_m / (a_init * a_init * a_init * e * e);
  const double d2 = -3.0 / 7.0 * d1 * d1 * std::pow(om_a, -1.0 / 143.0);
  const double f2 = 2.0 * std::pow(om_a, 6.0 / 11.0);
  const double pfac = a_init * a_init * e;
  const std::vector<double> t64 = ic_table64(n, box, cosmo, a_init, nullptr);
  std::vector<float> table(t64.size());
  for (size_t i = 0; i < t64.size(); ++i) table[i] = static_cast<float>(t64[i] / d1);  // unit growth
  hrt_pm tmp;
  hrt_status st = pm_make(n, box, 0, s, &tmp);
  float* tab = nullptr;
  float* h = nullptr;  // six real fields: the Hessian of phi1, then the source (field 0) and Psi2 (fields 1..3)
  if (st == HRT_OK) st = upload(table, &tab, s, "IC table");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&h), 6 * np * sizeof(float), s, "2LPT fields");
  const size_t sb = spectrum_bytes(n);
  char* gh = static_cast<char*>(tmp.grad_hat);
  auto c2r3 = [&](float* out) {
    for (int j = 0; j < 3 && st == HRT_OK; ++j)
      st = cufft_status(cufftExecC2R(tmp.c2r, reinterpret_cast<cufftComplex*>(gh + j * sb), out + j * np), "2LPT C2R");
  };
  if (st == HRT_OK)
    st = cufft_status(cufftExecR2C(tmp.r2c, const_cast<float*>(noise), static_cast<cufftComplex*>(tmp.rho_hat)), "IC R2C");
  // Psi1 at unit growth into disp
  if (st == HRT_OK) st = launch_ic_kspace(tmp.rho_hat, n, box, tab, tmp.grad_hat, s);
  c2r3(disp);
  // Hessian of phi1 (two sets of three), then the source in field 0
  for (int set = 0; set < 2 && st == HRT_OK; ++set) {
    st = launch_ic_hessian(tmp.rho_hat, n, box, tab, set, tmp.grad_hat, s);
    c2r3(h + 3 * set * np);
  }
  if (st == HRT_OK) st = launch_lpt2_source(h, np, h, s);
  if (st == HRT_OK) st = cufft_status(cufftExecR2C(tmp.r2c, h, static_cast<cufftComplex*>(tmp.rho_hat)), "2LPT R2C");
  if (st == HRT_OK) st = launch_lpt2_kspace(tmp.rho_hat, n, box, tmp.grad_hat, s);
  c2r3(h + np);
  if (st == HRT_OK)
    st = launch_lpt_combine(disp, h + np, 3 * np, d1, d2, pfac * f1 * d1, pfac * f2 * d2, disp, mom, s);
  device_free(tab, s);
  device_free(h, s);
  pm_release(&tmp);
  return st;
}

// ---------------------------------------------------------------------------------------------------------
// Adjoints
// ---------------------------------------------------------------------------------------------------------
hrt_status hrt_cic_scatter_adjoint(const float* rho_bar, const float* disp, int64_t n_side, int64_t n, double box,
                                   float* disp_bar, void* stream) {
  HRT_TRY(check_mesh(n, box));
  HRT_TRY(check_particles(n_side, n));
  if (!rho_bar || !disp || !disp_bar) return fail(HRT_ERR_INVALID_ARG, "NULL buffer");
  return launch_deposit_adjoint(rho_bar, disp, n_side, n, box, disp_bar, as_stream(stream));
}

hrt_status hrt_particle_kick_drift_adjoint(const float* grad, int64_t n, double box, int64_t n_side, const float* disp,
                                           const float* mom, double kick, double drift, const float* rho_bar,
                                           float* disp_bar, float* mom_bar, float* grad_bar, double* coef_bar,
                                           void* stream) {
  HRT_TRY(check_mesh(n, box));
  HRT_TRY(check_particles(n_side, n));
  if (!grad || !disp || !mom || !disp_bar || !mom_bar || !grad_bar || !coef_bar)
    return fail(HRT_ERR_INVALID_ARG, "NULL buffer");
  return launch_kick_drift_adjoint(grad, n, box, n_side, disp, mom, kick, drift, rho_bar, disp_bar, mom_bar, grad_bar,
                                   coef_bar, as_stream(stream));
}

hrt_status hrt_pm_solve_adjoint(hrt_pm* pm, float* grad_bar, double pref, const hrt_filter* f, float* ray_grad_bar,
                                const hrt_filter* f_ray, float* rho_bar) {
  if (!pm || !grad_bar || !rho_bar) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  HRT_TRY(check_filter(f));
  if (ray_grad_bar && (pm->n_ray == 0 || !f_ray)) return fail(HRT_ERR_INVALID_ARG, "PM object has no ray fields");
  if (ray_grad_bar) HRT_TRY(check_filter(f_ray));
  HRT_TRY(pm_tables(pm, *f, &pm->tab_a, &pm->key_a));
  if (ray_grad_bar) HRT_TRY(pm_tables(pm, *f_ray, &pm->tab_b, &pm->key_b));
  const size_t sb = spectrum_bytes(pm->n), mb = static_cast<size_t>(pm->n) * pm->n * pm->n;
  char* gh = static_cast<char*>(pm->grad_hat);
  for (int j = 0; j < 3; ++j)
    HRT_CUFFT(cufftExecR2C(pm->r2c, grad_bar + j * mb, reinterpret_cast<cufftComplex*>(gh + j * sb)));
  HRT_TRY(launch_kspace_adjoint(gh, 3, pm->n, pm->box, pref, pm->tab_a, f, pm->rho_hat, false, pm->stream));
  if (ray_grad_bar) {
    for (int j = 0; j < pm->n_ray; ++j)
      HRT_CUFFT(cufftExecR2C(pm->r2c, ray_grad_bar + j * mb, reinterpret_cast<cufftComplex*>(gh + (3 + j) * sb)));
    HRT_TRY(launch_kspace_adjoint(gh + 3 * sb, pm->n_ray, pm->n, pm->box, pref, pm->tab_b, f_ray, pm->rho_hat, true,
                                  pm->stream));
  }
  HRT_CUFFT(cufftExecC2R(pm->c2r, static_cast<cufftComplex*>(pm->rho_hat), rho_bar));
  return HRT_OK;
}

hrt_status hrt_ray_step_adjoint(const hrt_rays* rays, const float* grad_x, const float* grad_y, const hrt_ray_geom* geom,
                                double chi_from, double chi_to, double a_ref, double omega_m, const hrt_rays* bar,
                                float* gx_bar, float* gy_bar, double* node_bar, double* drift_bar, void* stream) {
  HRT_TRY(check_rays(rays));
  HRT_TRY(check_rays(bar));
  if (!geom || !grad_x || !grad_y || !gx_bar || !gy_bar || !node_bar || !drift_bar)
    return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (bar->n_rays != rays->n_rays) return fail(HRT_ERR_INVALID_ARG, "ray counts differ");
  if (geom->n_replicas > 0) return fail(HRT_ERR_INVALID_ARG, "a tiled light cone needs hrt_ray_step_tiled_adjoint");
  static thread_local RayStepParams p;
  HRT_TRY(build_ray_params(*geom, chi_from, chi_to, a_ref, omega_m, p));
  set_tiles(*geom, rays->n_rays, p);
  return launch_ray_step_adjoint(*rays, grad_x, grad_y, p, *bar, gx_bar, gy_bar, node_bar, drift_bar, as_stream(stream));
}

hrt_status hrt_ray_step_tiled_adjoint(const hrt_rays* rays, const float* grad_x, const float* grad_y,
                                      const float* grad_z, const hrt_ray_geom* geom, double chi_from, double chi_to,
                                      double a_ref, double omega_m, const hrt_rays* bar, float* gx_bar, float* gy_bar,
                                      float* gz_bar, double* node_bar, double* drift_bar, void* stream) {
  HRT_TRY(check_rays(rays));
  HRT_TRY(check_rays(bar));
  if (!geom || !grad_x || !grad_y || !grad_z || !gx_bar || !gy_bar || !gz_bar || !node_bar || !drift_bar)
    return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (bar->n_rays != rays->n_rays) return fail(HRT_ERR_INVALID_ARG, "ray counts differ");
  if (geom->n_replicas < 1) return fail(HRT_ERR_INVALID_ARG, "the tiled adjoint needs n_replicas >= 1");
  static thread_local RayStepParams p;
  HRT_TRY(build_ray_params(*geom, chi_from, chi_to, a_ref, omega_m, p));
  set_tiles(*geom, rays->n_rays, p);
  return launch_ray_step_adjoint(*rays, grad_x, grad_y, p, *bar, gx_bar, gy_bar, node_bar, drift_bar, as_stream(stream),
                                 grad_z, gz_bar);
}

hrt_status hrt_ray_step_coefficients(const hrt_ray_geom* geom, double chi_from, double chi_to, double a_ref,
                                     double omega_m, int32_t* n1, int32_t* n2, double* cw, double* cwr, double* chi,
                                     double* drift) {
  if (!geom || !n1 || !n2 || !cw || !cwr || !chi || !drift) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  static thread_local RayStepParams p;
  HRT_TRY(build_ray_params(*geom, chi_from, chi_to, a_ref, omega_m, p, cw, cwr, chi));
  *n1 = p.n1;
  *n2 = p.n2;
  *drift = p.drift_d;
  return HRT_OK;
}

hrt_status hrt_kappa_power_adjoint(const float* kappa, int64_t m, double dtheta, int32_t nbins, double ell_min,
                                   double ell_max, const double* dl_dp, float* kappa_bar, void* stream) {
  if (!kappa || !dl_dp || !kappa_bar) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (m < 2 || m % 2 || m > 16384 || nbins < 1 || nbins > 256 || !(dtheta > 0.0) || !(ell_min > 0.0) ||
      !(ell_max > ell_min))
    return fail(HRT_ERR_INVALID_ARG, "bad power-spectrum arguments");
  cudaStream_t s = as_stream(stream);
  cufftHandle fwd, inv;
  HRT_CUFFT(cufftPlan2d(&fwd, static_cast<int>(m), static_cast<int>(m), CUFFT_R2C));
  hrt_status st = cufft_status(cufftPlan2d(&inv, static_cast<int>(m), static_cast<int>(m), CUFFT_C2R), "plan C2R");
  if (st != HRT_OK) {
    cufftDestroy(fwd);
    return st;
  }
  void* spec = nullptr;
  double* sums = nullptr;
  double* wbin = nullptr;
  st = cufft_status(cufftSetStream(fwd, s), "cufftSetStream");
  if (st == HRT_OK) st = cufft_status(cufftSetStream(inv, s), "cufftSetStream");
  if (st == HRT_OK) st = device_alloc(&spec, static_cast<size_t>(m) * (m / 2 + 1) * sizeof(float2), s, "spectrum");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&sums), 3 * nbins * sizeof(double), s, "bins");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&wbin), nbins * sizeof(double), s, "bin weights");
  if (st == HRT_OK)
    st = cufft_status(cufftExecR2C(fwd, const_cast<float*>(kappa), static_cast<cufftComplex*>(spec)), "R2C");
  if (st == HRT_OK) st = launch_power_bin(spec, m, dtheta, nbins, ell_min, ell_max, sums, s);
  std::vector<double> h(3 * nbins), w(nbins, 0.0);
  if (st == HRT_OK) st = cuda_status(cudaMemcpyAsync(h.data(), sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "bins");
  if (st == HRT_OK) st = cuda_status(cudaStreamSynchronize(s), "sync");
  if (st == HRT_OK) {
    const double theta_field = m * dtheta;
    const double c = std::pow(dtheta, 4) / (theta_field * theta_field);
    for (int b = 0; b < nbins; ++b) {
      const double cnt = h[2 * nbins + b];
      w[b] = cnt > 0 ? 2.0 * c * dl_dp[b] / cnt : 0.0;
    }
    st = cuda_status(cudaMemcpyAsync(wbin, w.data(), nbins * sizeof(double), cudaMemcpyHostToDevice, s), "weights");
  }
  if (st == HRT_OK) st = launch_power_adjoint_weight(spec, m, dtheta, nbins, ell_min, ell_max, wbin, s);
  if (st == HRT_OK)
    st = cufft_status(cufftExecC2R(inv, static_cast<cufftComplex*>(spec), kappa_bar), "C2R");
  if (st == HRT_OK) st = cuda_status(cudaStreamSynchronize(s), "sync");
  device_free(spec, s);
  device_free(sums, s);
  device_free(wbin, s);
  cudaStreamSynchronize(s);
  cufftDestroy(fwd);
  cufftDestroy(inv);
  return st;
}

hrt_status hrt_ic_table(int64_t n_side, double box, const hrt_cosmology* cosmo, double a_init, double* table_host,
                        double* ratio_host) {
  HRT_TRY(check_mesh(n_side, box));
  if (!cosmo || !table_host || !ratio_host) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  const std::vector<double> t = ic_table64(n_side, box, cosmo, a_init, ratio_host);
  std::memcpy(table_host, t.data(), t.size() * sizeof(double));
  return HRT_OK;
}

// Growth factors of the 2LPT combine (R21): disp = d1 Psi1 + d2 Psi2, mom = c1 Psi1 + c2 Psi2.
static void lpt2_coefficients(const hrt_cosmology& cosmo, double a_init, double& d1, double& d2, double& c1, double& c2) {
  Cosmo c(cosmo.omega_m);
  d1 = c.D1(a_init);
  const double f1 = c.f(a_init), e = c.E(a_init);
  const double om_a = cosmo.omega_m / (a_init * a_init * a_init * e * e);
  d2 = -3.0 / 7.0 * d1 * d1 * std::pow(om_a, -1.0 / 143.0);
  const double f2 = 2.0 * std::pow(om_a, 6.0 / 11.0);
  const double pfac = a_init * a_init * e;
  c1 = pfac * f1 * d1;
  c2 = pfac * f2 * d2;
}

hrt_status hrt_ic_2lpt_coefficients(const hrt_cosmology* cosmo, double a_init, double* out_host) {
  if (!cosmo || !out_host || !(a_init > 0.0 && a_init <= 1.0) || !(cosmo->omega_m > 0.0 && cosmo->omega_m <= 1.0))
    return fail(HRT_ERR_INVALID_ARG, "bad arguments");
  lpt2_coefficients(*cosmo, a_init, out_host[0], out_host[1], out_host[2], out_host[3]);
  return HRT_OK;
}

hrt_status hrt_ic_2lpt_adjoint(const float* noise, int64_t n_side, double box, const hrt_cosmology* cosmo,
                               double a_init, const float* disp_bar, const float* mom_bar, float* noise_bar,
                               double* table_bar_host, double* coef_bar_host, void* stream) {
  HRT_TRY(check_mesh(n_side, box));
  if (!noise || !cosmo || !disp_bar || !mom_bar || !noise_bar) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (!(a_init > 0.0 && a_init <= 1.0) || !(cosmo->omega_m > 0.0 && cosmo->omega_m <= 1.0))
    return fail(HRT_ERR_INVALID_ARG, "bad cosmology");
  cudaStream_t s = as_stream(stream);
  const int64_t n = n_side, np = n * n * n;
  double d1, d2, c1, c2;
  lpt2_coefficients(*cosmo, a_init, d1, d2, c1, c2);
  const std::vector<double> t64 = ic_table64(n, box, cosmo, a_init, nullptr);
  std::vector<float> table(t64.size());
  for (size_t i = 0; i < t64.size(); ++i) table[i] = static_cast<float>(t64[i] / d1);  // unit growth, as the forward
  const size_t nt = table.size();
  hrt_pm tmp;
  hrt_status st = pm_make(n, box, 0, s, &tmp);
  float *tab = nullptr, *psi1 = nullptr, *psi2 = nullptr, *h = nullptr, *sf = nullptr;
  void *w_hat = nullptr, *acc = nullptr;
  double* dbuf = nullptr;  // [0..3] combine coefficient cotangents, [4..] table cotangent
  if (st == HRT_OK) st = upload(table, &tab, s, "IC table");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&psi1), 3 * np * sizeof(float), s, "Psi1");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&psi2), 3 * np * sizeof(float), s, "Psi2");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&h), 6 * np * sizeof(float), s, "Hessian");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&sf), np * sizeof(float), s, "source");
  const size_t sb = spectrum_bytes(n);
  if (st == HRT_OK) st = device_alloc(&w_hat, sb, s, "noise spectrum");
  if (st == HRT_OK) st = device_alloc(&acc, sb, s, "noise_bar spectrum");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&dbuf), (4 + nt) * sizeof(double), s, "cotangents");
  if (st == HRT_OK) st = cuda_status(cudaMemsetAsync(dbuf, 0, (4 + nt) * sizeof(double), s), "memset");
  char* gh = static_cast<char*>(tmp.grad_hat);
  auto c2r3 = [&](float* out) {
    for (int j = 0; j < 3 && st == HRT_OK; ++j)
      st = cufft_status(cufftExecC2R(tmp.c2r, reinterpret_cast<cufftComplex*>(gh + j * sb), out + j * np), "2LPT C2R");
  };
  auto r2c3 = [&](const float* in) {
    for (int j = 0; j < 3 && st == HRT_OK; ++j)
      st = cufft_status(cufftExecR2C(tmp.r2c, const_cast<float*>(in + j * np), reinterpret_cast<cufftComplex*>(gh + j * sb)),
                        "2LPT adj R2C");
  };
  // forward recompute: Psi1, the Hessian, the source and Psi2 at unit growth
  if (st == HRT_OK) st = cufft_status(cufftExecR2C(tmp.r2c, const_cast<float*>(noise), static_cast<cufftComplex*>(w_hat)), "IC R2C");
  if (st == HRT_OK) st = launch_ic_kspace(w_hat, n, box, tab, tmp.grad_hat, s);
  c2r3(psi1);
  for (int set = 0; set < 2 && st == HRT_OK; ++set) {
    st = launch_ic_hessian(w_hat, n, box, tab, set, tmp.grad_hat, s);
    c2r3(h + 3 * set * np);
  }
  if (st == HRT_OK) st = launch_lpt2_source(h, np, sf, s);
  if (st == HRT_OK) st = cufft_status(cufftExecR2C(tmp.r2c, sf, static_cast<cufftComplex*>(tmp.rho_hat)), "2LPT R2C");
  if (st == HRT_OK) st = launch_lpt2_kspace(tmp.rho_hat, n, box, tmp.grad_hat, s);
  c2r3(psi2);
  // combine coefficients: d(disp, mom)/d(d1, d2, c1, c2)
  if (st == HRT_OK) st = launch_dot(disp_bar, psi1, 3 * np, dbuf, s);
  if (st == HRT_OK) st = launch_dot(disp_bar, psi2, 3 * np, dbuf + 1, s);
  if (st == HRT_OK) st = launch_dot(mom_bar, psi1, 3 * np, dbuf + 2, s);
  if (st == HRT_OK) st = launch_dot(mom_bar, psi2, 3 * np, dbuf + 3, s);
  // Psi1_bar = d1 disp_bar + c1 mom_bar, Psi2_bar = d2 disp_bar + c2 mom_bar (over the forward fields)
  if (st == HRT_OK) st = launch_lpt_combine(disp_bar, mom_bar, 3 * np, d1, c1, d2, c2, psi1, psi2, s);
  // Psi1 part of the noise cotangent (the Zel'dovich transpose at unit growth)
  r2c3(psi1);
  if (st == HRT_OK) st = launch_ic_adjoint(tmp.grad_hat, w_hat, n, box, tab, acc, table_bar_host ? dbuf + 4 : nullptr, s);
  // Psi2 -> source cotangent -> Hessian cotangents (in place) -> noise cotangent
  r2c3(psi2);
  if (st == HRT_OK) st = launch_lpt2_kspace_adjoint(tmp.grad_hat, n, box, tmp.rho_hat, s);
  if (st == HRT_OK) st = cufft_status(cufftExecC2R(tmp.c2r, static_cast<cufftComplex*>(tmp.rho_hat), sf), "2LPT adj C2R");
  if (st == HRT_OK) st = launch_lpt2_source_adjoint(h, sf, np, s);
  for (int set = 0; set < 2 && st == HRT_OK; ++set) {
    r2c3(h + 3 * set * np);
    if (st == HRT_OK)
      st = launch_ic_hessian_adjoint(tmp.grad_hat, w_hat, n, box, tab, set, acc, table_bar_host ? dbuf + 4 : nullptr, s);
  }
  if (st == HRT_OK) st = cufft_status(cufftExecC2R(tmp.c2r, static_cast<cufftComplex*>(acc), noise_bar), "IC adj C2R");
  std::vector<double> hb(4 + nt);
  if (st == HRT_OK) st = cuda_status(cudaMemcpyAsync(hb.data(), dbuf, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
  if (st == HRT_OK) st = cuda_status(cudaStreamSynchronize(s), "sync");
  device_free(tab, s);
  device_free(psi1, s);
  device_free(psi2, s);
  device_free(h, s);
  device_free(sf, s);
  device_free(w_hat, s);
  device_free(acc, s);
  device_free(dbuf, s);
  pm_release(&tmp);
  if (st != HRT_OK) return st;
  if (coef_bar_host)
    for (int k = 0; k < 4; ++k) coef_bar_host[k] = hb[k];
  if (table_bar_host)
    for (size_t i = 0; i < nt; ++i) table_bar_host[i] = hb[4 + i];
  return HRT_OK;
}

hrt_status hrt_ic_zeldovich_adjoint(const float* noise, int64_t n_side, double box, const hrt_cosmology* cosmo,
                                    double a_init, const float* disp_bar, const float* mom_bar, const float* disp,
                                    float* noise_bar, double* table_bar_host, double* ratio_bar_host, void* stream) {
  HRT_TRY(check_mesh(n_side, box));
  if (!noise || !cosmo || !disp_bar || !mom_bar || !disp || !noise_bar || !ratio_bar_host)
    return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = as_stream(stream);
  const int64_t n = n_side, np = n * n * n;
  double ratio = 0.0;
  const std::vector<double> t64 = ic_table64(n, box, cosmo, a_init, &ratio);
  std::vector<float> table(t64.begin(), t64.end());
  hrt_pm tmp;
  hrt_status st = pm_make(n, box, 0, s, &tmp);
  float* tab = nullptr;
  float* tot = nullptr;
  double* dbuf = nullptr;  // [0] ratio_bar, [1..] table_bar
  const size_t nt = table.size();
  if (st == HRT_OK) st = upload(table, &tab, s, "IC table");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&tot), 3 * np * sizeof(float), s, "disp_bar total");
  if (st == HRT_OK) st = device_alloc(reinterpret_cast<void**>(&dbuf), (1 + nt) * sizeof(double), s, "IC cotangents");
  if (st == HRT_OK) st = cuda_status(cudaMemsetAsync(dbuf, 0, (1 + nt) * sizeof(double), s), "memset");
  // mom = ratio * disp: ratio_bar = <mom_bar, disp>, disp_bar_total = disp_bar + ratio * mom_bar
  if (st == HRT_OK) st = launch_dot(mom_bar, disp, 3 * np, dbuf, s);
  if (st == HRT_OK) st = cuda_status(cudaMemcpyAsync(tot, disp_bar, 3 * np * sizeof(float), cudaMemcpyDeviceToDevice, s), "copy");
  if (st == HRT_OK) st = launch_axpy(mom_bar, tot, ratio, 3 * np, s);
  const size_t sb = spectrum_bytes(n);
  char* gh = static_cast<char*>(tmp.grad_hat);
  for (int j = 0; j < 3 && st == HRT_OK; ++j)
    st = cufft_status(cufftExecR2C(tmp.r2c, tot + j * np, reinterpret_cast<cufftComplex*>(gh + j * sb)), "IC adj R2C");
  // w_hat into the rho_hat buffer, the adjoint spectrum written over the third disp spectrum's neighbour:
  // use the FFT work-free C2R input buffer = rho_hat after the table cotangent pass
  void* out = nullptr;
  if (st == HRT_OK) st = device_alloc(&out, sb, s, "noise_bar spectrum");
  if (st == HRT_OK)
    st = cufft_status(cufftExecR2C(tmp.r2c, const_cast<float*>(noise), static_cast<cufftComplex*>(tmp.rho_hat)), "IC R2C");
  if (st == HRT_OK) st = launch_ic_adjoint(gh, tmp.rho_hat, n, box, tab, out, table_bar_host ? dbuf + 1 : nullptr, s);
  if (st == HRT_OK) st = cufft_status(cufftExecC2R(tmp.c2r, static_cast<cufftComplex*>(out), noise_bar), "IC adj C2R");
  std::vector<double> hb(1 + nt);
  if (st == HRT_OK) st = cuda_status(cudaMemcpyAsync(hb.data(), dbuf, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
  if (st == HRT_OK) st = cuda_status(cudaStreamSynchronize(s), "sync");
  device_free(tab, s);
  device_free(tot, s);
  device_free(dbuf, s);
  device_free(out, s);
  pm_release(&tmp);
  if (st != HRT_OK) return st;
  *ratio_bar_host = hb[0];
  if (table_bar_host) std::memcpy(table_bar_host, hb.data() + 1, nt * sizeof(double));
  return HRT_OK;
}

hrt_status hrt_dot(const float* a, const float* b, int64_t m, double* out_host, void* stream) {
  if (!a || !b || !out_host || m < 0) return fail(HRT_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = as_stream(stream);
  double* d = nullptr;
  HRT_TRY(device_alloc(reinterpret_cast<void**>(&d), sizeof(double), s, "dot"));
  hrt_status st = cuda_status(cudaMemsetAsync(d, 0, sizeof(double), s), "memset");
  if (st == HRT_OK) st = launch_dot(a, b, m, d, s);
  if (st == HRT_OK) st = cuda_status(cudaMemcpyAsync(out_host, d, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
  if (st == HRT_OK) st = cuda_status(cudaStreamSynchronize(s), "sync");
  device_free(d, s);
  return st;
}

// ---------------------------------------------------------------------------------------------------------
// Learned correction
// ---------------------------------------------------------------------------------------------------------
hrt_status hrt_mlp_forward(const float* x, int32_t rows, const void* w_bf16, const float* w_f32, float* g,
                           void* stream) {
  if (!x || !w_bf16 || !w_f32 || !g || rows < 0) return fail(HRT_ERR_INVALID_ARG, "bad MLP arguments");
  if (rows == 0) return HRT_OK;
  return launch_mlp_forward(x, rows, w_bf16, w_f32, g, as_stream(stream));
}

hrt_status hrt_mlp_backward(const float* x, int32_t rows, const void* w_bf16, const float* w_f32, const float* g_bar,
                            float* grad, void* stream) {
  if (!x || !w_bf16 || !w_f32 || !g_bar || !grad || rows < 0) return fail(HRT_ERR_INVALID_ARG, "bad MLP arguments");
  if (rows == 0) return HRT_OK;
  return launch_mlp_backward(x, rows, w_bf16, w_f32, g_bar, grad, as_stream(stream));
}

hrt_status hrt_mlp_adam(float* w_f32, void* w_bf16, const float* grad, float* m, float* v, double lr, double beta1,
                        double beta2, double eps, int32_t step, void* stream) {
  if (!w_f32 || !w_bf16 || !grad || !m || !v || step < 1) return fail(HRT_ERR_INVALID_ARG, "bad Adam arguments");
  return launch_adam(w_f32, w_bf16, grad, m, v, lr, beta1, beta2, eps, step, as_stream(stream));
}

hrt_status hrt_mlp_to_bf16(const float* w_f32, void* w_bf16, void* stream) {
  if (!w_f32 || !w_bf16) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  return launch_to_bf16(w_f32, w_bf16, as_stream(stream));
}

hrt_status hrt_kspace_table_adjoint(const void* gbar_hat, int32_t n_comp, const void* rho_hat, int64_t n, double box,
                                    double pref, const hrt_filter* f, float* table_bar, void* stream) {
  HRT_TRY(check_mesh(n, box));
  HRT_TRY(check_filter(f));
  if (!gbar_hat || !rho_hat || !table_bar || n_comp < 1 || n_comp > 3 || !f->g_table)
    return fail(HRT_ERR_INVALID_ARG, "bad table-adjoint arguments");
  cudaStream_t s = as_stream(stream);
  float* tab = nullptr;
  hrt_status st = filter_upload(n, box, *f, &tab, s);
  if (st == HRT_OK)
    st = launch_kspace_table_adjoint(gbar_hat, n_comp, rho_hat, n, box, pref, tab, f->g_nk, f->g_kmax, table_bar, s);
  device_free(tab, s);
  return st;
}

hrt_status hrt_pm_gradient_from_spectrum(hrt_pm* pm, const void* rho_hat, double pref, const hrt_filter* f,
                                         int32_t n_out, float* fields) {
  if (!pm || !rho_hat || !fields || n_out < 1 || n_out > 3) return fail(HRT_ERR_INVALID_ARG, "bad arguments");
  HRT_TRY(check_filter(f));
  float* tab = nullptr;
  HRT_TRY(filter_upload(pm->n, pm->box, *f, &tab, pm->stream));
  char* gh = static_cast<char*>(pm->grad_hat);
  const size_t sb = spectrum_bytes(pm->n), mb = static_cast<size_t>(pm->n) * pm->n * pm->n;
  hrt_status st = launch_kspace(rho_hat, pm->n, pm->box, pref, tab, f, n_out, gh, nullptr, f, 0, nullptr, pm->stream);
  for (int j = 0; j < n_out && st == HRT_OK; ++j)
    st = cufft_status(cufftExecC2R(pm->c2r, reinterpret_cast<cufftComplex*>(gh + j * sb), fields + j * mb), "C2R");
  device_free(tab, pm->stream);
  return st;
}

hrt_status hrt_pm_forward_fft(hrt_pm* pm, const float* real, void* out) {
  if (!pm || !real || !out) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  return cufft_status(cufftExecR2C(pm->r2c, const_cast<float*>(real), static_cast<cufftComplex*>(out)), "R2C");
}

hrt_status hrt_pm_density_spectrum(hrt_pm* pm, void* out) {
  if (!pm || !out) return fail(HRT_ERR_INVALID_ARG, "NULL argument");
  if (pm->last_split)
    return fail(HRT_ERR_STATE, "the last solve took the split path, which keeps no 3D spectrum (hrt_pm_set_split 0)");
  return cuda_status(cudaMemcpyAsync(out, pm->rho_hat, spectrum_bytes(pm->n), cudaMemcpyDeviceToDevice, pm->stream),
                     "copy density spectrum");
}

// ---------------------------------------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------------------------------------
static hrt_status check_config(const hrt_config* c) {
  if (!c) return fail(HRT_ERR_INVALID_ARG, "config is NULL");
  HRT_TRY(check_mesh(c->n_mesh, c->box));
  HRT_TRY(check_particles(c->n_side, c->n_mesh));
  if (!(c->samples_per_cell > 0.0)) return fail(HRT_ERR_INVALID_ARG, "samples_per_cell must be > 0");
  if (!(c->smooth_cells >= 0.0) || !std::isfinite(c->deconv_p)) return fail(HRT_ERR_INVALID_ARG, "bad filter");
  if (c->n_sources < 0 || c->n_sources > 64) return fail(HRT_ERR_INVALID_ARG, "n_sources must be 0..64");
  if (c->ray_fields != 0 && c->ray_fields != 2) return fail(HRT_ERR_INVALID_ARG, "ray_fields must be 0 or 2");
  if (!c->static_mode && !(c->cosmo.omega_m > 0.0 && c->cosmo.omega_m <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "bad omega_m");
  if (!(c->window_hi > c->window_lo)) return fail(HRT_ERR_INVALID_ARG, "empty force window");
  return HRT_OK;
}

hrt_status hrt_workspace_bytes(const hrt_config* cfg, int64_t n_rays, size_t* bytes) {
  HRT_TRY(check_config(cfg));
  if (!bytes || n_rays < 0) return fail(HRT_ERR_INVALID_ARG, "bad arguments");
  const size_t n = cfg->n_mesh, mesh = n * n * n * sizeof(float), np = cfg->n_side * cfg->n_side * cfg->n_side;
  size_t b = 6 * np * sizeof(float) + mesh * (4 + cfg->ray_fields);
  b += spectrum_alloc(cfg->n_mesh) * (1 + 3 + cfg->ray_fields) + 2 * spectrum_bytes(cfg->n_mesh);  // + cuFFT work
  b += static_cast<size_t>(n_rays) * (2 * sizeof(double) + 10 * sizeof(float));
  b += static_cast<size_t>(n_rays) * 4 * sizeof(float) * cfg->n_sources;
  // cell-order storage of the particles (on by default): second copies, two order maps, keys, ranks, sources and
  // the per-segment counters
  b += np * (6 * sizeof(float) + 5 * sizeof(int32_t)) + static_cast<size_t>(particle_sort_counts(cfg->n_mesh)) * sizeof(int32_t);
  *bytes = b;
  return HRT_OK;
}

hrt_status hrt_destroy(hrt_ctx* ctx) {
  if (!ctx) return HRT_OK;
  cudaStream_t s = ctx->stream;
  if (ctx->ray_stream) cudaStreamSynchronize(ctx->ray_stream);
  if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
  cudaStreamSynchronize(s);
  for (auto& v : ctx->phases)
    for (auto& ev : v) {
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
  tape_free(ctx);
  device_free(ctx->disp_alt, s);
  device_free(ctx->mom_alt, s);
  device_free(ctx->order_buf[0], s);
  device_free(ctx->order_buf[1], s);
  device_free(ctx->sort_scratch, s);
  hrt_pm_destroy(ctx->pm);
  hrt_raymesh_destroy(ctx->raymesh);
  device_free(ctx->disp, s);
  device_free(ctx->mom, s);
  device_free(ctx->rho, s);
  device_free(ctx->grad, s);
  device_free(ctx->ray_grad, s);
  device_free(ctx->rays.theta, s);
  device_free(ctx->rays.eta, s);
  device_free(ctx->rays.A, s);
  device_free(ctx->rays.B, s);
  device_free(ctx->maps, s);
  device_free(ctx->finite_flag, s);
  device_free(ctx->corr_w, s);
  device_free(ctx->corr_wb, s);
  device_free(ctx->corr_x, s);
  device_free(ctx->pcorr_w, s);
  device_free(ctx->pcorr_wb, s);
  device_free(ctx->pcorr_x, s);
  device_free(ctx->pcorr_table, s);
  device_free(ctx->corr_table, s);
  device_free(ctx->ray_table, s);
  device_free(ctx->stage, s);
  cudaStreamSynchronize(s);
  if (ctx->ev_staged) cudaEventDestroy(ctx->ev_staged);
  for (cudaEvent_t e : ctx->ev_copied)
    if (e) cudaEventDestroy(e);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->ev_fields) cudaEventDestroy(ctx->ev_fields);
  if (ctx->ev_rays) cudaEventDestroy(ctx->ev_rays);
  if (ctx->ray_stream) cudaStreamDestroy(ctx->ray_stream);
  cudaGetLastError();
  delete ctx;
  return HRT_OK;
}

hrt_status hrt_create(const hrt_config* cfg, void* stream, hrt_ctx** out) {
  if (!out) return fail(HRT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  HRT_TRY(check_config(cfg));
  hrt_ctx* ctx = new (std::nothrow) hrt_ctx();
  if (!ctx) return fail(HRT_ERR_OOM, "host allocation");
  ctx->cfg = *cfg;
  ctx->sort_every = 8;
  ctx->stream = as_stream(stream);
  const int64_t n = cfg->n_mesh, m = n * n * n, np = cfg->n_side * cfg->n_side * cfg->n_side;
  hrt_status s = hrt_pm_create(n, cfg->box, cfg->ray_fields, stream, &ctx->pm);
  if (s == HRT_OK) s = cuda_status(cudaStreamCreateWithFlags(&ctx->ray_stream, cudaStreamNonBlocking), "ray stream");
  if (s == HRT_OK) s = cuda_status(cudaEventCreateWithFlags(&ctx->ev_fields, cudaEventDisableTiming), "event");
  if (s == HRT_OK) s = cuda_status(cudaEventCreateWithFlags(&ctx->ev_rays, cudaEventDisableTiming), "event");
  if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&ctx->disp), 3 * np * sizeof(float), ctx->stream, "disp");
  if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&ctx->mom), 3 * np * sizeof(float), ctx->stream, "mom");
  if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&ctx->rho), m * sizeof(float), ctx->stream, "rho");
  if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&ctx->grad), 3 * m * sizeof(float), ctx->stream, "grad");
  if (s == HRT_OK && cfg->ray_fields)
    s = device_alloc(reinterpret_cast<void**>(&ctx->ray_grad), 2 * m * sizeof(float), ctx->stream, "ray grad");
  if (s != HRT_OK) {
    hrt_destroy(ctx);
    return s;
  }
  *out = ctx;
  return HRT_OK;
}

hrt_status hrt_init_particles_zeldovich(hrt_ctx* ctx, const float* noise, double a_init) {
  HRT_TRY(ctx_guard(ctx));
  if (ctx->cfg.static_mode) return fail(HRT_ERR_STATE, "Zel'dovich ICs need the expanding mode");
  hrt_status s = hrt_ic_zeldovich(noise, ctx->cfg.n_side, ctx->cfg.box, &ctx->cfg.cosmo, a_init, ctx->disp,
                                  ctx->mom, ctx->stream);
  if (s == HRT_OK) s = tape_on_ics(ctx, noise, a_init, false);
  if (s != HRT_OK) return ctx_mark(ctx, s);
  ctx_lattice_order(ctx);
  ctx->a = ctx->a_mom = a_init;
  ctx->have_particles = true;
  return ctx_mark(ctx, ctx_force(ctx));
}

hrt_status hrt_init_particles_2lpt(hrt_ctx* ctx, const float* noise, double a_init) {
  HRT_TRY(ctx_guard(ctx));
  if (ctx->cfg.static_mode) return fail(HRT_ERR_STATE, "2LPT ICs need the expanding mode");
  hrt_status s = hrt_ic_2lpt(noise, ctx->cfg.n_side, ctx->cfg.box, &ctx->cfg.cosmo, a_init, ctx->disp, ctx->mom,
                             ctx->stream);
  if (s == HRT_OK) s = tape_on_ics(ctx, noise, a_init, true);
  if (s != HRT_OK) return ctx_mark(ctx, s);
  ctx_lattice_order(ctx);
  ctx->a = ctx->a_mom = a_init;
  ctx->have_particles = true;
  return ctx_mark(ctx, ctx_force(ctx));
}

hrt_status hrt_init_particles(hrt_ctx* ctx, const float* disp, const float* mom, double a) {
  HRT_TRY(ctx_guard(ctx));
  if (!disp || !mom || !(a > 0.0 && a <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "bad particle arguments");
  tape_invalidate(ctx, "the adjoint starts from initial conditions drawn from white noise");
  const size_t bytes = 3 * static_cast<size_t>(ctx->cfg.n_side * ctx->cfg.n_side * ctx->cfg.n_side) * sizeof(float);
  hrt_status s = cuda_status(cudaMemcpyAsync(ctx->disp, disp, bytes, cudaMemcpyDefault, ctx->stream), "copy disp");
  if (s == HRT_OK) s = cuda_status(cudaMemcpyAsync(ctx->mom, mom, bytes, cudaMemcpyDefault, ctx->stream), "copy mom");
  if (s == HRT_OK && ctx->check_finite) {
    const int64_t n3 = static_cast<int64_t>(bytes / sizeof(float));
    s = ctx_scan(ctx, {{ctx->disp, n3, false}, {ctx->mom, n3, false}}, "hrt_init_particles");
    if (s != HRT_OK) ctx->have_particles = false;  // the force is not computed from a non-finite state
  }
  if (s != HRT_OK) return ctx_mark(ctx, s);
  ctx_lattice_order(ctx, true);
  ctx->a = ctx->a_mom = ctx->cfg.static_mode ? 1.0 : a;
  ctx->have_particles = true;
  return ctx_mark(ctx, ctx_force(ctx));
}

hrt_status hrt_init_rays(hrt_ctx* ctx, const double* theta0, int64_t n_rays) {
  HRT_TRY(ctx_guard(ctx));
  if (n_rays < 1 || !theta0) return fail(HRT_ERR_INVALID_ARG, "bad ray arguments");
  cudaStream_t st = ctx->stream;
  device_free(ctx->rays.theta, st);
  device_free(ctx->rays.eta, st);
  device_free(ctx->rays.A, st);
  device_free(ctx->rays.B, st);
  device_free(ctx->maps, st);
  ctx->rays = hrt_rays{};
  ctx->maps = nullptr;
  hrt_rays r{};
  r.n_rays = n_rays;
  hrt_status s = device_alloc(reinterpret_cast<void**>(&r.theta), 2 * n_rays * sizeof(double), st, "theta");
  if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&r.eta), 2 * n_rays * sizeof(float), st, "eta");
  if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&r.A), 4 * n_rays * sizeof(float), st, "A");
  if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&r.B), 4 * n_rays * sizeof(float), st, "B");
  if (s == HRT_OK && ctx->cfg.n_sources > 0)
    s = device_alloc(reinterpret_cast<void**>(&ctx->maps), 4 * n_rays * ctx->cfg.n_sources * sizeof(float), st, "maps");
  if (s == HRT_OK && ctx->maps)
    s = cuda_status(cudaMemsetAsync(ctx->maps, 0, 4 * n_rays * ctx->cfg.n_sources * sizeof(float), st), "maps memset");
  // theta0 may be host or device memory: it is copied into the context first and initialised in place
  if (s == HRT_OK)
    s = cuda_status(cudaMemcpyAsync(r.theta, theta0, 2 * n_rays * sizeof(double), cudaMemcpyDefault, st), "theta0");
  if (s == HRT_OK && ctx->check_finite) s = ctx_scan(ctx, {{r.theta, 2 * n_rays, true}}, "hrt_init_rays");
  if (s == HRT_OK) s = launch_rays_init(r, r.theta, st);
  if (s == HRT_OK) s = tape_on_rays(ctx, r.theta, n_rays);
  if (s != HRT_OK) {
    device_free(r.theta, st);
    device_free(r.eta, st);
    device_free(r.A, st);
    device_free(r.B, st);
    return ctx_mark(ctx, s);
  }
  ctx->rays = r;
  return HRT_OK;
}

namespace hrt {
static hrt_status ctx_step(hrt_ctx* ctx, double a_next, int32_t source, double weight, bool accumulate);
}

hrt_status hrt_step(hrt_ctx* ctx, double a_next, int32_t source) { return ctx_step(ctx, a_next, source, 1.0, false); }

hrt_status hrt_step_accumulate(hrt_ctx* ctx, double a_next, int32_t source, double weight) {
  if (source < 0) return fail(HRT_ERR_INVALID_ARG, "accumulation needs a map (source >= 0)");
  if (!std::isfinite(weight)) return fail(HRT_ERR_INVALID_ARG, "weight must be finite");
  return ctx_step(ctx, a_next, source, weight, true);
}

hrt_status hrt::ctx_step(hrt_ctx* ctx, double a_next, int32_t source, double weight, bool accumulate) {
  HRT_TRY(ctx_guard(ctx));
  if (ctx->cfg.static_mode) return fail(HRT_ERR_STATE, "hrt_step needs the expanding mode");
  if (!ctx->have_particles) return fail(HRT_ERR_STATE, "no particles");
  if (!ctx->force_valid) return fail(HRT_ERR_STATE, "no force: an earlier call failed while computing it");
  if (!(a_next > 0.0 && a_next <= 1.0) || a_next == ctx->a) return fail(HRT_ERR_INVALID_ARG, "bad a_next");
  // a sort due in this step gets its buffers before anything moves, so that an allocation failure leaves the
  // state as it was
  const bool sort_due =
      ctx->sort_every > 0 && (ctx->sort_first || ctx->steps_since_sort + 1 >= ctx->sort_every);
  if (sort_due) HRT_TRY(ctx_sort_alloc(ctx));
  if (ctx->tape) {
    const char kind = (ctx->rays.n_rays > 0 && a_next < ctx->a) ? 'R' : 'F';
    HRT_TRY(ctx_mark(ctx, tape_on_step(ctx, kind, a_next, source, weight, accumulate)));
  }
  Cosmo c(ctx->cfg.cosmo.omega_m);
  hrt_status s = HRT_OK;
  PhaseScope whole(ctx, 6);
  if (ctx->rays.n_rays > 0 && a_next < ctx->a) {
    if (ctx->profiling || ctx->raymesh) {
      // serialised on the context stream so that each phase has its own time; the ray mesh always runs there
      // (its projection and FFTs beside the kick-drift-deposit made the step 2.5 ms slower than in sequence)
      PhaseScope ps(ctx, 0);
      s = ctx_ray_step(ctx, c.chi(ctx->a), c.chi(a_next), ctx->a, source, ctx->stream, weight, accumulate);
    } else {
      // the ray step runs on the ray stream beside the particle update; the next force waits for it
      s = cuda_status(cudaEventRecord(ctx->ev_fields, ctx->stream), "record fields");
      if (s == HRT_OK) s = cuda_status(cudaStreamWaitEvent(ctx->ray_stream, ctx->ev_fields, 0), "wait fields");
      if (s == HRT_OK)
        s = ctx_ray_step(ctx, c.chi(ctx->a), c.chi(a_next), ctx->a, source, ctx->ray_stream, weight, accumulate);
      if (s == HRT_OK) s = cuda_status(cudaEventRecord(ctx->ev_rays, ctx->ray_stream), "record rays");
      if (s == HRT_OK) ctx->rays_pending = true;
    }
    if (s != HRT_OK) return ctx_mark(ctx, s);
  }
  const double a_half = 0.5 * (ctx->a + a_next);
  const double kick = c.kick(ctx->a_mom, a_half), drift = c.drift(ctx->a, a_next);
  if (sort_due) {
    PhaseScope ps(ctx, 7);
    s = ctx_sort(ctx);
    if (s != HRT_OK) return ctx_mark(ctx, s);
    ctx->steps_since_sort = 0;
  } else if (ctx->sort_every > 0) {
    ++ctx->steps_since_sort;
  }
  {
    // kick, drift and the CIC deposit of the drifted particles (the density of the next force) in one pass
    PhaseScope ps(ctx, 1);
    // brick-sorted particles (the counts scratch of the last sort holds every key's first slot): shared-memory
    // tiles; otherwise the per-particle gathers and reductions
    if (ctx->tiled_deposit != 0 && ctx->order_cur >= 0 && ctx->sort_bricks)
      s = launch_kick_drift_tiled(ctx->grad, ctx->cfg.n_mesh, ctx->cfg.box, ctx->cfg.n_side, ctx->disp, ctx->mom,
                                  kick, drift, ctx->rho, ctx_order(ctx), ctx->sort_scratch, ctx->stream,
                                  ctx->tiled_deposit, ctx->pm ? ctx->pm->xerr : nullptr, ctx->rho_clear);
    else
      s = launch_kick_drift(ctx->grad, ctx->cfg.n_mesh, ctx->cfg.box, ctx->cfg.n_side, ctx->disp, ctx->mom, kick,
                            drift, ctx->stream, ctx->rho, ctx_order(ctx), ctx->rho_clear);
    ctx->rho_clear = false;
  }
  if (s != HRT_OK) return ctx_mark(ctx, s);
  ctx->a = a_next;
  ctx->a_mom = a_half;
  s = ctx_solve(ctx);
  if (s == HRT_OK) s = ctx_scan_state(ctx, "hrt_step");
  return ctx_mark(ctx, s);
}

namespace hrt {
// Sets (params != NULL: copies the FP32 parameters, refreshes the BF16 copy) or removes one learned correction
// network of the context; its buffers are allocated all or none.
static hrt_status set_correction(hrt_ctx* ctx, const float* params, float*& w, void*& wb, float*& x, float*& t) {
  cudaStream_t st = ctx->stream;
  if (!params) {
    device_free(w, st);
    device_free(wb, st);
    device_free(x, st);
    device_free(t, st);
    w = t = x = nullptr;
    wb = nullptr;
    return HRT_OK;
  }
  if (!w) {
    float *nw = nullptr, *nx = nullptr, *nt = nullptr;
    void* nwb = nullptr;
    hrt_status s = device_alloc(reinterpret_cast<void**>(&nw), kMlpParams * sizeof(float), st, "correction");
    if (s == HRT_OK) s = device_alloc(&nwb, kMlpParams * 2, st, "correction bf16");
    if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&nx), 3 * kCorrectionRows * sizeof(float), st, "inputs");
    if (s == HRT_OK) s = device_alloc(reinterpret_cast<void**>(&nt), kCorrectionRows * sizeof(float), st, "table");
    if (s != HRT_OK) {
      device_free(nw, st);
      device_free(nwb, st);
      device_free(nx, st);
      device_free(nt, st);
      return s;
    }
    w = nw;
    wb = nwb;
    x = nx;
    t = nt;
  }
  hrt_status s = cuda_status(cudaMemcpyAsync(w, params, kMlpParams * sizeof(float), cudaMemcpyDeviceToDevice, st),
                             "copy correction");
  if (s == HRT_OK) s = launch_to_bf16(w, wb, st);
  return ctx_mark(ctx, s);
}
}  // namespace hrt

hrt_status hrt_set_ray_correction(hrt_ctx* ctx, const float* params) {
  HRT_TRY(ctx_guard(ctx));
  if (ctx->cfg.ray_fields != 2) return fail(HRT_ERR_STATE, "a ray correction needs ray_fields == 2");
  return set_correction(ctx, params, ctx->corr_w, ctx->corr_wb, ctx->corr_x, ctx->corr_table);
}

hrt_status hrt_set_particle_correction(hrt_ctx* ctx, const float* params) {
  HRT_TRY(ctx_guard(ctx));
  if (ctx->cfg.static_mode) return fail(HRT_ERR_STATE, "a particle-force correction needs the expanding mode");
  if (params) tape_invalidate(ctx, "a learned particle force is not differentiated");
  return set_correction(ctx, params, ctx->pcorr_w, ctx->pcorr_wb, ctx->pcorr_x, ctx->pcorr_table);
}

hrt_status hrt_sync_particles(hrt_ctx* ctx) {
  HRT_TRY(ctx_guard(ctx));
  if (!ctx->have_particles) return fail(HRT_ERR_STATE, "no particles");
  if (ctx->cfg.static_mode || ctx->a_mom == ctx->a) return HRT_OK;
  if (!ctx->force_valid) return fail(HRT_ERR_STATE, "no force: an earlier call failed while computing it");
  Cosmo c(ctx->cfg.cosmo.omega_m);
  HRT_TRY(ctx_mark(ctx, tape_on_step(ctx, 'S', ctx->a, -1, 1.0, false)));
  hrt_status s = launch_kick_drift(ctx->grad, ctx->cfg.n_mesh, ctx->cfg.box, ctx->cfg.n_side, ctx->disp, ctx->mom,
                                   c.kick(ctx->a_mom, ctx->a), 0.0, ctx->stream, nullptr, ctx_order(ctx));
  if (s == HRT_OK) ctx->a_mom = ctx->a;
  return ctx_mark(ctx, s);
}

hrt_status hrt_step_static(hrt_ctx* ctx, double chi_from, double chi_to, int32_t source) {
  HRT_TRY(ctx_guard(ctx));
  if (!ctx->cfg.static_mode) return fail(HRT_ERR_STATE, "hrt_step_static needs the static mode");
  if (!ctx->have_particles) return fail(HRT_ERR_STATE, "no lens particles");
  if (ctx->rays.n_rays == 0) return fail(HRT_ERR_STATE, "no rays");
  if (!ctx->force_valid) return fail(HRT_ERR_STATE, "no force: an earlier call failed while computing it");
  tape_invalidate(ctx, "static-lens steps are not differentiated");
  return ctx_mark(ctx, ctx_ray_step(ctx, chi_from, chi_to, 0.0, source, ctx->stream));
}

hrt_status hrt_drift_free(hrt_ctx* ctx, double chi_from, double chi_to) {
  HRT_TRY(ctx_guard(ctx));
  if (ctx->rays.n_rays == 0) return fail(HRT_ERR_STATE, "no rays");
  tape_invalidate(ctx, "free drifts are not differentiated");
  return ctx_mark(ctx, hrt_ray_drift_free(&ctx->rays, chi_from, chi_to, ctx->stream));
}

hrt_status hrt_read_rays(hrt_ctx* ctx, double* theta, float* eta, float* A, float* B) {
  HRT_TRY(ctx_guard(ctx));
  const int64_t r = ctx->rays.n_rays;
  if (r == 0) return fail(HRT_ERR_STATE, "no rays");
  hrt_status s = HRT_OK;
  if (theta) s = cuda_status(cudaMemcpyAsync(theta, ctx->rays.theta, 2 * r * sizeof(double), cudaMemcpyDefault, ctx->stream), "read theta");
  if (s == HRT_OK && eta) s = cuda_status(cudaMemcpyAsync(eta, ctx->rays.eta, 2 * r * sizeof(float), cudaMemcpyDefault, ctx->stream), "read eta");
  if (s == HRT_OK && A) s = cuda_status(cudaMemcpyAsync(A, ctx->rays.A, 4 * r * sizeof(float), cudaMemcpyDefault, ctx->stream), "read A");
  if (s == HRT_OK && B) s = cuda_status(cudaMemcpyAsync(B, ctx->rays.B, 4 * r * sizeof(float), cudaMemcpyDefault, ctx->stream), "read B");
  return ctx_mark(ctx, s);
}

hrt_status hrt_read_maps(hrt_ctx* ctx, int32_t source, float* kappa, float* gamma1, float* gamma2, float* omega) {
  HRT_TRY(ctx_guard(ctx));
  const int64_t r = ctx->rays.n_rays;
  if (r == 0 || !ctx->maps) return fail(HRT_ERR_STATE, "no maps");
  if (source < 0 || source >= ctx->cfg.n_sources) return fail(HRT_ERR_INVALID_ARG, "source out of range");
  float* base = ctx->maps + static_cast<int64_t>(source) * 4 * r;
  float* dst[4] = {kappa, gamma1, gamma2, omega};
  for (int i = 0; i < 4; ++i)
    if (dst[i]) {
      hrt_status s = cuda_status(cudaMemcpyAsync(dst[i], base + i * r, r * sizeof(float), cudaMemcpyDefault, ctx->stream), "read map");
      if (s != HRT_OK) return ctx_mark(ctx, s);
    }
  return HRT_OK;
}

namespace hrt {
// The copy stream, its events and a staging buffer of at least `bytes` for the asynchronous read-outs, made on
// first use (stream and events all or none).  The regions' offsets follow the ray count, so a new layout (rays
// initialised again with another count) first lets the copies still reading the old regions finish; a larger
// buffer then replaces the old one.
static hrt_status ctx_stage(hrt_ctx* ctx, size_t bytes) {
  if (!ctx->copy_stream) {
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    hrt_status s = cuda_status(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "copy stream");
    for (int i = 0; i < 3 && s == HRT_OK; ++i)
      s = cuda_status(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming), "read-out event");
    if (s != HRT_OK) {
      for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
      if (cs) cudaStreamDestroy(cs);
      return s;
    }
    ctx->copy_stream = cs;
    ctx->ev_staged = ev[0];
    ctx->ev_copied[0] = ev[1];
    ctx->ev_copied[1] = ev[2];
  }
  if (bytes != ctx->stage_layout && (ctx->copy_pending[0] || ctx->copy_pending[1])) {
    HRT_TRY(wait_stream(ctx->copy_stream, "read-out copies"));
    ctx->copy_pending[0] = ctx->copy_pending[1] = false;
  }
  ctx->stage_layout = bytes;
  if (ctx->stage_bytes >= bytes) return HRT_OK;
  char* p = nullptr;
  HRT_TRY(device_alloc(reinterpret_cast<void**>(&p), bytes, ctx->stream, "read-out staging"));
  device_free(ctx->stage, ctx->stream);
  ctx->stage = p;
  ctx->stage_bytes = bytes;
  return HRT_OK;
}

// One asynchronous read-out through staging region `region` (offset off): the device data is copied into the
// region on the context stream, in order after the work queued so far and after the last copy out of the same
// region, and from there to the host on the copy stream, where it runs beside the context's next kernels.
static hrt_status ctx_read_async(hrt_ctx* ctx, int region, size_t off, const void* dev, size_t bytes, void* host) {
  cudaStream_t st = ctx->stream;
  if (ctx->copy_pending[region]) HRT_CUDA(cudaStreamWaitEvent(st, ctx->ev_copied[region], 0));
  HRT_CUDA(cudaMemcpyAsync(ctx->stage + off, dev, bytes, cudaMemcpyDeviceToDevice, st));
  HRT_CUDA(cudaEventRecord(ctx->ev_staged, st));
  HRT_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_staged, 0));
  HRT_CUDA(cudaMemcpyAsync(host, ctx->stage + off, bytes, cudaMemcpyDefault, ctx->copy_stream));
  HRT_CUDA(cudaEventRecord(ctx->ev_copied[region], ctx->copy_stream));
  ctx->copy_pending[region] = true;
  return HRT_OK;
}
}  // namespace hrt

hrt_status hrt_read_rays_async(hrt_ctx* ctx, double* theta_host) {
  HRT_TRY(ctx_guard(ctx));
  const int64_t r = ctx->rays.n_rays;
  if (r == 0) return fail(HRT_ERR_STATE, "no rays");
  if (!theta_host) return fail(HRT_ERR_INVALID_ARG, "NULL destination");
  HRT_TRY(ctx_mark(ctx, ctx_stage(ctx, 20 * static_cast<size_t>(r))));
  return ctx_mark(ctx, ctx_read_async(ctx, 0, 0, ctx->rays.theta, 16 * static_cast<size_t>(r), theta_host));
}

hrt_status hrt_read_kappa_async(hrt_ctx* ctx, int32_t source, float* kappa_host) {
  HRT_TRY(ctx_guard(ctx));
  const int64_t r = ctx->rays.n_rays;
  if (r == 0 || !ctx->maps) return fail(HRT_ERR_STATE, "no maps");
  if (source < 0 || source >= ctx->cfg.n_sources) return fail(HRT_ERR_INVALID_ARG, "source out of range");
  if (!kappa_host) return fail(HRT_ERR_INVALID_ARG, "NULL destination");
  HRT_TRY(ctx_mark(ctx, ctx_stage(ctx, 20 * static_cast<size_t>(r))));
  return ctx_mark(ctx, ctx_read_async(ctx, 1, 16 * static_cast<size_t>(r),
                                      ctx->maps + static_cast<int64_t>(source) * 4 * r, 4 * static_cast<size_t>(r),
                                      kappa_host));
}

hrt_status hrt_read_wait(hrt_ctx* ctx) {
  HRT_TRY(ctx_guard(ctx));
  if (!ctx->copy_stream) return HRT_OK;
  HRT_TRY(ctx_mark(ctx, wait_stream(ctx->copy_stream, "hrt_read_wait")));
  ctx->copy_pending[0] = ctx->copy_pending[1] = false;
  return HRT_OK;
}

hrt_status hrt_read_particles(hrt_ctx* ctx, float* disp, float* mom, double* a_host, double* a_mom_host) {
  HRT_TRY(ctx_guard(ctx));
  if (!ctx->have_particles) return fail(HRT_ERR_STATE, "no particles");
  hrt_status s = ctx_particles_lattice(ctx, disp, mom);
  if (a_host) *a_host = ctx->a;
  if (a_mom_host) *a_mom_host = ctx->a_mom;
  return ctx_mark(ctx, s);
}

hrt_status hrt_read_grad(hrt_ctx* ctx, float* grad) {
  HRT_TRY(ctx_guard(ctx));
  if (!grad) return fail(HRT_ERR_INVALID_ARG, "grad is NULL");
  if (!ctx->have_particles || !ctx->force_valid) return fail(HRT_ERR_STATE, "no force");
  const size_t n = ctx->cfg.n_mesh;
  return ctx_mark(ctx, cuda_status(cudaMemcpyAsync(grad, ctx->grad, 3 * n * n * n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream), "read grad"));
}

hrt_status hrt_set_replicas(hrt_ctx* ctx, int32_t n, const int32_t* perm, const int32_t* sign, const int32_t* shift) {
  HRT_TRY(ctx_guard(ctx));
  if (n == 0) {
    ctx->rep_perm.clear();
    ctx->rep_sign.clear();
    ctx->rep_shift.clear();
    return HRT_OK;
  }
  if (ctx->cfg.ray_fields != 0) return fail(HRT_ERR_STATE, "light-cone tiling uses the particle fields (ray_fields == 0)");
  if (n < 0 || n > kMaxReplicas || !perm || !sign || !shift)
    return fail(HRT_ERR_INVALID_ARG, "tiling needs 1..%d replicas with their perm, sign and shift tables", kMaxReplicas);
  // validate through the node-table builder (one empty shell at the observer's replica)
  hrt_ray_geom g = ctx_geom(ctx->cfg, nullptr);
  g.n_replicas = n;
  g.replica_perm = perm;
  g.replica_sign = sign;
  g.replica_shift = shift;
  static thread_local RayStepParams p;
  g.window_lo = g.window_hi = 0.0;
  HRT_TRY(build_ray_params(g, 1.0, 2.0, 0.0, ctx->cfg.cosmo.omega_m, p));
  ctx->rep_perm.assign(perm, perm + 3 * n);
  ctx->rep_sign.assign(sign, sign + 3 * n);
  ctx->rep_shift.assign(shift, shift + 3 * n);
  return HRT_OK;
}

hrt_status hrt_set_particle_sort(hrt_ctx* ctx, int32_t every) {
  HRT_TRY(ctx_guard(ctx));
  if (every < 0) return fail(HRT_ERR_INVALID_ARG, "sort interval must be >= 0");
  ctx->sort_every = every;
  ctx->steps_since_sort = 0;
  return HRT_OK;
}

hrt_status hrt_set_tiled_deposit(hrt_ctx* ctx, int32_t mode) {
  HRT_TRY(ctx_guard(ctx));
  if (mode < 0 || mode > kTilesTma) return fail(HRT_ERR_INVALID_ARG, "tile mode must be 0, 1 or 2");
  ctx->tiled_deposit = mode;
  return HRT_OK;
}

hrt_status hrt_set_checkpointing(hrt_ctx* ctx, int32_t every) {
  HRT_TRY(ctx_guard(ctx));
  if (every < 0) return fail(HRT_ERR_INVALID_ARG, "checkpoint interval must be >= 0");
  tape_free(ctx);
  if (every > 0) {
    ctx->tape = new (std::nothrow) Tape;
    if (!ctx->tape) return fail(HRT_ERR_OOM, "tape");
    ctx->tape->every = every;
  }
  return HRT_OK;
}

hrt_status hrt_adjoint(hrt_ctx* ctx, const float* kappa_bar, const double* theta_bar, float* noise_bar,
                       double* omega_bar_host) {
  HRT_TRY(ctx_guard(ctx));
  if (ctx->ray_stream) cudaStreamSynchronize(ctx->ray_stream);
  hrt_status s = tape_adjoint(ctx, kappa_bar, theta_bar, noise_bar, omega_bar_host);
  if (s == HRT_OK) s = cuda_status(cudaStreamSynchronize(ctx->stream), "adjoint sync");
  return ctx_mark(ctx, s);
}

hrt_status hrt_set_ray_mesh(hrt_ctx* ctx, const hrt_raymesh_config* cfg) {
  HRT_TRY(ctx_guard(ctx));
  hrt_raymesh* rm = nullptr;
  if (cfg) HRT_TRY(hrt_raymesh_create(cfg, &rm));
  if (ctx->ray_stream) cudaStreamSynchronize(ctx->ray_stream);
  cudaStreamSynchronize(ctx->stream);
  hrt_raymesh_destroy(ctx->raymesh);
  ctx->raymesh = rm;
  return HRT_OK;
}

hrt_status hrt_set_ray_kernel_table(hrt_ctx* ctx, const float* g, int32_t nk, double kmax) {
  HRT_TRY(ctx_guard(ctx));
  if (ctx->cfg.ray_fields != 2) return fail(HRT_ERR_STATE, "a ray kernel table needs ray_fields == 2");
  cudaStream_t st = ctx->stream;
  device_free(ctx->ray_table, st);
  ctx->ray_table = nullptr;
  ctx->ray_table_nk = 0;
  if (!g) return HRT_OK;
  if (nk < 2 || !(kmax > 0.0) || !std::isfinite(kmax)) return fail(HRT_ERR_INVALID_ARG, "table needs nk >= 2, kmax > 0");
  float* t = nullptr;
  HRT_TRY(device_alloc(reinterpret_cast<void**>(&t), static_cast<size_t>(nk) * sizeof(float), st, "ray table"));
  hrt_status s = cuda_status(cudaMemcpyAsync(t, g, static_cast<size_t>(nk) * sizeof(float), cudaMemcpyDeviceToDevice, st),
                             "copy ray table");
  if (s != HRT_OK) {
    device_free(t, st);
    return ctx_mark(ctx, s);
  }
  // the network-based correction and a fixed table are exclusive
  if (ctx->corr_w) HRT_TRY(hrt_set_ray_correction(ctx, nullptr));
  ctx->ray_table = t;
  ctx->ray_table_nk = nk;
  ctx->ray_table_kmax = kmax;
  return HRT_OK;
}

// ---- checkpoint / resume: a header, then the particle and ray state and the maps, in caller device memory
namespace hrt {
struct StateHeader {
  uint64_t magic;
  int64_t n_side, n_mesh, n_rays;
  int32_t n_sources, have_particles;
  double a, a_mom;
  uint64_t bytes;
};
constexpr uint64_t kStateMagic = 0x3154415453545248ull;  // "HRTSTAT1"

static size_t state_bytes(const hrt_ctx* ctx) {
  const size_t np = static_cast<size_t>(ctx->cfg.n_side * ctx->cfg.n_side * ctx->cfg.n_side);
  const size_t r = static_cast<size_t>(ctx->rays.n_rays);
  const size_t maps = ctx->maps ? 4 * r * static_cast<size_t>(ctx->cfg.n_sources) : 0;
  return 256 + 6 * np * sizeof(float) + r * (2 * sizeof(double) + 10 * sizeof(float)) + maps * sizeof(float);
}
}  // namespace hrt

hrt_status hrt_state_bytes(hrt_ctx* ctx, size_t* bytes) {
  HRT_TRY(ctx_guard(ctx));
  if (!bytes) return fail(HRT_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = state_bytes(ctx);
  return HRT_OK;
}

hrt_status hrt_save_state(hrt_ctx* ctx, void* buf, size_t bytes) {
  HRT_TRY(ctx_guard(ctx));
  if (!buf) return fail(HRT_ERR_INVALID_ARG, "buffer is NULL");
  if (!ctx->have_particles) return fail(HRT_ERR_STATE, "no particles to save");
  const size_t need = state_bytes(ctx);
  if (bytes < need) return fail(HRT_ERR_INVALID_ARG, "state needs %zu bytes, buffer has %zu", need, bytes);
  StateHeader h{kStateMagic, ctx->cfg.n_side, ctx->cfg.n_mesh, ctx->rays.n_rays, ctx->maps ? ctx->cfg.n_sources : 0,
                1, ctx->a, ctx->a_mom, need};
  const size_t np3 = 3 * static_cast<size_t>(ctx->cfg.n_side * ctx->cfg.n_side * ctx->cfg.n_side);
  const size_t r = static_cast<size_t>(ctx->rays.n_rays);
  cudaStream_t st = ctx->stream;
  char* p = static_cast<char*>(buf);
  hrt_status s = cuda_status(cudaMemcpyAsync(p, &h, sizeof(h), cudaMemcpyHostToDevice, st), "save header");
  p += 256;
  auto put = [&](const void* src, size_t n) {
    if (s == HRT_OK && n) s = cuda_status(cudaMemcpyAsync(p, src, n, cudaMemcpyDeviceToDevice, st), "save state");
    p += n;
  };
  // particles in lattice order
  if (s == HRT_OK) s = ctx_particles_lattice(ctx, reinterpret_cast<float*>(p), reinterpret_cast<float*>(p) + np3);
  p += 2 * np3 * sizeof(float);
  put(ctx->rays.theta, 2 * r * sizeof(double));
  put(ctx->rays.eta, 2 * r * sizeof(float));
  put(ctx->rays.A, 4 * r * sizeof(float));
  put(ctx->rays.B, 4 * r * sizeof(float));
  if (ctx->maps) put(ctx->maps, 4 * r * static_cast<size_t>(ctx->cfg.n_sources) * sizeof(float));
  // the header copy reads host memory on the stream: wait before it goes out of scope
  if (s == HRT_OK) s = cuda_status(cudaStreamSynchronize(st), "save state");
  return ctx_mark(ctx, s);
}

hrt_status hrt_load_state(hrt_ctx* ctx, const void* buf, size_t bytes) {
  HRT_TRY(ctx_guard(ctx));
  tape_invalidate(ctx, "a loaded state is not differentiated");
  ctx_lattice_order(ctx, true);
  if (!buf || bytes < 256) return fail(HRT_ERR_INVALID_ARG, "state buffer is NULL or too small");
  StateHeader h{};
  cudaStream_t st = ctx->stream;
  HRT_TRY(ctx_mark(ctx, cuda_status(cudaMemcpyAsync(&h, buf, sizeof(h), cudaMemcpyDeviceToHost, st), "load header")));
  HRT_TRY(ctx_mark(ctx, cuda_status(cudaStreamSynchronize(st), "load header")));
  if (h.magic != kStateMagic) return fail(HRT_ERR_INVALID_ARG, "not a saved HRT state");
  if (h.n_side != ctx->cfg.n_side || h.n_mesh != ctx->cfg.n_mesh)
    return fail(HRT_ERR_INVALID_ARG, "saved state is for %lld particles per side and mesh %lld",
                static_cast<long long>(h.n_side), static_cast<long long>(h.n_mesh));
  if (h.bytes > bytes) return fail(HRT_ERR_INVALID_ARG, "state buffer shorter than the saved state");
  if (h.n_sources > ctx->cfg.n_sources) return fail(HRT_ERR_INVALID_ARG, "saved state has more source planes");
  if (!(h.a > 0.0 && h.a <= 1.0) || !(h.a_mom > 0.0 && h.a_mom <= 1.0)) return fail(HRT_ERR_INVALID_ARG, "bad scale factors");
  const size_t np3 = 3 * static_cast<size_t>(h.n_side * h.n_side * h.n_side);
  const size_t r = static_cast<size_t>(h.n_rays);
  const char* p = static_cast<const char*>(buf) + 256;
  hrt_status s = HRT_OK;
  auto get = [&](void* dst, size_t n) {
    if (s == HRT_OK && n) s = cuda_status(cudaMemcpyAsync(dst, p, n, cudaMemcpyDeviceToDevice, st), "load state");
    p += n;
  };
  get(ctx->disp, np3 * sizeof(float));
  get(ctx->mom, np3 * sizeof(float));
  if (s != HRT_OK) return ctx_mark(ctx, s);
  if (r > 0) {
    // reallocates the ray state and the maps for r rays (initialised from the saved angles, then overwritten)
    HRT_TRY(hrt_init_rays(ctx, reinterpret_cast<const double*>(p), static_cast<int64_t>(r)));
    get(ctx->rays.theta, 2 * r * sizeof(double));
    get(ctx->rays.eta, 2 * r * sizeof(float));
    get(ctx->rays.A, 4 * r * sizeof(float));
    get(ctx->rays.B, 4 * r * sizeof(float));
    if (h.n_sources > 0 && ctx->maps) get(ctx->maps, 4 * r * static_cast<size_t>(h.n_sources) * sizeof(float));
  }
  if (s != HRT_OK) return ctx_mark(ctx, s);
  ctx->a = ctx->cfg.static_mode ? 1.0 : h.a;
  ctx->a_mom = ctx->cfg.static_mode ? 1.0 : h.a_mom;
  ctx->have_particles = true;
  return ctx_mark(ctx, ctx_force(ctx));
}

hrt_status hrt_ctx_kappa_power(hrt_ctx* ctx, int32_t source, int64_t m, double dtheta, int32_t nbins, double ell_min,
                               double ell_max, double* ell_host, double* p_host, int64_t* count_host) {
  HRT_TRY(ctx_guard(ctx));
  if (!ctx->maps || source < 0 || source >= ctx->cfg.n_sources) return fail(HRT_ERR_INVALID_ARG, "no such map");
  if (m * m != ctx->rays.n_rays) return fail(HRT_ERR_INVALID_ARG, "rays do not form an m x m image");
  const float* kappa = ctx->maps + static_cast<int64_t>(source) * 4 * ctx->rays.n_rays;
  return ctx_mark(ctx, hrt_kappa_power(kappa, m, dtheta, nbins, ell_min, ell_max, ell_host, p_host, count_host, ctx->stream));
}

hrt_status hrt_set_nonfinite_check(hrt_ctx* ctx, int32_t on) {
  HRT_TRY(ctx_guard(ctx));
  if (on && !ctx->finite_flag)
    HRT_TRY(device_alloc(reinterpret_cast<void**>(&ctx->finite_flag), sizeof(int), ctx->stream, "finite flag"));
  ctx->check_finite = on != 0;
  return HRT_OK;
}

hrt_status hrt_static_prefactor(double mass, double box, double* pref) {
  if (!pref) return fail(HRT_ERR_INVALID_ARG, "pref is NULL");
  if (!(mass > 0.0) || !std::isfinite(mass) || !(box > 0.0) || !std::isfinite(box))
    return fail(HRT_ERR_INVALID_ARG, "mass and box must be positive and finite");
  // the Poisson equation of a static lens, lap(phi) = 4 pi G rho_mean delta with rho_mean = M / L^3
  *pref = 4.0 * M_PI * kGNewton * mass / (box * box * box);
  return HRT_OK;
}

hrt_status hrt_set_ray_theta_bits(hrt_ctx* ctx, int32_t bits) {
  HRT_TRY(ctx_guard(ctx));
  if (bits != 32 && bits != 64) return fail(HRT_ERR_INVALID_ARG, "ray angle bits must be 32 or 64");
  if (bits == 32) tape_invalidate(ctx, "the FP32 ray-angle ablation is not differentiated");
  ctx->theta32 = bits == 32;
  return HRT_OK;
}

hrt_status hrt_inject_alloc_failure(int64_t k) {
  if (k < 0) return fail(HRT_ERR_INVALID_ARG, "k must be >= 0");
  set_alloc_failure(k);
  return HRT_OK;
}

hrt_status hrt_set_host_wait_limit(double seconds) {
  if (std::isnan(seconds)) return fail(HRT_ERR_INVALID_ARG, "the wait limit must be a number");
  g_wait_limit.store(seconds);
  return HRT_OK;
}

hrt_status hrt_ctx_set_profiling(hrt_ctx* ctx, int32_t on) {
  HRT_TRY(ctx_guard(ctx));
  ctx->profiling = on != 0;
  return HRT_OK;
}

hrt_status hrt_ctx_phase_times(hrt_ctx* ctx, double* ms, int64_t* counts) {
  HRT_TRY(ctx_guard(ctx));
  if (!ms || !counts) return fail(HRT_ERR_INVALID_ARG, "NULL output");
  hrt_status st = cuda_status(cudaStreamSynchronize(ctx->stream), "phase sync");
  for (int p = 0; p < 8; ++p) {
    double sum = 0.0;
    for (auto& ev : ctx->phases[p]) {
      float t = 0.f;
      if (st == HRT_OK && cudaEventElapsedTime(&t, ev.first, ev.second) == cudaSuccess) sum += t;
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
    ms[p] = sum;
    counts[p] = static_cast<int64_t>(ctx->phases[p].size());
    ctx->phases[p].clear();
  }
  return ctx_mark(ctx, st);
}

hrt_status hrt_ctx_rays(hrt_ctx* ctx, hrt_rays* out) {
  HRT_TRY(ctx_guard(ctx));
  if (!out) return fail(HRT_ERR_INVALID_ARG, "out is NULL");
  *out = ctx->rays;
  return HRT_OK;
}

}  // extern "C"
