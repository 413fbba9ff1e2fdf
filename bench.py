#!/usr/bin/env python
"""Throughput of the HRT hot path on GB300: reverse co-evolution sim-steps/s (Alg. 1 per step: ray KDK with
readout, particle gather-kick-drift, CIC scatter, R2C FFT, fused k-space kernel, 3 C2R FFTs).

Default workload: 512^3 particles, 1024^3 mesh, box 1 Gpc/h, 2048^2 rays over 10 deg, reverse steps uniform in a
from 1 to 1/3 (source planes z = 0.5, 1, 2), synthetic Zel'dovich ICs evolved forward from a = 0.02 first.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun each rank runs an independent replica (its own seed); the timed region is bracketed by a
barrier and a device synchronise, and rank 0 reports the maximum over ranks.  The reference arm times the
FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HRT sim-steps/s (512³ p,1024³ mesh,4M rays) vs plain path at κ P(ℓ) err<1%"
UNIT = "sim-steps/s"
KERNEL_SOURCES = {
    "ray_step": ["ray_kernels.cu", "mesh_kernels.h"],
    "kick_drift": ["mesh_kernels.cu"],
    "cic_scatter": ["mesh_kernels.cu"],
    "kspace": ["mesh_kernels.cu", "xpass_kernels.cu", "tma.h"],
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=64)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="cosmo_512p_1024m_2048r")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-next", action="store_true",
                   help="skip the timings of the widened rows (tiled light cone, accumulated sources, 2LPT ICs)")
    p.add_argument("--no-learned", action="store_true",
                   help="skip the learned-correction comparison (coarse learned vs coarse plain vs fine plain)")
    p.add_argument("--no-precision", action="store_true",
                   help="skip the per-output errors against the stored FP64 oracle outputs (and the FP32-angle ablation)")
    p.add_argument("--sort-every", type=int, default=None,
                   help="re-sort the particles by mesh cell every K particle steps (default: the library's, 8; 0: never)")
    p.add_argument("--tiled-deposit", type=int, default=0, choices=[0, 1, 2],
                   help="kick-drift-deposit: 0 per-particle gathers and reductions on z-row order (default), "
                        "2 shared-memory tiles by TMA on brick order, 1 tiles by row copies")
    p.add_argument("--kick", default="direct", choices=["direct", "mesh"],
                   help="kick operator of the rays: the direct line-of-sight gather or the ray mesh of Sec. 5.2")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="hrt_clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------------------------- replicas
def replica_seed(W, rank: int) -> int:
    """Each rank runs an independent replica of the workload on its own seed."""
    return W.seed + rank


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (the job's time); `device` is the rank's device ("cpu" under gloo)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(steps: int, ms_max: float, world: int) -> float:
    """Whole-job sim-steps/s: every rank did `steps` steps, the job took the slowest rank's time."""
    return world * steps / (ms_max / 1e3)


# ----------------------------------------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(kernel: str) -> str:
    """Hash of the kernel's source files with comments, trailing blanks and empty lines removed, so that only a
    change of the code voids a recorded traffic figure."""
    import re
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES.get(kernel, []):
        text = open(os.path.join(ROOT, "paper_2405_12913_gb300", "csrc", fn), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [ln.rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(workload, {}).get(kernel)
    if not d or d.get("source_hash") != kernel_source_hash(kernel):
        return None
    return d.get("dram_bytes_per_launch")


# the ray mesh with the paper's hyper-parameters (iota = 0.5, p_min = 256; App. C) and the image's pixel size
RAYMESH_IOTA, RAYMESH_P_MIN = 0.5, 256.0


def raymesh_config(hrt, W, iota=None, p_min=None):
    return hrt.make_raymesh_config(RAYMESH_IOTA if iota is None else iota, RAYMESH_P_MIN if p_min is None else p_min,
                                   W.dtheta, W.n_pix)


def raymesh_sides(hrt, W, iota=None, p_min=None):
    """Smallest and largest ray-mesh side over the half shells of the reverse grid."""
    from paper_2405_12913_gb300.hrt import hrt_cosmo_eval
    chis = [hrt_cosmo_eval(W.omega_m, a)[1] for a in W.reverse_grid]
    sides = []
    for a, b in zip(chis[:-1], chis[1:]):
        m = 0.5 * (a + b)
        for lo, hi in ((a, m), (m, b)):
            sides.append(hrt.hrt_raymesh_geometry(raymesh_config(hrt, W, iota, p_min), lo, hi, W.box / W.n_mesh)[2])
    return min(sides), max(sides)


def algorithmic_bytes(W):
    """Algorithmic HBM bytes per launch (one read or write per element)."""
    mesh = W.n_mesh ** 3 * 4
    spec = W.n_mesh * W.n_mesh * (W.n_mesh // 2 + 1) * 8
    npart = W.n_side ** 3
    rays = W.n_rays
    return {
        "cic_scatter": 3 * 4 * npart + mesh,                 # positions read + density written
        # density spectrum read + 3 gradient spectra written; on the split path (mesh sides 256, 512, 1024) the
        # x-pass also zeroes the consumed density for the next deposit
        "kspace": spec + 3 * spec + (mesh if W.n_mesh in (256, 512, 1024) else 0),
        "kick_drift": 4 * mesh + 2 * 2 * 3 * 4 * npart,      # 3 fields read, density written, disp/mom r+w
        "ray_step": 2 * rays * (16 + 8 + 16 + 16),           # ray state read and written (slab reads extra)
        "fft_r2c": mesh + spec,
        "fft_c2r": 3 * (spec + mesh),
    }


# ----------------------------------------------------------------------------------------------- GPU arm
def run_gpu(args, W, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12913_gb300 import hrt
    import synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    seed = replica_seed(W, rank)
    cfg = hrt.make_config(W.n_mesh, W.box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p, W.smooth_cells,
                          W.samples_per_cell, W.observer, n_sources=len(W.source_steps))
    ctx = hrt.Context(cfg)
    if args.sort_every is not None:
        ctx.hrt_set_particle_sort(args.sort_every)
    if args.tiled_deposit != 0:
        ctx.hrt_set_tiled_deposit(args.tiled_deposit)
    noise = torch.from_numpy(synthetic.white_noise(seed, W.n_side).astype(np.float32)).to(dev)
    theta0_h = torch.from_numpy(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE))
    theta0 = theta0_h.to(dev)
    ctx.hrt_init_particles_zeldovich(noise, W.a_init)
    del noise
    for a in W.forward_grid[1:]:
        ctx.hrt_step(a)
    ctx.hrt_sync_particles()
    disp0, mom0, _, _ = ctx.hrt_read_particles()
    grid = W.reverse_grid
    slots = {s: i for i, s in enumerate(W.source_steps)}
    # own kernels per ray step: the direct gather is one launch; the ray mesh is, per half shell, the projection
    # and the filter (around cuFFT's transforms), then the ray kernel
    ray_launches = 1
    if args.kick == "mesh":
        ctx.hrt_set_ray_mesh(raymesh_config(hrt, W))
        ray_launches = 5

    # the context sorts particles given by the caller before their first force, then every sort_every particle
    # steps (6 own launches: cell keys, three scan passes, inversion, gather)
    sort_every = 8 if args.sort_every is None else args.sort_every
    since_sort = [0]

    def reset():
        ctx.hrt_init_particles(disp0, mom0, 1.0)
        ctx.hrt_init_rays(theta0)
        since_sort[0] = 0

    reset.state = (disp0, mom0, theta0)

    def run_steps(k, start=0):
        """k reverse steps continuing at reverse index `start`, cycling through the reverse grid."""
        launches = 0
        pos = start
        for _ in range(k):
            if pos == len(grid) - 1:
                reset()
                launches += 3 + (6 if sort_every > 0 else 0)  # sort, CIC scatter, k-space pass, ray initialisation
                pos = 0
            n = pos + 1
            ctx.hrt_step(grid[n], slots.get(n, -1))
            launches += 2 + ray_launches  # ray step, kick-drift-deposit, k-space pass (x-pass on the split path)
            since_sort[0] += 1
            if sort_every > 0 and since_sort[0] >= sort_every:
                launches += 6
                since_sort[0] = 0
            pos = n
        return pos, launches

    reset()
    pos, _ = run_steps(args.warmup)
    reset()  # the timed run starts at a = 1 like the workload
    pos = 0
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    pos, launches = run_steps(args.steps, pos)
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    ms_max = max_over_ranks(t0.elapsed_time(t1), world, dev)
    value = replica_rate(args.steps, ms_max, world)

    # per-phase timing pass (CUDA events on the context stream around each kernel of the step)
    reset()
    ctx.hrt_ctx_set_profiling(True)
    run_steps(min(args.steps, len(grid) - 1), 0)
    phases = ctx.hrt_ctx_phase_times()
    ctx.hrt_ctx_set_profiling(False)

    # end-to-end through the C ABI with host buffers: the initial state goes in from pinned host memory through
    # hrt_init_particles / hrt_init_rays (their copies run inside the calls), and every step's result comes back
    # through hrt_read_rays_async into a pinned host buffer (the ray angles theta, i.e. the deflections), plus the
    # convergence map through hrt_read_kappa_async at source-plane steps; the copies overlap the next steps, and
    # hrt_read_wait inside the timed region waits for the last of them
    e2e = None
    if not args.no_e2e:
        disp_h = torch.empty(disp0.shape, dtype=torch.float32, pin_memory=True)
        mom_h = torch.empty(mom0.shape, dtype=torch.float32, pin_memory=True)
        disp_h.copy_(disp0)
        mom_h.copy_(mom0)
        th_h = theta0_h.contiguous().pin_memory()
        theta_out_h = torch.empty(W.n_rays, 2, dtype=torch.float64, pin_memory=True)
        kmaps_h = torch.empty(len(slots), W.n_rays, dtype=torch.float32, pin_memory=True)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h2d = d2h = 0
        p = len(grid) - 1
        for i in range(args.steps):
            if p == len(grid) - 1:
                ctx.hrt_init_particles(disp_h, mom_h, 1.0)
                ctx.hrt_init_rays(th_h)
                h2d += disp_h.numel() * 4 + mom_h.numel() * 4 + th_h.numel() * 8
                p = 0
            n = p + 1
            ctx.hrt_step(grid[n], slots.get(n, -1))
            # the step's results leave on the context's copy stream, beside the next step's kernels
            ctx.hrt_read_rays_async(theta_out_h)
            d2h += theta_out_h.numel() * 8
            if n in slots:
                ctx.hrt_read_kappa_async(slots[n], kmaps_h[slots[n]])
                d2h += W.n_rays * 4
            p = n
        ctx.hrt_read_wait()  # every step's copy has landed in host memory
        e1.record(stream)
        barrier()
        e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        assert bool(torch.isfinite(theta_out_h).all()), "non-finite ray angles read back"
        e2e = {"value": replica_rate(args.steps, e_ms, world), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
               "returned": "ray angles theta every step, kappa maps at source-plane steps (asynchronous "
                           "read-outs on the copy stream, all landed before the end of the timed region)"}

    # roofline of the dominant kernel of this library (by time in the phase pass)
    algo = algorithmic_bytes(W)
    if args.kick == "mesh":
        algo.pop("ray_step")   # the ray-mesh phase is mesh builds and FFTs, not the ray-state traffic
    own = {k: phases[k] for k in ("ray_step", "kick_drift", "cic_scatter", "kspace") if k in algo}
    dom = max(own, key=lambda k: own[k][0])
    t_ms, cnt = own[dom]
    peak, peak_kind = measured_peaks()
    achieved = algo[dom] / (t_ms / cnt / 1e3) / 1e9
    phase_summary = {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches": v[1],
                         "algo_GBps": (algo[k] / (v[0] / max(v[1], 1) / 1e3) / 1e9) if k in algo and v[1] else None}
                     for k, v in phases.items()}
    extra = None if args.no_next else next_rows(args, W, ctx, reset, grid, slots, run_steps, stream, seed)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 ray angles and time coefficients)",
        "data": "synthetic (seeded Gaussian ICs, power law x BBKS, sigma8 = 0.8)",
        "config": {"workload": W.name, "n_particles": W.n_side ** 3, "n_mesh": W.n_mesh, "box_mpc_h": W.box,
                   "n_rays": W.n_rays, "fov_deg": W.fov_deg, "reverse_steps": W.n_reverse,
                   "timed_steps_start_at_a": 1.0, "parallelism": f"replicas{world}",
                   "particle_sort_every": sort_every,
                   "deposit": {0: "per-particle", 1: "shared-memory tiles by row copies",
                               2: "shared-memory tiles by TMA"}[args.tiled_deposit],
                   "kick": ("ray mesh (iota %g, p_min %g)" % (RAYMESH_IOTA, RAYMESH_P_MIN)
                            if args.kick == "mesh" else "direct line-of-sight gather"),
                   "l2": "inputs larger than L2 (%.2g GB mesh per field)" % (W.n_mesh ** 3 * 4 / 1e9)},
        "clocks": clk, "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": recorded_traffic(dom, W.name), "algorithmic_bytes": algo[dom]},
        "phases": phase_summary,
        "next_rows": extra,
        "e2e": e2e,
    }
    return line


# ----------------------------------------------------------------------------------------------- widened rows
def next_rows(args, W, ctx, reset, grid, slots, run_steps, stream, seed):
    """Timings of the rows beyond the measured step, on the same workload and context: the ray step through a
    light cone tiled by rotated, translated replicas against the plain one (phase timing), the step with the
    accumulating readout of a source distribution, the ray-mesh kick operator against the direct gather
    (ray-step time and kappa power of full reverse runs), and 2LPT against Zel'dovich initial conditions."""
    import numpy as np
    import torch
    import synthetic
    from paper_2405_12913_gb300 import hrt
    steps = min(16, len(grid) - 1)
    out = {"steps": steps}
    ctx.hrt_set_ray_mesh(None)   # the rows below start from the direct gather
    # tiled light cone: enough replicas for the deepest node
    from paper_2405_12913_gb300.hrt import hrt_cosmo_eval
    n_rep = int(math.floor((W.observer[2] + hrt_cosmo_eval(W.omega_m, W.a_min)[1]) / W.box)) + 2
    ctx.hrt_set_replicas(synthetic.replica_transforms(seed, n_rep, W.n_mesh))
    reset()
    ctx.hrt_ctx_set_profiling(True)
    run_steps(steps, 0)
    ph = ctx.hrt_ctx_phase_times()
    ctx.hrt_ctx_set_profiling(False)
    ctx.hrt_set_replicas(None)
    out["tiled_ray_step_ms"] = ph["ray_step"][0] / max(ph["ray_step"][1], 1)
    out["replicas"] = n_rep
    # accumulated source distribution: every reverse step adds n_g(chi_n) O_n
    reset()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for n in range(1, steps + 1):
        ctx.hrt_step_accumulate(grid[n], 0, 1.0 / steps)
    e1.record(stream)
    torch.cuda.synchronize()
    out["accumulate_step_ms"] = e0.elapsed_time(e1) / steps
    # kappa power spectrum of one source map: a synchronous call (2D R2C plan, transform, binning, bins to the
    # host), timed on the host clock
    import time
    lmin, lmax = W.ell_range
    kmap = ctx.hrt_read_maps(0)[0].contiguous()
    hrt.hrt_kappa_power(kmap, W.n_pix, W.dtheta, W.nbins, lmin, lmax)
    torch.cuda.synchronize()
    reps_p = 10
    t_p = time.perf_counter()
    for _ in range(reps_p):
        hrt.hrt_kappa_power(kmap, W.n_pix, W.dtheta, W.nbins, lmin, lmax)
    out["kappa_power_call_ms"] = (time.perf_counter() - t_p) * 1e3 / reps_p
    # the paper's ray-mesh kick operator against the direct gather: full reverse runs from a = 1 on the same
    # particles, ray-step phase time and the kappa power spectra of every source plane
    lmin, lmax = W.ell_range
    runs = {}
    for name, cfg in (("direct", None), ("mesh", raymesh_config(hrt, W))):
        ctx.hrt_set_ray_mesh(cfg)
        reset()
        ctx.hrt_ctx_set_profiling(True)
        run_steps(len(grid) - 1, 0)
        ph = ctx.hrt_ctx_phase_times()
        ctx.hrt_ctx_set_profiling(False)
        pk = {s: ctx.hrt_ctx_kappa_power(i, W.n_pix, W.dtheta, W.nbins, lmin, lmax) for s, i in slots.items()}
        runs[name] = (ph["ray_step"][0] / max(ph["ray_step"][1], 1), pk)
    ctx.hrt_set_ray_mesh(None)
    # the paper's arrangement: the rays' 3D fields carry only the CIC deconvolution and the ray mesh does the
    # smoothing (separately filtered ray fields in a second context on the same particles)
    cfg2 = hrt.make_config(W.n_mesh, W.box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p, W.smooth_cells,
                           W.samples_per_cell, W.observer, n_sources=len(W.source_steps), ray_fields=2,
                           ray_deconv_p=W.deconv_p, ray_smooth_cells=0.0)
    ctx2 = hrt.Context(cfg2)
    # the hyper-parameters of the paper's ray-mesh tests (App. C): (iota, p_min) = (1, 4), (1, 256), (0.5, 256),
    # and a finer (0.25, 256)
    sweep = ((RAYMESH_IOTA, RAYMESH_P_MIN), (1.0, 4.0), (1.0, 256.0), (0.25, 256.0))
    sides = {"mesh": list(raymesh_sides(hrt, W))}
    for iota, p_min in sweep:
        ctx2.hrt_set_ray_mesh(raymesh_config(hrt, W, iota, p_min))
        ctx2.hrt_init_particles(*reset.state[:2], 1.0)
        ctx2.hrt_init_rays(reset.state[2])
        ctx2.hrt_ctx_set_profiling(True)
        for n in range(1, len(grid)):
            ctx2.hrt_step(grid[n], slots.get(n, -1))
        ph = ctx2.hrt_ctx_phase_times()
        ctx2.hrt_ctx_set_profiling(False)
        pk = {s: ctx2.hrt_ctx_kappa_power(i, W.n_pix, W.dtheta, W.nbins, lmin, lmax) for s, i in slots.items()}
        name = "mesh_unsmoothed_3d" if (iota, p_min) == sweep[0] else f"mesh_unsmoothed_3d_iota{iota:g}_p{p_min:g}"
        runs[name] = (ph["ray_step"][0] / max(ph["ray_step"][1], 1), pk)
        sides[name] = list(raymesh_sides(hrt, W, iota, p_min))
    ctx2.close()
    cmp = {"iota": RAYMESH_IOTA, "p_min": RAYMESH_P_MIN, "ray_mesh_sides": sides,
           "forms": {"direct": "direct gather of the 3D fields (Gaussian of 1 cell)",
                     "mesh": "ray mesh over the same fields (3D Gaussian and 2D Gaussian at lambda_lim)",
                     "mesh_unsmoothed_3d": "ray mesh over 3D fields without the Gaussian (the paper's arrangement)",
                     "mesh_unsmoothed_3d_iota*_p*": "the same with other (iota, p_min)"},
           "ray_step_ms": {k: v[0] for k, v in runs.items()}, "sources": {}}
    for s in W.source_steps:
        ell, p_d, cnt = runs["direct"][1][s]
        ok = cnt > 0
        e = ell[ok]
        row = {"ell": [round(float(x), 1) for x in e]}
        for name in [k for k in runs if k != "direct"]:
            ratio = runs[name][1][s][1][ok] / p_d[ok]
            row[f"power_ratio_{name}_over_direct"] = [round(float(x), 4) for x in ratio]
            for cut in (1200, 3000):
                row[f"{name}_max_dev_ell_le_{cut}"] = float(np.abs(ratio[e <= cut] - 1).max()) if (e <= cut).any() else None
        cmp["sources"][str(s)] = row
    out["kick_operators"] = cmp
    out["adjoint"] = adjoint_timing(hrt, seed)
    # initial conditions on the particle lattice
    noise = torch.from_numpy(synthetic.white_noise(seed, W.n_side).astype(np.float32)).cuda().reshape(-1)
    disp = torch.empty(3, W.n_side ** 3, device="cuda")
    mom = torch.empty_like(disp)
    for name, fn in (("zeldovich", hrt.hrt_ic_zeldovich), ("2lpt", hrt.hrt_ic_2lpt)):
        fn(noise, W.n_side, W.box, W.omega_m, W.h, W.n_s, W.sigma8, W.a_init, disp, mom)  # plans and memory
        torch.cuda.synchronize()
        e0.record(stream)
        fn(noise, W.n_side, W.box, W.omega_m, W.h, W.n_s, W.sigma8, W.a_init, disp, mom)
        e1.record(stream)
        torch.cuda.synchronize()
        out[f"ic_{name}_ms"] = e0.elapsed_time(e1)
    # the CIC deposit: plain reductions against warp-aggregated ones, on the ICs (a_init) and on the particles
    # at a = 1 (clustered)
    rho = torch.empty(W.n_mesh ** 3, device="cuda")
    hrt.hrt_ic_zeldovich(noise, W.n_side, W.box, W.omega_m, W.h, W.n_s, W.sigma8, W.a_init, disp, mom)
    states = {"a_init": disp, "a_1": reset.state[0]}
    dep = {}
    for tag, d in states.items():
        for name, fn in (("plain", hrt.hrt_cic_scatter), ("warp_aggregated", hrt.hrt_cic_scatter_warp_aggregated)):
            times = []
            for _ in range(5):
                e0.record(stream)
                fn(d, W.n_side, W.n_mesh, W.box, rho)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            dep[f"{tag}_{name}_ms"] = sorted(times)[2]
    out["cic_deposit"] = dep
    return out


def adjoint_timing(hrt, seed):
    """Gradient of a kappa-map loss with respect to the white noise and Omega_m by the context's native adjoint
    on the differentiation workload (128^3 particles, 256^3 mesh, 512^2 rays, 32 + 16 steps, checkpoint every
    4 steps): wall-clock of the recorded forward run and of hrt_adjoint."""
    import time
    import numpy as np
    import torch
    import synthetic
    from paper_2405_12913_gb300.configs import COSMO_GRAD_256 as G
    cfg = hrt.make_config(G.n_mesh, G.box, G.n_side, G.omega_m, G.h, G.n_s, G.sigma8, G.deconv_p, G.smooth_cells,
                          G.samples_per_cell, G.observer, n_sources=len(G.source_steps))
    ctx = hrt.Context(cfg)
    ctx.hrt_set_checkpointing(4)
    noise = torch.from_numpy(synthetic.white_noise(seed, G.n_side).astype(np.float32)).cuda().reshape(-1)
    theta0 = torch.from_numpy(synthetic.pixel_grid(G.n_pix, G.fov_deg * synthetic.DEGREE)).cuda()
    kbar = torch.from_numpy(synthetic.gaussian_field(seed + 1, (len(G.source_steps), G.n_rays)).astype(np.float32)).cuda()
    slots = {s: i for i, s in enumerate(G.source_steps)}
    out = {"workload": G.name, "checkpoint_every": 4}
    for rep in range(2):   # the first pass creates plans and memory pools
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.hrt_init_particles_zeldovich(noise, G.a_init)
        for a in G.forward_grid[1:]:
            ctx.hrt_step(a)
        ctx.hrt_sync_particles()
        ctx.hrt_init_rays(theta0)
        for n, a in enumerate(G.reverse_grid[1:], start=1):
            ctx.hrt_step(a, slots.get(n, -1))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, om_bar = ctx.hrt_adjoint(kbar)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out.update({"forward_s": t1 - t0, "adjoint_s": t2 - t1, "dL_dOmega_m": om_bar})
    ctx.close()
    return out


# ----------------------------------------------------------------------------------------------- learned form
LEARNED_256 = os.path.join(ROOT, "paper_2405_12913_gb300", "data", "ray_correction_256m.npy")
LEARNED_256_512 = os.path.join(ROOT, "paper_2405_12913_gb300", "data", "ray_correction_256m_512m.npy")
LEARNED_PARTICLE = os.path.join(ROOT, "paper_2405_12913_gb300", "data", "particle_correction_256m_512m.npy")


def learned_comparison(seeds=(100, 101, 102, 103)):
    """The learned ray-force correction against the plain kernel on the four held-out seeds of the coarse/fine pair
    workload (256^3 particles, box 256 Mpc/h, 4096^2 rays over 3.5 deg, source z = 1): the plain form on 256^3,
    512^3 and 768^3 meshes, the network trained on 256^3 pairs on the 256^3 mesh and the network trained on
    256^3 and 512^3 pairs on the 512^3 mesh, and the particle-force network (force matching on 256^3 and 512^3
    snapshots) on the 512^3 mesh, each against the plain 1024^3 run of the same seed: reverse
    co-evolution sim-steps/s (CUDA events, median over the seeds), the largest and the mean kappa P(ell) error over
    the seeds and the bins with ell <= 3000 (the range the networks were trained on) and ell <= 1e4, the largest
    error per bin, and the coarsest mesh of each form within 1 % in every bin on all four seeds (None: no mesh)."""
    import numpy as np
    import torch
    from dataclasses import replace
    from paper_2405_12913_gb300 import learned
    if not (os.path.exists(LEARNED_256) and os.path.exists(LEARNED_256_512)):
        return {"unavailable": "no trained parameters committed"}
    w256 = torch.tensor(np.load(LEARNED_256), dtype=torch.float32, device="cuda")
    w512 = torch.tensor(np.load(LEARNED_256_512), dtype=torch.float32, device="cuda")
    forms = [(256, w256, "learned (256^3 pairs)"), (512, w512, "learned (256^3 + 512^3 pairs)")]
    if os.path.exists(LEARNED_PARTICLE):
        wp = torch.tensor(np.load(LEARNED_PARTICLE), dtype=torch.float32, device="cuda")
        forms.append((512, None, "learned particle force (force matching)", wp))
    S = replace(learned.PairSpec(), n_pix=4096)
    res = learned.ladder_seeds(S, seeds, meshes=(256, 512, 768), cuts=(3000.0, S.ell_cut), log=lambda m: None,
                               learned_forms=forms)
    rows = res["forms"]
    fine = rows[0]["sim_steps_per_s"]
    return {"workload": "pair_256p_{256,512,768}m_vs_1024m_4096r", "seeds": list(seeds),
            "ell_cuts": [3000.0, S.ell_cut], "reference": "plain 1024^3 mesh, same seed", "forms": rows,
            "coarsest_mesh_within_1pct": res["coarsest_mesh_within_1pct"],
            "speed_over_fine": {f"{r['mesh']} {r['form']}": r["sim_steps_per_s"] / fine for r in rows[1:]}}


# ----------------------------------------------------------------------------------------------- oracle (CPU)
# The bounded sample of the workload the FP64 oracle steps through (particles per side, mesh side, rays per side):
# about a second of host work per step, extrapolated linearly in the work units to the full size.
ORACLE_SAMPLE = (128, 256, 512)


def oracle_sample(W, n_side, n_mesh, n_pix, seed=7):
    """Times one reverse sim-step of the FP64 oracle on a scaled copy of the workload (same box and field of
    view; particles, mesh and rays reduced), and extrapolates linearly in the work units to the full size.

    Returns (seconds per full-size step, sample description, threads, seconds of the sampled step itself)."""
    import numpy as np
    import torch
    import synthetic
    from oracle import cosmology as oc
    from oracle import pm as opm
    from oracle import rays as orays
    from oracle import sim as osim

    torch.set_num_threads(os.cpu_count() or 1)
    threads = torch.get_num_threads()
    om = W.omega_m
    grid = W.reverse_grid
    mid = len(grid) // 2
    a0, a1 = grid[mid], grid[mid + 1]
    q = opm.lattice(n_side, W.box)
    disp = torch.tensor(synthetic.small_displacements(seed, n_side, 2.0).T.copy())
    mom = torch.tensor(synthetic.small_displacements(seed + 1, n_side, 1.0).T.copy())
    flt = osim.Filter(W.deconv_p, W.smooth_cells)
    t = time.perf_counter()
    rho = opm.cic_deposit(q + disp, W.box, n_mesh)
    grads = opm.poisson_gradient(rho, W.box, 1.5 * om / a0, flt.deconv_p, flt.smooth_cells * W.box / n_mesh)
    kick = oc.kick_integral(a0, 0.5 * (a0 + a1), om)
    drift = oc.drift_integral(a0, a1, om)
    opm.particle_kick_drift(disp, mom, q, grads, W.box, kick, drift)
    t_pm = time.perf_counter() - t
    theta0 = torch.tensor(synthetic.pixel_grid(n_pix, W.fov_deg * synthetic.DEGREE))
    st = orays.init_state(theta0)
    c0, c1 = oc.chi_of_a(a0, om), oc.chi_of_a(a1, om)
    t = time.perf_counter()
    orays.ray_step(st, grads[0], grads[1], W.box, W.observer, c0, c1, W.samples_per_cell,
                   osim.growth_weight(a0, om))
    t_ray = time.perf_counter() - t
    # work units: particles + mesh cells for the PM part, ray-node evaluations for the rays
    ratio_pm = (W.n_side / n_side) ** 3
    cell_s, cell_f = W.box / n_mesh, W.box / W.n_mesh
    nodes_s = math.ceil(abs(c1 - c0) / 2 / cell_s) * 2
    nodes_f = math.ceil(abs(c1 - c0) / 2 / cell_f) * 2
    ratio_ray = (W.n_rays / n_pix ** 2) * (nodes_f / nodes_s)
    full = t_pm * ratio_pm + t_ray * ratio_ray
    desc = (f"one reverse step (a {a0:.4f}->{a1:.4f}) at {n_side}^3 particles, {n_mesh}^3 mesh, {n_pix}^2 rays "
            f"({t_pm:.2f} s PM + {t_ray:.2f} s rays), scaled x{ratio_pm:.0f} (particles, cells) and "
            f"x{ratio_ray:.0f} (ray-node samples) to the full workload")
    return full, desc, threads, t_pm + t_ray


def run_reference(args, W, rank):
    if rank != 0:
        return None
    sizes = ORACLE_SAMPLE  # n_side, n_mesh, n_pix per sampled step
    for _ in range(args.warmup):
        oracle_sample(W, *sizes)
    per, own = [], []
    desc = threads = None
    for i in range(args.steps):
        full, desc, threads, t_sample = oracle_sample(W, *sizes, seed=100 + i)
        per.append(full)
        own.append(t_sample)
    sec = sum(per) / len(per)
    value = 1.0 / sec
    n_side, n_mesh, n_pix = sizes
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": W.name, "parallelism": "cpu"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
                         "measured_at_sample_size": {
                             "value": len(own) / sum(own), "unit": UNIT,
                             "workload": f"{n_side}^3 particles, {n_mesh}^3 mesh, {n_pix}^2 rays (timed directly)"}},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def precision_errors():
    """Per-output error of the GPU path against the FP64 oracle on the 1024^3 workload's recipe scaled to 128^3
    particles, 256^3 mesh and 512^2 rays (the oracle's outputs are the ones stored by
    tests/golden/make_cosmo_1024_recipe_128p.py), for the method as built (FP64 ray angles and positions, FP32
    mesh, FFT and gathers) and for the FP32 ray-angle ablation.  Deflections: |theta - theta_oracle| over the
    largest deflection; maps: |error| over the rms of the oracle's kappa map; P(ell): relative error per bin."""
    import numpy as np
    import torch
    from paper_2405_12913_gb300 import hrt
    from paper_2405_12913_gb300.configs import COSMO_1024_SCALED as W
    import synthetic
    g = np.load(os.path.join(ROOT, "tests", "golden", "cosmo_1024_recipe_128p.npz"))
    noise = torch.tensor(synthetic.white_noise(W.seed, W.n_side), dtype=torch.float32, device="cuda")
    theta0 = torch.tensor(synthetic.pixel_grid(W.n_pix, W.fov_deg * synthetic.DEGREE), device="cuda")
    slots = {s: i for i, s in enumerate(W.source_steps)}
    ir = g["ray_index"]
    lmin, lmax = W.ell_range
    out = {"workload": W.name, "reference": "FP64 oracle (stored outputs at 4096 sampled rays; all P(ell) bins)"}
    for bits in (64, 32):
        cfg = hrt.make_config(W.n_mesh, W.box, W.n_side, W.omega_m, W.h, W.n_s, W.sigma8, W.deconv_p,
                              W.smooth_cells, W.samples_per_cell, W.observer, n_sources=len(W.source_steps))
        ctx = hrt.Context(cfg)
        ctx.hrt_set_ray_theta_bits(bits)
        ctx.hrt_init_particles_zeldovich(noise, W.a_init)
        for a in W.forward_grid[1:]:
            ctx.hrt_step(a)
        ctx.hrt_init_rays(theta0)
        for n, a in enumerate(W.reverse_grid[1:], start=1):
            ctx.hrt_step(a, slots.get(n, -1))
        th = ctx.hrt_read_rays()[0].cpu().numpy()
        row = {}
        d = np.abs(th[ir] - g["theta"]).max(axis=1) / float(g["alpha_absmax"])
        row["deflection"] = {"max": float(d.max()), "median": float(np.median(d))}
        for s, i in slots.items():
            maps = ctx.hrt_read_maps(i).cpu().double().numpy()[:, ir]
            rms = float(g[f"kappa_rms_{s}"])
            per = {}
            for k, name in enumerate(("kappa", "gamma1", "gamma2", "omega")):
                e = np.abs(maps[k] - g[f"maps_{s}"][k]) / rms
                per[name] = {"max": float(e.max()), "p99": float(np.quantile(e, 0.99)), "median": float(np.median(e))}
            _, p, cnt = ctx.hrt_ctx_kappa_power(i, W.n_pix, W.dtheta, W.nbins, lmin, lmax)
            ok = cnt > 0
            rel = np.abs(p[ok] / g[f"power_{s}"][ok] - 1.0)
            per["power_per_bin"] = [float(x) for x in rel]
            per["power_max"] = float(rel.max())
            row[f"source_step_{s}"] = per
        ctx.close()
        out["fp64_angles" if bits == 64 else "fp32_angles_ablation"] = row
    return out


def main():
    args = parse()
    world, rank, local = dist_env()
    from paper_2405_12913_gb300.configs import WORKLOADS
    W = WORKLOADS[args.workload]
    if args.impl == "reference":
        line = run_reference(args, W, rank)
        if line is not None:
            print(json.dumps(line))
        return 0
    line = run_gpu(args, W, world, rank, local)
    if line is None:
        return 0
    if world == 1 and not args.no_precision:
        line["precision"] = precision_errors()
    if world == 1 and not args.no_learned:
        line["learned"] = learned_comparison()
    if world == 1 and not args.no_cpu_baseline:
        full, desc, threads, t_sample = oracle_sample(W, *ORACLE_SAMPLE)
        n_side, n_mesh, n_pix = ORACLE_SAMPLE
        line["cpu_baseline"] = {"value": 1.0 / full, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": desc,
                                "measured_at_sample_size": {
                                    "value": 1.0 / t_sample, "unit": UNIT,
                                    "workload": f"{n_side}^3 particles, {n_mesh}^3 mesh, {n_pix}^2 rays (timed directly)"}}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
