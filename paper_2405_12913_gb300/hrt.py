"""Thin Python binding of the C ABI in ``include/hrt.h`` (argument marshalling only).

Every function keeps the C name and forwards torch CUDA tensors as raw device pointers on the current torch
stream (or an explicit ``stream``).  All arithmetic happens in ``libhrt.so``; if the library is missing the
import of this module raises, so there is no silent CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhrt.so")

HRT_OK = 0
STATUS_NAMES = {0: "HRT_OK", 1: "HRT_ERR_INVALID_ARG", 2: "HRT_ERR_OOM", 3: "HRT_ERR_CUDA", 4: "HRT_ERR_STATE",
                5: "HRT_ERR_NONFINITE", 6: "HRT_ERR_TIMEOUT"}


class HRTError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class hrt_filter(C.Structure):
    _fields_ = [("deconv_p", C.c_double), ("smooth", C.c_double), ("g_table", C.c_void_p), ("g_nk", C.c_int32),
                ("g_kmax", C.c_double)]


class hrt_rays(C.Structure):
    _fields_ = [("theta", C.c_void_p), ("eta", C.c_void_p), ("A", C.c_void_p), ("B", C.c_void_p),
                ("n_rays", C.c_int64)]


class hrt_ray_geom(C.Structure):
    _fields_ = [("n", C.c_int64), ("box", C.c_double), ("observer", C.c_double * 3),
                ("samples_per_cell", C.c_double), ("window_lo", C.c_double), ("window_hi", C.c_double),
                ("image_width", C.c_int64), ("n_replicas", C.c_int32), ("replica_perm", C.c_void_p),
                ("replica_sign", C.c_void_p), ("replica_shift", C.c_void_p)]


class hrt_raymesh_config(C.Structure):
    _fields_ = [("iota", C.c_double), ("p_min", C.c_double), ("mu", C.c_double), ("m_pix", C.c_int64),
                ("n2d_max", C.c_int64)]


class hrt_cosmology(C.Structure):
    _fields_ = [("omega_m", C.c_double), ("h", C.c_double), ("n_s", C.c_double), ("sigma8", C.c_double)]


class hrt_config(C.Structure):
    _fields_ = [("n_mesh", C.c_int64), ("box", C.c_double), ("n_side", C.c_int64), ("cosmo", hrt_cosmology),
                ("deconv_p", C.c_double), ("smooth_cells", C.c_double), ("samples_per_cell", C.c_double),
                ("observer", C.c_double * 3), ("static_mode", C.c_int32), ("static_pref", C.c_double),
                ("window_lo", C.c_double), ("window_hi", C.c_double), ("n_sources", C.c_int32),
                ("ray_fields", C.c_int32), ("ray_deconv_p", C.c_double), ("ray_smooth_cells", C.c_double)]


_P = C.c_void_p
_D = C.c_double
_I64 = C.c_int64
_I32 = C.c_int32
_SIGS = {
    "hrt_status_string": ([C.c_int], C.c_char_p),
    "hrt_last_error": ([], C.c_char_p),
    "hrt_cosmo_eval": ([_D, _D, _P], C.c_int),
    "hrt_cosmo_time_integrals": ([_D, _D, _D, _P], C.c_int),
    "hrt_cosmo_a_of_chi": ([_D, _D, _P], C.c_int),
    "hrt_cosmo_power_amplitude": ([_D, _D, _D, _D, _P], C.c_int),
    "hrt_cic_scatter": ([_P, _I64, _I64, _D, _P, _P], C.c_int),
    "hrt_cic_scatter_warp_aggregated": ([_P, _I64, _I64, _D, _P, _P], C.c_int),
    "hrt_particle_kick_drift": ([_P, _I64, _D, _I64, _P, _P, _D, _D, _P], C.c_int),
    "hrt_particle_kick_drift_deposit": ([_P, _I64, _D, _I64, _P, _P, _D, _D, _P, _P], C.c_int),
    "hrt_particle_kick_drift_deposit_bricks": ([_P, _I64, _D, _I64, _P, _P, _P, _P, _D, _D, _P, _P], C.c_int),
    "hrt_kspace_gradient": ([_P, _I64, _D, _D, _P, _I32, _P, _P, _I32, _P, _P], C.c_int),
    "hrt_kspace_gradient_noalloc": ([_P, _I64, _D, _D, _P, _I32, _P, _P, _I32, _P, _P], C.c_int),
    "hrt_pm_create": ([_I64, _D, _I32, _P, _P], C.c_int),
    "hrt_pm_destroy": ([_P], C.c_int),
    "hrt_pm_solve": ([_P, _P, _D, _P, _P, _P, _P], C.c_int),
    "hrt_pm_set_fused": ([_P, _I32], C.c_int),
    "hrt_pm_set_split": ([_P, _I32], C.c_int),
    "hrt_rays_init": ([_P, _P, _P], C.c_int),
    "hrt_ray_step": ([_P, _P, _P, _P, _D, _D, _D, _D, _P, _P], C.c_int),
    "hrt_ray_step_tiled": ([_P, _P, _P, _P, _P, _D, _D, _D, _D, _P, _P], C.c_int),
    "hrt_set_replicas": ([_P, _I32, _P, _P, _P], C.c_int),
    "hrt_raymesh_geometry": ([_P, _D, _D, _D, _P, _P, _P], C.c_int),
    "hrt_raymesh_create": ([_P, _P], C.c_int),
    "hrt_raymesh_destroy": ([_P], C.c_int),
    "hrt_raymesh_kick": ([_P, _P, _P, _P, _D, _D, _D, _D, _P, _P], C.c_int),
    "hrt_raymesh_ray_step": ([_P, _P, _P, _P, _P, _D, _D, _D, _D, _P, _P], C.c_int),
    "hrt_raymesh_kick_tiled": ([_P, _P, _P, _P, _P, _D, _D, _D, _D, _P, _P], C.c_int),
    "hrt_raymesh_kick_adjoint": ([_P, _P, _P, _P, _P, _D, _D, _D, _D, _P, _P, _P, _P], C.c_int),
    "hrt_raymesh_ray_step_adjoint": ([_P, _P, _P, _P, _P, _D, _D, _D, _D, _P, _P, _P, _P, _P, _P], C.c_int),
    "hrt_raymesh_kick_tiled_adjoint": ([_P, _P, _P, _P, _P, _P, _D, _D, _D, _D, _P, _P, _P, _P, _P], C.c_int),
    "hrt_raymesh_ray_step_tiled_adjoint": ([_P, _P, _P, _P, _P, _P, _D, _D, _D, _D, _P, _P, _P, _P, _P, _P, _P],
                                           C.c_int),
    "hrt_raymesh_step_planes": ([_P, _P, _D, _D, _D, _D, _P, _P, _P, _P, _P], C.c_int),
    "hrt_raymesh_ray_step_tiled": ([_P, _P, _P, _P, _P, _P, _D, _D, _D, _D, _P, _P], C.c_int),
    "hrt_set_ray_mesh": ([_P, _P], C.c_int),
    "hrt_set_checkpointing": ([_P, _I32], C.c_int),
    "hrt_set_particle_sort": ([_P, _I32], C.c_int),
    "hrt_set_tiled_deposit": ([_P, _I32], C.c_int),
    "hrt_adjoint": ([_P, _P, _P, _P, _P], C.c_int),
    "hrt_ray_drift_free": ([_P, _D, _D, _P], C.c_int),
    "hrt_ray_readout": ([_P, _P, _P], C.c_int),
    "hrt_kappa_power": ([_P, _I64, _D, _I32, _D, _D, _P, _P, _P, _P], C.c_int),
    "hrt_ic_zeldovich": ([_P, _I64, _D, _P, _D, _P, _P, _P], C.c_int),
    "hrt_ic_2lpt": ([_P, _I64, _D, _P, _D, _P, _P, _P], C.c_int),
    "hrt_ic_2lpt_adjoint": ([_P, _I64, _D, _P, _D, _P, _P, _P, _P, _P, _P], C.c_int),
    "hrt_ic_2lpt_coefficients": ([_P, _D, _P], C.c_int),
    "hrt_init_particles_2lpt": ([_P, _P, _D], C.c_int),
    "hrt_create": ([_P, _P, _P], C.c_int),
    "hrt_destroy": ([_P], C.c_int),
    "hrt_workspace_bytes": ([_P, _I64, _P], C.c_int),
    "hrt_init_particles_zeldovich": ([_P, _P, _D], C.c_int),
    "hrt_init_particles": ([_P, _P, _P, _D], C.c_int),
    "hrt_init_rays": ([_P, _P, _I64], C.c_int),
    "hrt_step": ([_P, _D, _I32], C.c_int),
    "hrt_sync_particles": ([_P], C.c_int),
    "hrt_set_ray_correction": ([_P, _P], C.c_int),
    "hrt_step_accumulate": ([_P, C.c_double, _I32, C.c_double], C.c_int),
    "hrt_set_ray_kernel_table": ([_P, _P, _I32, C.c_double], C.c_int),
    "hrt_state_bytes": ([_P, _P], C.c_int),
    "hrt_save_state": ([_P, _P, C.c_size_t], C.c_int),
    "hrt_load_state": ([_P, _P, C.c_size_t], C.c_int),
    "hrt_step_static": ([_P, _D, _D, _I32], C.c_int),
    "hrt_drift_free": ([_P, _D, _D], C.c_int),
    "hrt_read_rays": ([_P, _P, _P, _P, _P], C.c_int),
    "hrt_read_maps": ([_P, _I32, _P, _P, _P, _P], C.c_int),
    "hrt_read_rays_async": ([_P, _P], C.c_int),
    "hrt_read_kappa_async": ([_P, _I32, _P], C.c_int),
    "hrt_read_wait": ([_P], C.c_int),
    "hrt_read_particles": ([_P, _P, _P, _P, _P], C.c_int),
    "hrt_read_grad": ([_P, _P], C.c_int),
    "hrt_ctx_kappa_power": ([_P, _I32, _I64, _D, _I32, _D, _D, _P, _P, _P], C.c_int),
    "hrt_cic_scatter_adjoint": ([_P, _P, _I64, _I64, _D, _P, _P], C.c_int),
    "hrt_particle_kick_drift_adjoint": ([_P, _I64, _D, _I64, _P, _P, _D, _D, _P, _P, _P, _P, _P, _P], C.c_int),
    "hrt_pm_solve_adjoint": ([_P, _P, _D, _P, _P, _P, _P], C.c_int),
    "hrt_ray_step_adjoint": ([_P, _P, _P, _P, _D, _D, _D, _D, _P, _P, _P, _P, _P, _P], C.c_int),
    "hrt_ray_step_tiled_adjoint": ([_P, _P, _P, _P, _P, _D, _D, _D, _D, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "hrt_ray_step_coefficients": ([_P, _D, _D, _D, _D, _P, _P, _P, _P, _P, _P], C.c_int),
    "hrt_kappa_power_adjoint": ([_P, _I64, _D, _I32, _D, _D, _P, _P, _P], C.c_int),
    "hrt_ic_table": ([_I64, _D, _P, _D, _P, _P], C.c_int),
    "hrt_ic_zeldovich_adjoint": ([_P, _I64, _D, _P, _D, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "hrt_dot": ([_P, _P, _I64, _P, _P], C.c_int),
    "hrt_mlp_forward": ([_P, _I32, _P, _P, _P, _P], C.c_int),
    "hrt_mlp_backward": ([_P, _I32, _P, _P, _P, _P, _P], C.c_int),
    "hrt_mlp_adam": ([_P, _P, _P, _P, _P, _D, _D, _D, _D, _I32, _P], C.c_int),
    "hrt_mlp_to_bf16": ([_P, _P, _P], C.c_int),
    "hrt_kspace_table_adjoint": ([_P, _I32, _P, _I64, _D, _D, _P, _P, _P], C.c_int),
    "hrt_pm_density_spectrum": ([_P, _P], C.c_int),
    "hrt_pm_gradient_from_spectrum": ([_P, _P, _D, _P, _I32, _P], C.c_int),
    "hrt_pm_forward_fft": ([_P, _P, _P], C.c_int),
    "hrt_ctx_set_profiling": ([_P, _I32], C.c_int),
    "hrt_set_nonfinite_check": ([_P, _I32], C.c_int),
    "hrt_set_host_wait_limit": ([_D], C.c_int),
    "hrt_inject_alloc_failure": ([_I64], C.c_int),
    "hrt_set_ray_theta_bits": ([_P, _I32], C.c_int),
    "hrt_set_particle_correction": ([_P, _P], C.c_int),
    "hrt_static_prefactor": ([_D, _D, _P], C.c_int),
    "hrt_ctx_phase_times": ([_P, _P, _P], C.c_int),
    "hrt_ctx_rays": ([_P, _P], C.c_int),
}
EXPORTED = tuple(_SIGS)


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def _check(status: int, where: str) -> None:
    if status != HRT_OK:
        raise HRTError(status, where, _lib.hrt_last_error().decode())


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None, dtype=None, name: str = "tensor") -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def _host_ptr(t: torch.Tensor, dtype, name: str) -> int:
    """Pointer of a contiguous host tensor (for the asynchronous read-outs)."""
    if t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def _any_ptr(t: torch.Tensor | None, dtype, name: str) -> int | None:
    """Pointer of a contiguous tensor in device or host memory (for calls that copy with either)."""
    if t is None:
        return None
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor")
    return t.data_ptr()


def _host_ptr(t: torch.Tensor | None, dtype, name: str) -> int | None:
    if t is None:
        return None
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous host {dtype} tensor")
    return t.data_ptr()


def hrt_set_host_wait_limit(seconds: float):
    """Process-wide limit of the library's host waits for a stream (<= 0: none)."""
    _check(_lib.hrt_set_host_wait_limit(seconds), "hrt_set_host_wait_limit")


def hrt_static_prefactor(mass: float, box: float) -> float:
    """4 pi G M / box^3: the Poisson prefactor of a static lens of mass M (Msun/h) in a box of side L (Mpc/h)."""
    out = C.c_double()
    _check(_lib.hrt_static_prefactor(mass, box, C.byref(out)), "hrt_static_prefactor")
    return out.value


def hrt_inject_alloc_failure(k: int):
    """Test hook: the k-th device allocation of the library from now reports out-of-memory (0: off)."""
    _check(_lib.hrt_inject_alloc_failure(k), "hrt_inject_alloc_failure")


def status_string(status: int) -> str:
    return _lib.hrt_status_string(status).decode()


# ------------------------------------------------------------------------------------------------ cosmology
def hrt_cosmo_eval(omega_m: float, a: float):
    out = (C.c_double * 4)()
    _check(_lib.hrt_cosmo_eval(omega_m, a, out), "hrt_cosmo_eval")
    return tuple(out)


def hrt_cosmo_time_integrals(omega_m: float, a: float, b: float):
    out = (C.c_double * 2)()
    _check(_lib.hrt_cosmo_time_integrals(omega_m, a, b, out), "hrt_cosmo_time_integrals")
    return tuple(out)


def hrt_cosmo_a_of_chi(omega_m: float, chi: float) -> float:
    out = C.c_double()
    _check(_lib.hrt_cosmo_a_of_chi(omega_m, chi, C.byref(out)), "hrt_cosmo_a_of_chi")
    return out.value


def hrt_cosmo_power_amplitude(omega_m: float, h: float, n_s: float, sigma8: float) -> float:
    out = C.c_double()
    _check(_lib.hrt_cosmo_power_amplitude(omega_m, h, n_s, sigma8, C.byref(out)), "hrt_cosmo_power_amplitude")
    return out.value


# ------------------------------------------------------------------------------------------------ mesh kernels
def make_filter(deconv_p: float = 0.0, smooth: float = 0.0, g_table: torch.Tensor | None = None,
                g_kmax: float = 0.0) -> hrt_filter:
    f = hrt_filter()
    f.deconv_p = deconv_p
    f.smooth = smooth
    if g_table is not None:
        f.g_table = _ptr(g_table, torch.float32, "g_table")
        f.g_nk = g_table.numel()
        f.g_kmax = g_kmax
    return f


def hrt_cic_scatter(disp: torch.Tensor, n_side: int, n: int, box: float, rho: torch.Tensor, stream=None):
    _check(_lib.hrt_cic_scatter(_ptr(disp, torch.float32, "disp"), n_side, n, box, _ptr(rho, torch.float32, "rho"),
                                _stream(stream)), "hrt_cic_scatter")


def hrt_cic_scatter_warp_aggregated(disp: torch.Tensor, n_side: int, n: int, box: float, rho: torch.Tensor,
                                    stream=None):
    _check(_lib.hrt_cic_scatter_warp_aggregated(_ptr(disp, torch.float32, "disp"), n_side, n, box,
                                                _ptr(rho, torch.float32, "rho"), _stream(stream)),
           "hrt_cic_scatter_warp_aggregated")


def hrt_particle_kick_drift(grad: torch.Tensor, n: int, box: float, n_side: int, disp: torch.Tensor,
                            mom: torch.Tensor, kick: float, drift: float, stream=None):
    _check(_lib.hrt_particle_kick_drift(_ptr(grad, torch.float32, "grad"), n, box, n_side,
                                        _ptr(disp, torch.float32, "disp"), _ptr(mom, torch.float32, "mom"), kick,
                                        drift, _stream(stream)), "hrt_particle_kick_drift")


def hrt_particle_kick_drift_deposit(grad: torch.Tensor, n: int, box: float, n_side: int, disp: torch.Tensor,
                                    mom: torch.Tensor, kick: float, drift: float, rho: torch.Tensor, stream=None):
    _check(_lib.hrt_particle_kick_drift_deposit(_ptr(grad, torch.float32, "grad"), n, box, n_side,
                                                _ptr(disp, torch.float32, "disp"), _ptr(mom, torch.float32, "mom"),
                                                kick, drift, _ptr(rho, torch.float32, "rho"), _stream(stream)),
           "hrt_particle_kick_drift_deposit")


def hrt_particle_kick_drift_deposit_bricks(grad: torch.Tensor, n: int, box: float, n_side: int, disp: torch.Tensor,
                                           mom: torch.Tensor, order: torch.Tensor, key_start: torch.Tensor,
                                           kick: float, drift: float, rho: torch.Tensor, stream=None):
    _check(_lib.hrt_particle_kick_drift_deposit_bricks(
        _ptr(grad, torch.float32, "grad"), n, box, n_side, _ptr(disp, torch.float32, "disp"),
        _ptr(mom, torch.float32, "mom"), _ptr(order, torch.int32, "order"), _ptr(key_start, torch.int32, "key_start"),
        kick, drift, _ptr(rho, torch.float32, "rho"), _stream(stream)), "hrt_particle_kick_drift_deposit_bricks")


def hrt_kspace_gradient(rho_hat: torch.Tensor, n: int, box: float, pref: float, f: hrt_filter, n_out: int,
                        out: torch.Tensor, f2: hrt_filter | None = None, n_second: int = 0,
                        second: torch.Tensor | None = None, stream=None):
    _check(_lib.hrt_kspace_gradient(_ptr(rho_hat, torch.complex64, "rho_hat"), n, box, pref, C.byref(f), n_out,
                                    _ptr(out, torch.complex64, "out"), C.byref(f2) if f2 is not None else None,
                                    n_second, _ptr(second, torch.complex64, "second"), _stream(stream)),
           "hrt_kspace_gradient")


def hrt_kspace_gradient_noalloc(rho_hat: torch.Tensor, n: int, box: float, pref: float, f: hrt_filter, n_out: int,
                                out: torch.Tensor, f2: hrt_filter | None = None, n_second: int = 0,
                                second: torch.Tensor | None = None, stream=None):
    """``hrt_kspace_gradient`` for callers that may not allocate device memory (fixed tables, n <= 2048)."""
    _check(_lib.hrt_kspace_gradient_noalloc(_ptr(rho_hat, torch.complex64, "rho_hat"), n, box, pref, C.byref(f),
                                            n_out, _ptr(out, torch.complex64, "out"),
                                            C.byref(f2) if f2 is not None else None, n_second,
                                            _ptr(second, torch.complex64, "second"), _stream(stream)),
           "hrt_kspace_gradient_noalloc")


class PM:
    """Owner of an ``hrt_pm`` object (cuFFT plans and spectra for one mesh size)."""

    def __init__(self, n: int, box: float, n_ray_fields: int = 0, stream=None):
        self._h = C.c_void_p()
        _check(_lib.hrt_pm_create(n, box, n_ray_fields, _stream(stream), C.byref(self._h)), "hrt_pm_create")
        self.n, self.box = n, box

    def solve(self, rho: torch.Tensor, pref: float, f: hrt_filter, grad: torch.Tensor,
              f_ray: hrt_filter | None = None, ray_grad: torch.Tensor | None = None):
        _check(_lib.hrt_pm_solve(self._h, _ptr(rho, torch.float32, "rho"), pref, C.byref(f),
                                 _ptr(grad, torch.float32, "grad"), C.byref(f_ray) if f_ray is not None else None,
                                 _ptr(ray_grad, torch.float32, "ray_grad")), "hrt_pm_solve")

    def solve_adjoint(self, grad_bar: torch.Tensor, pref: float, f: hrt_filter, rho_bar: torch.Tensor,
                      ray_grad_bar: torch.Tensor | None = None, f_ray: hrt_filter | None = None):
        _check(_lib.hrt_pm_solve_adjoint(self._h, _ptr(grad_bar, torch.float32, "grad_bar"), pref, C.byref(f),
                                         _ptr(ray_grad_bar, torch.float32, "ray_grad_bar"),
                                         C.byref(f_ray) if f_ray is not None else None,
                                         _ptr(rho_bar, torch.float32, "rho_bar")), "hrt_pm_solve_adjoint")

    def density_spectrum(self, out: torch.Tensor):
        _check(_lib.hrt_pm_density_spectrum(self._h, _ptr(out, torch.complex64, "out")), "hrt_pm_density_spectrum")

    def gradient_from_spectrum(self, rho_hat: torch.Tensor, pref: float, f: hrt_filter, n_out: int,
                               fields: torch.Tensor):
        _check(_lib.hrt_pm_gradient_from_spectrum(self._h, _ptr(rho_hat, torch.complex64, "rho_hat"), pref,
                                                  C.byref(f), n_out, _ptr(fields, torch.float32, "fields")),
               "hrt_pm_gradient_from_spectrum")

    def forward_fft(self, real: torch.Tensor, out: torch.Tensor):
        _check(_lib.hrt_pm_forward_fft(self._h, _ptr(real, torch.float32, "real"), _ptr(out, torch.complex64, "out")),
               "hrt_pm_forward_fft")

    def set_fused(self, on: bool):
        _check(_lib.hrt_pm_set_fused(self._h, int(on)), "hrt_pm_set_fused")

    def set_split(self, on: bool):
        _check(_lib.hrt_pm_set_split(self._h, int(on)), "hrt_pm_set_split")

    def close(self):
        if self._h:
            _lib.hrt_pm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


# ------------------------------------------------------------------------------------------------ rays
class RayState:
    """Caller-owned device ray state (theta f64 [R,2], eta f32 [R,2], A, B f32 [R,4])."""

    def __init__(self, n_rays: int, device="cuda"):
        self.theta = torch.empty(n_rays, 2, dtype=torch.float64, device=device)
        self.eta = torch.empty(n_rays, 2, dtype=torch.float32, device=device)
        self.A = torch.empty(n_rays, 4, dtype=torch.float32, device=device)
        self.B = torch.empty(n_rays, 4, dtype=torch.float32, device=device)
        self.n_rays = n_rays

    def c(self) -> hrt_rays:
        r = hrt_rays()
        r.theta, r.eta, r.A, r.B = self.theta.data_ptr(), self.eta.data_ptr(), self.A.data_ptr(), self.B.data_ptr()
        r.n_rays = self.n_rays
        return r


def make_geom(n: int, box: float, observer, samples_per_cell: float = 1.0, window=(-1e300, 1e300),
              image_width: int = 0, replicas=None) -> hrt_ray_geom:
    """Ray geometry; ``replicas`` = (perm, sign, shift) [k][3] integer arrays tile the light cone."""
    g = hrt_ray_geom()
    g.image_width = image_width
    if replicas is not None:
        import numpy as np
        g._tables = [np.ascontiguousarray(t, dtype=np.int32) for t in replicas]  # kept alive with the struct
        g.n_replicas = g._tables[0].shape[0]
        g.replica_perm, g.replica_sign, g.replica_shift = (t.ctypes.data for t in g._tables)
    g.n, g.box = n, box
    for i in range(3):
        g.observer[i] = observer[i]
    g.samples_per_cell = samples_per_cell
    g.window_lo, g.window_hi = window
    return g


def hrt_rays_init(rays: RayState, theta0: torch.Tensor, stream=None):
    r = rays.c()
    _check(_lib.hrt_rays_init(C.byref(r), _ptr(theta0, torch.float64, "theta0"), _stream(stream)), "hrt_rays_init")


def hrt_ray_step(rays: RayState, grad_x: torch.Tensor, grad_y: torch.Tensor, geom: hrt_ray_geom, chi_from: float,
                 chi_to: float, a_ref: float = 0.0, omega_m: float = 0.3, maps: torch.Tensor | None = None,
                 stream=None):
    r = rays.c()
    _check(_lib.hrt_ray_step(C.byref(r), _ptr(grad_x, torch.float32, "grad_x"), _ptr(grad_y, torch.float32, "grad_y"),
                             C.byref(geom), chi_from, chi_to, a_ref, omega_m, _ptr(maps, torch.float32, "maps"),
                             _stream(stream)), "hrt_ray_step")


def hrt_ray_step_tiled(rays: RayState, grad: torch.Tensor, geom: hrt_ray_geom, chi_from: float, chi_to: float,
                       a_ref: float = 0.0, omega_m: float = 0.3, maps: torch.Tensor | None = None, stream=None):
    """hrt_ray_step through the tiled light cone of geom; grad holds the three gradient fields [3][n^3]."""
    r = rays.c()
    g = grad.reshape(3, -1)
    _check(_lib.hrt_ray_step_tiled(C.byref(r), _ptr(g[0], torch.float32, "grad_x"), _ptr(g[1], torch.float32, "grad_y"),
                                   _ptr(g[2], torch.float32, "grad_z"), C.byref(geom), chi_from, chi_to, a_ref, omega_m,
                                   _ptr(maps, torch.float32, "maps"), _stream(stream)), "hrt_ray_step_tiled")


def make_raymesh_config(iota: float, p_min: float, mu: float, m_pix: int, n2d_max: int = 0) -> hrt_raymesh_config:
    return hrt_raymesh_config(iota, p_min, mu, m_pix, n2d_max)


def hrt_raymesh_geometry(cfg: hrt_raymesh_config, chi_a: float, chi_b: float, cell: float):
    """(lambda_lim, x2d, N) of the ray mesh of the half shell [chi_a, chi_b)."""
    lam, x2d, n2d = C.c_double(), C.c_double(), C.c_int64()
    _check(_lib.hrt_raymesh_geometry(C.byref(cfg), chi_a, chi_b, cell, C.byref(lam), C.byref(x2d), C.byref(n2d)),
           "hrt_raymesh_geometry")
    return lam.value, x2d.value, n2d.value


def hrt_raymesh_step_planes(cfg: hrt_raymesh_config, geom: hrt_ray_geom, chi_from: float, chi_to: float,
                            a_ref: float, omega_m: float):
    """Planes of a ray-mesh step: ([n1, n2], chi [2][512], w [2][512], drift) (numpy, FP64)."""
    import numpy as np
    n1, n2 = C.c_int32(), C.c_int32()
    chi, w, d = np.zeros(1024), np.zeros(1024), np.zeros(1)
    _check(_lib.hrt_raymesh_step_planes(C.byref(cfg), C.byref(geom), chi_from, chi_to, a_ref, omega_m, C.byref(n1),
                                        C.byref(n2), chi.ctypes.data, w.ctypes.data, d.ctypes.data),
           "hrt_raymesh_step_planes")
    return [n1.value, n2.value], chi.reshape(2, 512), w.reshape(2, 512), float(d[0])


class RayMesh:
    """Owner of an ``hrt_raymesh`` workspace (ray-mesh kick operator)."""

    def __init__(self, cfg: hrt_raymesh_config):
        self.cfg = cfg
        self._h = C.c_void_p()
        _check(_lib.hrt_raymesh_create(C.byref(cfg), C.byref(self._h)), "hrt_raymesh_create")

    def hrt_raymesh_kick(self, grad_x, grad_y, geom: hrt_ray_geom, chi_a: float, chi_b: float, a_ref: float = 0.0,
                         omega_m: float = 0.3, stream=None, grad_z=None) -> torch.Tensor:
        """The filtered ray mesh of one half shell as a (N, N, 2) float32 device tensor (``grad_z`` and a geometry
        with replicas: through the tiled light cone)."""
        _, _, n2d = hrt_raymesh_geometry(self.cfg, chi_a, chi_b, geom.box / geom.n)
        out = torch.empty(n2d, n2d, 2, dtype=torch.float32, device=grad_x.device)
        gx, gy = _ptr(grad_x, torch.float32, "grad_x"), _ptr(grad_y, torch.float32, "grad_y")
        if grad_z is None:
            _check(_lib.hrt_raymesh_kick(self._h, gx, gy, C.byref(geom), chi_a, chi_b, a_ref, omega_m,
                                         _ptr(out, torch.float32, "mesh"), _stream(stream)), "hrt_raymesh_kick")
        else:
            _check(_lib.hrt_raymesh_kick_tiled(self._h, gx, gy, _ptr(grad_z, torch.float32, "grad_z"), C.byref(geom),
                                               chi_a, chi_b, a_ref, omega_m, _ptr(out, torch.float32, "mesh"),
                                               _stream(stream)), "hrt_raymesh_kick_tiled")
        return out

    def hrt_raymesh_ray_step(self, rays: RayState, grad_x, grad_y, geom: hrt_ray_geom, chi_from: float, chi_to: float,
                             a_ref: float = 0.0, omega_m: float = 0.3, maps: torch.Tensor | None = None, stream=None,
                             grad_z=None):
        r = rays.c()
        gx, gy = _ptr(grad_x, torch.float32, "grad_x"), _ptr(grad_y, torch.float32, "grad_y")
        if grad_z is None:
            _check(_lib.hrt_raymesh_ray_step(self._h, C.byref(r), gx, gy, C.byref(geom), chi_from, chi_to, a_ref,
                                             omega_m, _ptr(maps, torch.float32, "maps"), _stream(stream)),
                   "hrt_raymesh_ray_step")
        else:
            _check(_lib.hrt_raymesh_ray_step_tiled(self._h, C.byref(r), gx, gy, _ptr(grad_z, torch.float32, "grad_z"),
                                                   C.byref(geom), chi_from, chi_to, a_ref, omega_m,
                                                   _ptr(maps, torch.float32, "maps"), _stream(stream)),
                   "hrt_raymesh_ray_step_tiled")

    def hrt_raymesh_kick_adjoint(self, grad_x, grad_y, mesh_bar: torch.Tensor, geom: hrt_ray_geom, chi_a: float,
                                 chi_b: float, a_ref: float, omega_m: float, gx_bar: torch.Tensor, gy_bar: torch.Tensor,
                                 stream=None, grad_z=None, gz_bar=None):
        """Accumulates dL/dgrad into gx_bar, gy_bar (and gz_bar through a tiled light cone, with grad_z); returns
        dL/dw_p of the shell's planes (numpy)."""
        import numpy as np
        pb = np.zeros(512)
        gx, gy = _ptr(grad_x, torch.float32, "grad_x"), _ptr(grad_y, torch.float32, "grad_y")
        mb = _ptr(mesh_bar, torch.float32, "mesh_bar")
        gxb, gyb = _ptr(gx_bar, torch.float32, "gx_bar"), _ptr(gy_bar, torch.float32, "gy_bar")
        if grad_z is None:
            _check(_lib.hrt_raymesh_kick_adjoint(self._h, gx, gy, mb, C.byref(geom), chi_a, chi_b, a_ref, omega_m,
                                                 gxb, gyb, pb.ctypes.data, _stream(stream)), "hrt_raymesh_kick_adjoint")
        else:
            _check(_lib.hrt_raymesh_kick_tiled_adjoint(self._h, gx, gy, _ptr(grad_z, torch.float32, "grad_z"), mb,
                                                       C.byref(geom), chi_a, chi_b, a_ref, omega_m, gxb, gyb,
                                                       _ptr(gz_bar, torch.float32, "gz_bar"), pb.ctypes.data,
                                                       _stream(stream)), "hrt_raymesh_kick_tiled_adjoint")
        return pb

    def hrt_raymesh_ray_step_adjoint(self, rays: RayState, grad_x, grad_y, geom: hrt_ray_geom, chi_from: float,
                                     chi_to: float, a_ref: float, omega_m: float, bar: RayState, gx_bar, gy_bar,
                                     stream=None, grad_z=None, gz_bar=None):
        """bar: post-step cotangent in, pre-step cotangent out; returns (dL/dw [2][512] numpy, dL/d drift).  With
        grad_z and gz_bar: through a tiled light cone."""
        import numpy as np
        pb = np.zeros(2 * 512)
        db = np.zeros(1)
        r, b = rays.c(), bar.c()
        gx, gy = _ptr(grad_x, torch.float32, "grad_x"), _ptr(grad_y, torch.float32, "grad_y")
        gxb, gyb = _ptr(gx_bar, torch.float32, "gx_bar"), _ptr(gy_bar, torch.float32, "gy_bar")
        if grad_z is None:
            _check(_lib.hrt_raymesh_ray_step_adjoint(self._h, C.byref(r), gx, gy, C.byref(geom), chi_from, chi_to,
                                                     a_ref, omega_m, C.byref(b), gxb, gyb, pb.ctypes.data,
                                                     db.ctypes.data, _stream(stream)), "hrt_raymesh_ray_step_adjoint")
        else:
            _check(_lib.hrt_raymesh_ray_step_tiled_adjoint(self._h, C.byref(r), gx, gy,
                                                           _ptr(grad_z, torch.float32, "grad_z"), C.byref(geom),
                                                           chi_from, chi_to, a_ref, omega_m, C.byref(b), gxb, gyb,
                                                           _ptr(gz_bar, torch.float32, "gz_bar"), pb.ctypes.data,
                                                           db.ctypes.data, _stream(stream)),
                   "hrt_raymesh_ray_step_tiled_adjoint")
        return pb.reshape(2, 512), float(db[0])

    def close(self):
        if self._h:
            _lib.hrt_raymesh_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hrt_ray_drift_free(rays: RayState, chi_from: float, chi_to: float, stream=None):
    r = rays.c()
    _check(_lib.hrt_ray_drift_free(C.byref(r), chi_from, chi_to, _stream(stream)), "hrt_ray_drift_free")


def hrt_ray_readout(rays: RayState, maps: torch.Tensor, stream=None):
    r = rays.c()
    _check(_lib.hrt_ray_readout(C.byref(r), _ptr(maps, torch.float32, "maps"), _stream(stream)), "hrt_ray_readout")


def hrt_kappa_power(kappa: torch.Tensor, m: int, dtheta: float, nbins: int, ell_min: float, ell_max: float,
                    stream=None):
    ell = torch.zeros(nbins, dtype=torch.float64)
    p = torch.zeros(nbins, dtype=torch.float64)
    cnt = torch.zeros(nbins, dtype=torch.int64)
    _check(_lib.hrt_kappa_power(_ptr(kappa, torch.float32, "kappa"), m, dtheta, nbins, ell_min, ell_max,
                                ell.data_ptr(), p.data_ptr(), cnt.data_ptr(), _stream(stream)), "hrt_kappa_power")
    return ell.numpy(), p.numpy(), cnt.numpy()


def hrt_ic_zeldovich(noise: torch.Tensor, n_side: int, box: float, omega_m: float, h: float, n_s: float,
                     sigma8: float, a_init: float, disp: torch.Tensor, mom: torch.Tensor, stream=None):
    c = hrt_cosmology(omega_m, h, n_s, sigma8)
    _check(_lib.hrt_ic_zeldovich(_ptr(noise, torch.float32, "noise"), n_side, box, C.byref(c), a_init,
                                 _ptr(disp, torch.float32, "disp"), _ptr(mom, torch.float32, "mom"), _stream(stream)),
           "hrt_ic_zeldovich")


# ------------------------------------------------------------------------------------------------ adjoints
MAX_RAY_NODES = 1024


def hrt_cic_scatter_adjoint(rho_bar, disp, n_side, n, box, disp_bar, stream=None):
    _check(_lib.hrt_cic_scatter_adjoint(_ptr(rho_bar, torch.float32, "rho_bar"), _ptr(disp, torch.float32, "disp"),
                                        n_side, n, box, _ptr(disp_bar, torch.float32, "disp_bar"), _stream(stream)),
           "hrt_cic_scatter_adjoint")


def hrt_particle_kick_drift_adjoint(grad, n, box, n_side, disp, mom, kick, drift, rho_bar, disp_bar, mom_bar,
                                    grad_bar, coef_bar, stream=None):
    _check(_lib.hrt_particle_kick_drift_adjoint(
        _ptr(grad, torch.float32, "grad"), n, box, n_side, _ptr(disp, torch.float32, "disp"),
        _ptr(mom, torch.float32, "mom"), kick, drift, _ptr(rho_bar, torch.float32, "rho_bar"),
        _ptr(disp_bar, torch.float32, "disp_bar"), _ptr(mom_bar, torch.float32, "mom_bar"),
        _ptr(grad_bar, torch.float32, "grad_bar"), _ptr(coef_bar, torch.float64, "coef_bar"), _stream(stream)),
        "hrt_particle_kick_drift_adjoint")


def hrt_ray_step_adjoint(rays: RayState, grad_x, grad_y, geom, chi_from, chi_to, a_ref, omega_m, bar: RayState,
                         gx_bar, gy_bar, node_bar, drift_bar, stream=None):
    r, b = rays.c(), bar.c()
    _check(_lib.hrt_ray_step_adjoint(C.byref(r), _ptr(grad_x, torch.float32, "grad_x"),
                                     _ptr(grad_y, torch.float32, "grad_y"), C.byref(geom), chi_from, chi_to, a_ref,
                                     omega_m, C.byref(b), _ptr(gx_bar, torch.float32, "gx_bar"),
                                     _ptr(gy_bar, torch.float32, "gy_bar"), _ptr(node_bar, torch.float64, "node_bar"),
                                     _ptr(drift_bar, torch.float64, "drift_bar"), _stream(stream)),
           "hrt_ray_step_adjoint")


def hrt_ray_step_tiled_adjoint(rays: RayState, grad, geom, chi_from, chi_to, a_ref, omega_m, bar: RayState, grad_bar,
                               node_bar, drift_bar, stream=None):
    """Tiled ray-step adjoint; grad and grad_bar hold the three fields [3][n^3]."""
    r, b = rays.c(), bar.c()
    g, gb = grad.reshape(3, -1), grad_bar.reshape(3, -1)
    _check(_lib.hrt_ray_step_tiled_adjoint(C.byref(r), _ptr(g[0], torch.float32, "grad_x"), _ptr(g[1], torch.float32, "grad_y"),
                                           _ptr(g[2], torch.float32, "grad_z"), C.byref(geom), chi_from, chi_to, a_ref,
                                           omega_m, C.byref(b), _ptr(gb[0], torch.float32, "gx_bar"),
                                           _ptr(gb[1], torch.float32, "gy_bar"), _ptr(gb[2], torch.float32, "gz_bar"),
                                           _ptr(node_bar, torch.float64, "node_bar"), _ptr(drift_bar, torch.float64, "drift_bar"),
                                           _stream(stream)), "hrt_ray_step_tiled_adjoint")


def hrt_ray_step_coefficients(geom, chi_from, chi_to, a_ref, omega_m):
    n1, n2 = C.c_int32(), C.c_int32()
    cw = (C.c_double * MAX_RAY_NODES)()
    cwr = (C.c_double * MAX_RAY_NODES)()
    chi = (C.c_double * MAX_RAY_NODES)()
    d = C.c_double()
    _check(_lib.hrt_ray_step_coefficients(C.byref(geom), chi_from, chi_to, a_ref, omega_m, C.byref(n1), C.byref(n2),
                                          cw, cwr, chi, C.byref(d)), "hrt_ray_step_coefficients")
    k = n1.value + n2.value
    import numpy as np
    return (n1.value, n2.value, np.array(cw[:k]), np.array(cwr[:k]), np.array(chi[:k]), d.value)


def hrt_kappa_power_adjoint(kappa, m, dtheta, nbins, ell_min, ell_max, dl_dp, kappa_bar, stream=None):
    import numpy as np
    w = np.ascontiguousarray(np.asarray(dl_dp, dtype=np.float64))
    _check(_lib.hrt_kappa_power_adjoint(_ptr(kappa, torch.float32, "kappa"), m, dtheta, nbins, ell_min, ell_max,
                                        w.ctypes.data, _ptr(kappa_bar, torch.float32, "kappa_bar"), _stream(stream)),
           "hrt_kappa_power_adjoint")


def hrt_ic_table(n_side, box, omega_m, h, n_s, sigma8, a_init):
    import numpy as np
    c = hrt_cosmology(omega_m, h, n_s, sigma8)
    t = np.zeros(3 * (n_side // 2) ** 2 + 1)
    ratio = C.c_double()
    _check(_lib.hrt_ic_table(n_side, box, C.byref(c), a_init, t.ctypes.data, C.byref(ratio)), "hrt_ic_table")
    return t, ratio.value


def hrt_ic_2lpt(noise: torch.Tensor, n_side: int, box: float, omega_m: float, h: float, n_s: float, sigma8: float,
                a_init: float, disp: torch.Tensor, mom: torch.Tensor, stream=None):
    c = hrt_cosmology(omega_m, h, n_s, sigma8)
    _check(_lib.hrt_ic_2lpt(_ptr(noise, torch.float32, "noise"), n_side, box, C.byref(c), a_init,
                            _ptr(disp, torch.float32, "disp"), _ptr(mom, torch.float32, "mom"), _stream(stream)),
           "hrt_ic_2lpt")


def hrt_ic_2lpt_adjoint(noise, n_side, box, omega_m, h, n_s, sigma8, a_init, disp_bar, mom_bar, noise_bar, stream=None):
    """Fills noise_bar; returns (dL/d unit-growth table, dL/d(D1, D2, c1, c2)) as numpy arrays."""
    import numpy as np
    c = hrt_cosmology(omega_m, h, n_s, sigma8)
    tb = np.zeros(3 * (n_side // 2) ** 2 + 1)
    cb = np.zeros(4)
    _check(_lib.hrt_ic_2lpt_adjoint(_ptr(noise, torch.float32, "noise"), n_side, box, C.byref(c), a_init,
                                    _ptr(disp_bar, torch.float32, "disp_bar"), _ptr(mom_bar, torch.float32, "mom_bar"),
                                    _ptr(noise_bar, torch.float32, "noise_bar"), tb.ctypes.data, cb.ctypes.data,
                                    _stream(stream)), "hrt_ic_2lpt_adjoint")
    return tb, cb


def hrt_ic_2lpt_coefficients(omega_m, h, n_s, sigma8, a_init):
    import numpy as np
    c = hrt_cosmology(omega_m, h, n_s, sigma8)
    out = np.zeros(4)
    _check(_lib.hrt_ic_2lpt_coefficients(C.byref(c), a_init, out.ctypes.data), "hrt_ic_2lpt_coefficients")
    return out


def hrt_ic_zeldovich_adjoint(noise, n_side, box, omega_m, h, n_s, sigma8, a_init, disp_bar, mom_bar, disp, noise_bar,
                             want_table=True, stream=None):
    import numpy as np
    c = hrt_cosmology(omega_m, h, n_s, sigma8)
    tb = np.zeros(3 * (n_side // 2) ** 2 + 1) if want_table else None
    rb = C.c_double()
    _check(_lib.hrt_ic_zeldovich_adjoint(_ptr(noise, torch.float32, "noise"), n_side, box, C.byref(c), a_init,
                                         _ptr(disp_bar, torch.float32, "disp_bar"),
                                         _ptr(mom_bar, torch.float32, "mom_bar"), _ptr(disp, torch.float32, "disp"),
                                         _ptr(noise_bar, torch.float32, "noise_bar"),
                                         tb.ctypes.data if tb is not None else None, C.byref(rb), _stream(stream)),
           "hrt_ic_zeldovich_adjoint")
    return tb, rb.value


def hrt_dot(a, b, stream=None) -> float:
    out = C.c_double()
    _check(_lib.hrt_dot(_ptr(a, torch.float32, "a"), _ptr(b, torch.float32, "b"), a.numel(), C.byref(out),
                        _stream(stream)), "hrt_dot")
    return out.value


# ------------------------------------------------------------------------------------------------ learned correction
MLP_PARAMS = 9473


def hrt_mlp_forward(x, w_bf16, w_f32, g, stream=None):
    _check(_lib.hrt_mlp_forward(_ptr(x, torch.float32, "x"), x.shape[0], _ptr(w_bf16, torch.bfloat16, "w_bf16"),
                                _ptr(w_f32, torch.float32, "w_f32"), _ptr(g, torch.float32, "g"), _stream(stream)),
           "hrt_mlp_forward")


def hrt_mlp_backward(x, w_bf16, w_f32, g_bar, grad, stream=None):
    _check(_lib.hrt_mlp_backward(_ptr(x, torch.float32, "x"), x.shape[0], _ptr(w_bf16, torch.bfloat16, "w_bf16"),
                                 _ptr(w_f32, torch.float32, "w_f32"), _ptr(g_bar, torch.float32, "g_bar"),
                                 _ptr(grad, torch.float32, "grad"), _stream(stream)), "hrt_mlp_backward")


def hrt_mlp_adam(w_f32, w_bf16, grad, m, v, lr, beta1, beta2, eps, step, stream=None):
    _check(_lib.hrt_mlp_adam(_ptr(w_f32, torch.float32, "w_f32"), _ptr(w_bf16, torch.bfloat16, "w_bf16"),
                             _ptr(grad, torch.float32, "grad"), _ptr(m, torch.float32, "m"),
                             _ptr(v, torch.float32, "v"), lr, beta1, beta2, eps, step, _stream(stream)),
           "hrt_mlp_adam")


def hrt_mlp_to_bf16(w_f32, w_bf16, stream=None):
    _check(_lib.hrt_mlp_to_bf16(_ptr(w_f32, torch.float32, "w_f32"), _ptr(w_bf16, torch.bfloat16, "w_bf16"),
                                _stream(stream)), "hrt_mlp_to_bf16")


def hrt_kspace_table_adjoint(gbar_hat, n_comp, rho_hat, n, box, pref, f: hrt_filter, table_bar, stream=None):
    _check(_lib.hrt_kspace_table_adjoint(_ptr(gbar_hat, torch.complex64, "gbar_hat"), n_comp,
                                         _ptr(rho_hat, torch.complex64, "rho_hat"), n, box, pref, C.byref(f),
                                         _ptr(table_bar, torch.float32, "table_bar"), _stream(stream)),
           "hrt_kspace_table_adjoint")


# ------------------------------------------------------------------------------------------------ context
def make_config(n_mesh: int, box: float, n_side: int, omega_m=0.3, h=0.7, n_s=0.96, sigma8=0.8, deconv_p=4.0,
                smooth_cells=1.0, samples_per_cell=1.0, observer=(0.0, 0.0, 0.0), static_mode=False,
                static_pref=0.0, window=(-1e300, 1e300), n_sources=1, ray_fields=0, ray_deconv_p=4.0,
                ray_smooth_cells=1.0) -> hrt_config:
    c = hrt_config()
    c.n_mesh, c.box, c.n_side = n_mesh, box, n_side
    c.cosmo = hrt_cosmology(omega_m, h, n_s, sigma8)
    c.deconv_p, c.smooth_cells, c.samples_per_cell = deconv_p, smooth_cells, samples_per_cell
    for i in range(3):
        c.observer[i] = observer[i]
    c.static_mode, c.static_pref = int(static_mode), static_pref
    c.window_lo, c.window_hi = window
    c.n_sources, c.ray_fields = n_sources, ray_fields
    c.ray_deconv_p, c.ray_smooth_cells = ray_deconv_p, ray_smooth_cells
    return c


def hrt_workspace_bytes(cfg: hrt_config, n_rays: int) -> int:
    out = C.c_size_t()
    _check(_lib.hrt_workspace_bytes(C.byref(cfg), n_rays, C.byref(out)), "hrt_workspace_bytes")
    return out.value


class Context:
    """Owner of an ``hrt_ctx`` (the co-evolution state); methods map one to one onto the C calls."""

    def __init__(self, cfg: hrt_config, stream=None):
        self.cfg = cfg
        self._h = C.c_void_p()
        _check(_lib.hrt_create(C.byref(cfg), _stream(stream), C.byref(self._h)), "hrt_create")
        self.n_rays = 0

    @property
    def handle(self):
        return self._h

    def hrt_init_particles_zeldovich(self, noise: torch.Tensor, a_init: float):
        _check(_lib.hrt_init_particles_zeldovich(self._h, _ptr(noise, torch.float32, "noise"), a_init),
               "hrt_init_particles_zeldovich")

    def hrt_init_particles_2lpt(self, noise: torch.Tensor, a_init: float):
        _check(_lib.hrt_init_particles_2lpt(self._h, _ptr(noise, torch.float32, "noise"), a_init),
               "hrt_init_particles_2lpt")

    def hrt_set_ray_theta_bits(self, bits: int):
        """64: FP64 ray angles (the method); 32: the FP32 ablation."""
        _check(_lib.hrt_set_ray_theta_bits(self._h, bits), "hrt_set_ray_theta_bits")

    def hrt_set_nonfinite_check(self, on: bool):
        _check(_lib.hrt_set_nonfinite_check(self._h, int(bool(on))), "hrt_set_nonfinite_check")

    def hrt_init_particles(self, disp: torch.Tensor, mom: torch.Tensor, a: float):
        """disp, mom: [3][N_p] float32 in device or host memory (pinned host memory keeps the copy asynchronous)."""
        _check(_lib.hrt_init_particles(self._h, _any_ptr(disp, torch.float32, "disp"),
                                       _any_ptr(mom, torch.float32, "mom"), a), "hrt_init_particles")

    def hrt_init_rays(self, theta0: torch.Tensor):
        """theta0: [R][2] float64 in device or host memory."""
        _check(_lib.hrt_init_rays(self._h, _any_ptr(theta0, torch.float64, "theta0"), theta0.shape[0]),
               "hrt_init_rays")
        self.n_rays = theta0.shape[0]

    def hrt_step(self, a_next: float, source: int = -1):
        _check(_lib.hrt_step(self._h, a_next, source), "hrt_step")

    def hrt_set_ray_correction(self, params: torch.Tensor | None):
        """Learned ray-force correction (float32 MLP parameters on the device), or None for the plain kernel."""
        if params is not None and params.numel() != MLP_PARAMS:
            raise ValueError(f"params must hold {MLP_PARAMS} values")
        _check(_lib.hrt_set_ray_correction(self._h, _ptr(params, torch.float32, "params")), "hrt_set_ray_correction")

    def hrt_set_particle_correction(self, params: torch.Tensor | None):
        """Learned particle-force correction (float32 MLP parameters on the device), or None for the plain force."""
        if params is not None and params.numel() != MLP_PARAMS:
            raise ValueError(f"params must hold {MLP_PARAMS} values")
        _check(_lib.hrt_set_particle_correction(self._h, _ptr(params, torch.float32, "params")),
               "hrt_set_particle_correction")

    def hrt_set_replicas(self, replicas=None):
        """Light-cone tiling: (perm, sign, shift) [k][3] integer arrays, or None to remove it."""
        if replicas is None:
            _check(_lib.hrt_set_replicas(self._h, 0, None, None, None), "hrt_set_replicas")
            return
        import numpy as np
        t = [np.ascontiguousarray(x, dtype=np.int32) for x in replicas]
        _check(_lib.hrt_set_replicas(self._h, t[0].shape[0], t[0].ctypes.data, t[1].ctypes.data, t[2].ctypes.data),
               "hrt_set_replicas")

    def hrt_set_particle_sort(self, every: int):
        """Re-sort the particles by mesh cell every `every` particle steps (0: keep lattice order)."""
        _check(_lib.hrt_set_particle_sort(self._h, every), "hrt_set_particle_sort")

    def hrt_set_tiled_deposit(self, mode: int):
        """Kick-drift-deposit: 0 per-particle gathers and reductions (the default), 2 shared-memory tiles by TMA on
        brick-sorted particles, 1 tiles by row copies."""
        _check(_lib.hrt_set_tiled_deposit(self._h, int(mode)), "hrt_set_tiled_deposit")

    def hrt_set_checkpointing(self, every: int):
        """Record the run from the next Zel'dovich ICs for hrt_adjoint (checkpoint every `every` steps; 0: off)."""
        _check(_lib.hrt_set_checkpointing(self._h, every), "hrt_set_checkpointing")

    def hrt_adjoint(self, kappa_bar: torch.Tensor | None, theta_bar: torch.Tensor | None = None):
        """(dL/dnoise float32 device tensor, dL/dOmega_m) of the recorded run for the map and angle cotangents."""
        noise_bar = torch.empty(self.cfg.n_side ** 3, dtype=torch.float32, device="cuda")
        om = C.c_double()
        _check(_lib.hrt_adjoint(self._h, _ptr(kappa_bar, torch.float32, "kappa_bar"),
                                _ptr(theta_bar, torch.float64, "theta_bar"), _ptr(noise_bar, torch.float32, "noise_bar"),
                                C.byref(om)), "hrt_adjoint")
        return noise_bar, om.value

    def hrt_set_ray_mesh(self, cfg: hrt_raymesh_config | None):
        """Ray-mesh kick operator for the context's rays (a ``make_raymesh_config``), or None for the direct gather."""
        _check(_lib.hrt_set_ray_mesh(self._h, None if cfg is None else C.byref(cfg)), "hrt_set_ray_mesh")

    def hrt_set_ray_kernel_table(self, table: torch.Tensor | None, kmax: float = 0.0):
        """Fixed learned table of the ray fields over |k| in [0, kmax] (float32 on the device), or None."""
        _check(_lib.hrt_set_ray_kernel_table(self._h, _ptr(table, torch.float32, "table"),
                                             0 if table is None else table.numel(), kmax), "hrt_set_ray_kernel_table")

    def hrt_state_bytes(self) -> int:
        n = C.c_size_t()
        _check(_lib.hrt_state_bytes(self._h, C.byref(n)), "hrt_state_bytes")
        return n.value

    def hrt_save_state(self) -> torch.Tensor:
        """The context's state in a new device byte tensor (synchronises the stream)."""
        buf = torch.empty(self.hrt_state_bytes(), dtype=torch.uint8, device="cuda")
        _check(_lib.hrt_save_state(self._h, _ptr(buf, torch.uint8, "buf"), buf.numel()), "hrt_save_state")
        return buf

    def hrt_load_state(self, buf: torch.Tensor):
        _check(_lib.hrt_load_state(self._h, _ptr(buf, torch.uint8, "buf"), buf.numel()), "hrt_load_state")
        self.n_rays = int(self.hrt_ctx_rays().n_rays)

    def hrt_step_accumulate(self, a_next: float, source: int, weight: float):
        """hrt_step with map `source` += weight x the observables at the end of the step (Eq. obs_accum)."""
        _check(_lib.hrt_step_accumulate(self._h, a_next, source, weight), "hrt_step_accumulate")

    def hrt_sync_particles(self):
        _check(_lib.hrt_sync_particles(self._h), "hrt_sync_particles")

    def hrt_step_static(self, chi_from: float, chi_to: float, source: int = -1):
        _check(_lib.hrt_step_static(self._h, chi_from, chi_to, source), "hrt_step_static")

    def hrt_drift_free(self, chi_from: float, chi_to: float):
        _check(_lib.hrt_drift_free(self._h, chi_from, chi_to), "hrt_drift_free")

    def hrt_read_rays(self):
        r = self.n_rays
        dev = "cuda"
        th = torch.empty(r, 2, dtype=torch.float64, device=dev)
        eta = torch.empty(r, 2, dtype=torch.float32, device=dev)
        A = torch.empty(r, 4, dtype=torch.float32, device=dev)
        B = torch.empty(r, 4, dtype=torch.float32, device=dev)
        _check(_lib.hrt_read_rays(self._h, th.data_ptr(), eta.data_ptr(), A.data_ptr(), B.data_ptr()), "hrt_read_rays")
        return th, eta, A, B

    def hrt_read_rays_into(self, theta: torch.Tensor | None, eta: torch.Tensor | None = None,
                           A: torch.Tensor | None = None, B: torch.Tensor | None = None):
        """Stream-ordered copies of the ray state into caller tensors in device or host memory (None skips)."""
        _check(_lib.hrt_read_rays(self._h, _any_ptr(theta, torch.float64, "theta"), _any_ptr(eta, torch.float32, "eta"),
                                  _any_ptr(A, torch.float32, "A"), _any_ptr(B, torch.float32, "B")), "hrt_read_rays")

    def hrt_read_rays_async(self, theta: torch.Tensor):
        """Asynchronous copy of the ray angles into a host tensor (float64 [n_rays, 2], pinned for overlap); valid
        once hrt_read_wait has returned."""
        if theta.numel() < 2 * self.n_rays:
            raise ValueError("theta holds fewer than 2 * n_rays values")
        _check(_lib.hrt_read_rays_async(self._h, _host_ptr(theta, torch.float64, "theta")), "hrt_read_rays_async")

    def hrt_read_kappa_async(self, source: int, kappa: torch.Tensor):
        """Asynchronous copy of the convergence map of `source` into a host tensor (float32 [n_rays])."""
        if kappa.numel() < self.n_rays:
            raise ValueError("kappa holds fewer than n_rays values")
        _check(_lib.hrt_read_kappa_async(self._h, source, _host_ptr(kappa, torch.float32, "kappa")),
               "hrt_read_kappa_async")

    def hrt_read_wait(self):
        """Waits (bounded) until every asynchronous read-out copy has landed."""
        _check(_lib.hrt_read_wait(self._h), "hrt_read_wait")

    def hrt_read_maps_into(self, source: int, kappa: torch.Tensor | None, gamma1: torch.Tensor | None = None,
                           gamma2: torch.Tensor | None = None, omega: torch.Tensor | None = None):
        """Stream-ordered copies of the maps of `source` into caller tensors in device or host memory."""
        _check(_lib.hrt_read_maps(self._h, source, _any_ptr(kappa, torch.float32, "kappa"),
                                  _any_ptr(gamma1, torch.float32, "gamma1"), _any_ptr(gamma2, torch.float32, "gamma2"),
                                  _any_ptr(omega, torch.float32, "omega")), "hrt_read_maps")

    def hrt_read_maps(self, source: int):
        r = self.n_rays
        out = torch.empty(4, r, dtype=torch.float32, device="cuda")
        _check(_lib.hrt_read_maps(self._h, source, out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(),
                                  out[3].data_ptr()), "hrt_read_maps")
        return out

    def hrt_read_particles(self):
        n = self.cfg.n_side ** 3
        disp = torch.empty(3, n, dtype=torch.float32, device="cuda")
        mom = torch.empty(3, n, dtype=torch.float32, device="cuda")
        a, ap = C.c_double(), C.c_double()
        _check(_lib.hrt_read_particles(self._h, disp.data_ptr(), mom.data_ptr(), C.byref(a), C.byref(ap)),
               "hrt_read_particles")
        return disp, mom, a.value, ap.value

    def hrt_read_grad(self):
        n = self.cfg.n_mesh
        g = torch.empty(3, n, n, n, dtype=torch.float32, device="cuda")
        _check(_lib.hrt_read_grad(self._h, g.data_ptr()), "hrt_read_grad")
        return g

    def hrt_ctx_kappa_power(self, source: int, m: int, dtheta: float, nbins: int, ell_min: float, ell_max: float):
        ell = torch.zeros(nbins, dtype=torch.float64)
        p = torch.zeros(nbins, dtype=torch.float64)
        cnt = torch.zeros(nbins, dtype=torch.int64)
        _check(_lib.hrt_ctx_kappa_power(self._h, source, m, dtheta, nbins, ell_min, ell_max, ell.data_ptr(),
                                        p.data_ptr(), cnt.data_ptr()), "hrt_ctx_kappa_power")
        return ell.numpy(), p.numpy(), cnt.numpy()

    PHASES = ("ray_step", "kick_drift", "cic_scatter", "fft_r2c", "kspace", "fft_c2r", "step", "particle_sort")

    def hrt_ctx_set_profiling(self, on: bool):
        _check(_lib.hrt_ctx_set_profiling(self._h, int(on)), "hrt_ctx_set_profiling")

    def hrt_ctx_phase_times(self):
        ms = (C.c_double * 8)()
        cnt = (C.c_int64 * 8)()
        _check(_lib.hrt_ctx_phase_times(self._h, ms, cnt), "hrt_ctx_phase_times")
        return {name: (ms[i], cnt[i]) for i, name in enumerate(self.PHASES)}

    def hrt_ctx_rays(self) -> hrt_rays:
        r = hrt_rays()
        _check(_lib.hrt_ctx_rays(self._h, C.byref(r)), "hrt_ctx_rays")
        return r

    def close(self):
        if self._h:
            _lib.hrt_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def raw_status(name: str, *args) -> int:
    """Calls a C entry point with raw ctypes arguments and returns its status (for error-path tests)."""
    return getattr(_lib, name)(*args)
