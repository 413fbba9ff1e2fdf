"""CPU checks of the C-ABI library: it loads, exports every declared symbol, and its host-only FP64 tables (the
cosmology, a ray step's nodes and weights, the Zel'dovich transfer, the static prefactor) match the oracle.  No
GPU compute is called here."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12913_gb300 import hrt
    return hrt


def _declared():
    text = open(os.path.join(ROOT, "include", "hrt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(hrt_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 30
    missing = [n for n in declared if not hasattr(so, n)]
    assert not missing, missing
    assert set(declared) == set(lib.EXPORTED)


def test_status_strings(lib):
    assert lib.status_string(0) == "HRT_OK"
    assert lib.status_string(1) == "HRT_ERR_INVALID_ARG"
    assert lib.status_string(6) == "HRT_ERR_TIMEOUT"


def test_host_cosmology_matches_oracle(lib):
    from oracle import cosmology as oc
    om = 0.3
    for a in (0.02, 1.0 / 3.0, 0.5, 0.9, 1.0):
        E, chi, d1, f = lib.hrt_cosmo_eval(om, a)
        assert E == pytest.approx(oc.E(a, om), rel=1e-14)
        assert chi == pytest.approx(oc.chi_of_a(a, om), rel=1e-12, abs=1e-9)
        assert d1 == pytest.approx(oc.growth_D1(a, om), rel=1e-12)
        assert f == pytest.approx(oc.growth_f(a, om), rel=1e-11)
    for a, b in ((0.02, 0.05), (0.5, 0.7), (1.0, 0.9), (0.5, 0.5)):
        k, d = lib.hrt_cosmo_time_integrals(om, a, b)
        assert k == pytest.approx(oc.kick_integral(a, b, om), rel=1e-12, abs=1e-15)
        assert d == pytest.approx(oc.drift_integral(a, b, om), rel=1e-12, abs=1e-15)
    for chi in (1.0, 500.0, 3000.0):
        assert lib.hrt_cosmo_a_of_chi(om, chi) == pytest.approx(oc.a_of_chi(chi, om), rel=1e-13)
    assert lib.hrt_cosmo_power_amplitude(om, 0.7, 0.96, 0.8) == pytest.approx(
        oc.power_amplitude(om, 0.7, 0.96, 0.8), rel=1e-9)


def test_host_argument_errors(lib):
    with pytest.raises(lib.HRTError) as e:
        lib.hrt_cosmo_eval(0.3, 0.0)
    assert e.value.status == 1
    with pytest.raises(lib.HRTError):
        lib.hrt_cosmo_time_integrals(-0.1, 0.5, 0.6)
    # config validation happens before any CUDA call
    bad = lib.make_config(n_mesh=63, box=100.0, n_side=21)
    with pytest.raises(lib.HRTError) as e:
        lib.hrt_workspace_bytes(bad, 10)
    assert e.value.status == 1
    bad = lib.make_config(n_mesh=64, box=100.0, n_side=24)
    with pytest.raises(lib.HRTError):
        lib.hrt_workspace_bytes(bad, 10)
    good = lib.make_config(n_mesh=64, box=100.0, n_side=32, n_sources=2)
    assert lib.hrt_workspace_bytes(good, 100) > 64 ** 3 * 4 * 4
    # NULL pointers are rejected without touching the device
    assert lib.raw_status("hrt_cic_scatter", None, 4, 8, 10.0, None, None) == 1
    assert lib.raw_status("hrt_destroy", None) == 0
    assert lib.raw_status("hrt_pm_destroy", None) == 0


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2405_12913_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cpp", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), fn
                assert "oracle/" not in src, fn


def test_binding_refuses_to_load_without_library(tmp_path):
    # a copy of the package without the built library must fail loudly on import
    code = ("import sys, os; sys.path.insert(0, %r); import paper_2405_12913_gb300.hrt as h" % str(tmp_path))
    pkg = tmp_path / "paper_2405_12913_gb300"
    pkg.mkdir()
    for fn in ("__init__.py", "hrt.py"):
        (pkg / fn).write_text(open(os.path.join(ROOT, "paper_2405_12913_gb300", fn)).read())
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert r.returncode != 0 and "is not built" in r.stderr


def test_host_raymesh_geometry_matches_oracle(lib):
    """The ray-mesh size rule of App. C on the host equals the oracle's, and bad configurations are refused
    before any device work."""
    from oracle import raymesh
    for chi_a, chi_b, cell, mu, m, iota, p in ((150.5, 181.3, 2.0, 0.001, 100, 0.5, 8), (181.3, 150.5, 2.0, 0.001, 100, 0.5, 8),
                                               (1000.0, 1010.0, 2.0, 0.003, 100, 1.0, 4), (30.0, 60.0, 0.98, 8.5e-5, 2048, 0.5, 256),
                                               (3000.0, 3050.0, 0.98, 8.5e-5, 2048, 0.5, 256), (10.0, 12.0, 3.125, 3e-4, 403, 0.25, 32)):
        want = raymesh.geometry(chi_a, chi_b, cell, mu, m, iota, p)
        got = lib.hrt_raymesh_geometry(lib.make_raymesh_config(iota, p, mu, m, 32768), chi_a, chi_b, cell)
        assert got[2] == want[2] and got[0] == pytest.approx(want[0], rel=1e-15) and got[1] == pytest.approx(want[1], rel=1e-15)
    for bad in ((0.0, 8, 0.001, 64), (1.5, 8, 0.001, 64), (0.5, -1, 0.001, 64), (0.5, 8, 0.0, 64), (0.5, 8, 0.001, 0)):
        with pytest.raises(lib.HRTError):
            lib.RayMesh(lib.make_raymesh_config(*bad))
    with pytest.raises(lib.HRTError):   # an 8192^2 mesh against a limit of 1024
        lib.hrt_raymesh_geometry(lib.make_raymesh_config(0.5, 8, 1e-3, 4096, 1024), 1000.0, 1010.0, 2.0)


def test_host_ray_step_table_matches_oracle(lib):
    # the FP64 node table of one ray step (Alg. 1: two half shells of midpoint nodes, the kick weights of Eq. "kick"
    # with its growth time correction, the drift coefficient of Eq. "drift"), either orientation, with and without a
    # window, against the oracle's nodes and weights
    import numpy as np
    from oracle import cosmology as oc
    from oracle import rays as orays
    from oracle import sim as osim
    from oracle.units import C_LIGHT
    om = 0.3
    g = lib.hrt_ray_geom()
    g.n, g.box = 32, 64.0
    g.observer[0], g.observer[1], g.observer[2] = 19.2, 38.4, 0.0
    g.samples_per_cell = 1.5
    cell = g.box / g.n
    cases = ((100.0, 160.0, False, None), (160.0, 100.0, False, None), (800.0, 870.5, True, None),
             (1500.0, 1400.0, True, None), (800.0, 870.5, True, (815.0, 850.0)))
    for chi_a, chi_b, expanding, window in cases:
        g.window_lo, g.window_hi = window if window else (-1e300, 1e300)
        a_ref = oc.a_of_chi(chi_a, om) if expanding else 0.0
        n1, n2, cw, cwr, chi, d = lib.hrt_ray_step_coefficients(g, chi_a, chi_b, a_ref, om)
        weight = osim.growth_weight(a_ref, om) if expanding else (lambda c: 1.0)
        chi_h = 0.5 * (chi_a + chi_b)
        want_n, want_chi, want_cw = [], [], []
        for lo, hi in ((chi_a, chi_h), (chi_h, chi_b)):
            nodes, h = orays.half_shell_nodes(lo, hi, g.samples_per_cell, cell)
            kept = [c for c in nodes if window is None or window[0] <= c < window[1]]
            want_n.append(len(kept))
            want_chi += kept
            want_cw += [-(2.0 / C_LIGHT) * h * c * weight(c) for c in kept]
        assert (n1, n2) == tuple(want_n)
        if window:
            # the window drops nodes of both half shells but keeps some
            full = [len(orays.half_shell_nodes(lo, hi, g.samples_per_cell, cell)[0])
                    for lo, hi in ((chi_a, chi_h), (chi_h, chi_b))]
            assert 0 < n1 < full[0] and 0 < n2 < full[1]
        want_chi, want_cw = np.array(want_chi), np.array(want_cw)
        np.testing.assert_allclose(chi, want_chi, rtol=1e-14)
        np.testing.assert_allclose(cw, want_cw, rtol=1e-9 if expanding else 1e-14)
        np.testing.assert_allclose(cwr, want_cw * want_chi / cell, rtol=1e-9 if expanding else 1e-14)
        assert d == pytest.approx((chi_b - chi_a) / (C_LIGHT * chi_h * chi_h), rel=1e-14)


def test_host_ic_table_matches_oracle(lib):
    # the Zel'dovich transfer per integer |n|^2, D1 sqrt(P(k) / V_cell) / k^2 / n_side^3 (0 at n = 0), and the
    # momentum ratio a^2 E f, against the oracle's cosmology
    import numpy as np
    from oracle import cosmology as oc
    n, box, a = 16, 200.0, 0.05
    om, h, ns, s8 = 0.3, 0.7, 0.96, 0.8
    t, ratio = lib.hrt_ic_table(n, box, om, h, ns, s8, a)
    assert t.size == 3 * (n // 2) ** 2 + 1
    n2 = np.arange(t.size, dtype=np.float64)
    k = 2.0 * np.pi * np.sqrt(n2) / box
    pk = oc.linear_power(k, om, h, ns, oc.power_amplitude(om, h, ns, s8))
    want = np.zeros_like(t)
    want[1:] = oc.growth_D1(a, om) * np.sqrt(pk[1:] / (box / n) ** 3) / k[1:] ** 2 / n ** 3
    assert t[0] == 0.0
    np.testing.assert_allclose(t, want, rtol=1e-8)
    assert ratio == pytest.approx(a * a * oc.E(a, om) * oc.growth_f(a, om), rel=1e-10)


def test_host_static_prefactor(lib):
    import math
    from oracle.units import G_NEWTON
    assert lib.hrt_static_prefactor(1e15, 200.0) == pytest.approx(4 * math.pi * G_NEWTON * 1e15 / 200.0 ** 3,
                                                                   rel=1e-14)
    for mass, box in ((0.0, 200.0), (-1.0, 200.0), (1e15, 0.0), (float("nan"), 200.0), (1e15, float("inf"))):
        with pytest.raises(lib.HRTError):
            lib.hrt_static_prefactor(mass, box)
