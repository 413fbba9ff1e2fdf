"""CPU checks of the C-ABI library: it loads, exports every declared symbol, and its host-only FP64 cosmology
matches the oracle.  No GPU compute is called here."""
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
