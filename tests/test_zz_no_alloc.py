"""The allocation-free k-space entry point against the ordinary one, through the C ABI.

hrt_kspace_gradient_noalloc serves callers that may not allocate device memory (their own memory pool, or no
allocation allowed mid-step); it keeps its filter tables in a fixed device array instead of a per-call buffer.
It must give the same spectra as hrt_kspace_gradient, also on a second call in a row (the fixed array then
holds the first call's tables, which the second call must overwrite)."""
import math

import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrt():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12913_gb300 import hrt as h
    return h


def _both(hrt, spec, n, box, pref, fa, fb):
    rho_hat = torch.as_tensor(spec, dtype=torch.complex64, device="cuda")
    shape = (n, n, n // 2 + 1)
    ref_a = torch.empty(3, *shape, dtype=torch.complex64, device="cuda")
    ref_b = torch.empty(2, *shape, dtype=torch.complex64, device="cuda")
    got_a = torch.full((3, *shape), float("nan"), dtype=torch.complex64, device="cuda")
    got_b = torch.full((2, *shape), float("nan"), dtype=torch.complex64, device="cuda")
    hrt.hrt_kspace_gradient(rho_hat, n, box, pref, fa, 3, ref_a, fb, 2, ref_b)
    hrt.hrt_kspace_gradient_noalloc(rho_hat, n, box, pref, fa, 3, got_a, fb, 2, got_b)
    torch.cuda.synchronize()
    return ref_a.cpu().numpy(), ref_b.cpu().numpy(), got_a.cpu().numpy(), got_b.cpu().numpy()


def test_noalloc_matches_ordinary_entry_point_on_two_calls(hrt):
    n, box = 48, 75.0
    kmax = 2 * math.pi / box * n
    table = torch.as_tensor(np.linspace(0.8, 1.3, 17, dtype=np.float32), device="cuda")
    calls = [
        (synthetic.complex_spectrum(21, n), 1.7, hrt.make_filter(4.0, box / n), hrt.make_filter(0.0, 0.0)),
        (synthetic.complex_spectrum(22, n), 0.6, hrt.make_filter(0.0, 0.0), hrt.make_filter(2.0, 2.5, table, kmax)),
    ]
    for spec, pref, fa, fb in calls:
        ra, rb, ga, gb = _both(hrt, spec, n, box, pref, fa, fb)
        for ref, got in ((ra, ga), (rb, gb)):
            assert np.isfinite(got).all()
            assert np.abs(got - ref).max() <= 3e-6 * np.abs(ref).max()


def test_noalloc_rejects_meshes_beyond_its_fixed_tables(hrt):
    x = torch.zeros(2, dtype=torch.complex64, device="cuda")
    with pytest.raises(hrt.HRTError) as e:
        hrt.hrt_kspace_gradient_noalloc(x, 4096, 100.0, 1.0, hrt.make_filter(), 3, x)
    assert e.value.status == 1 and "fixed table limit" in str(e.value)


def test_noalloc_rejects_what_the_ordinary_entry_point_rejects(hrt):
    # an infinite box or prefactor, a non-finite deconvolution power and a negative or NaN smoothing length are
    # refused by both entry points before anything is enqueued
    n = 8
    x = torch.zeros(n * n * (n // 2 + 1) * 3, dtype=torch.complex64, device="cuda")
    good = hrt.make_filter(4.0, 1.0)
    cases = [
        (math.inf, 1.0, good),
        (100.0, math.inf, good),
        (100.0, math.nan, good),
        (100.0, 1.0, hrt.make_filter(math.nan, 1.0)),
        (100.0, 1.0, hrt.make_filter(4.0, -1.0)),
        (100.0, 1.0, hrt.make_filter(4.0, math.nan)),
    ]
    for box, pref, f in cases:
        for call in (hrt.hrt_kspace_gradient, hrt.hrt_kspace_gradient_noalloc):
            with pytest.raises(hrt.HRTError) as e:
                call(x, n, box, pref, f, 3, x)
            assert e.value.status == 1, (call.__name__, box, pref)
    torch.cuda.synchronize()


def test_noalloc_refuses_a_call_during_stream_capture(hrt):
    # the tables are staged from a host buffer during the call, which a captured graph could not replay, so a
    # call on a capturing stream returns HRT_ERR_STATE and enqueues nothing (the captured graph stays empty)
    n = 8
    x = torch.zeros(n * n * (n // 2 + 1) * 3, dtype=torch.complex64, device="cuda")
    f = hrt.make_filter(4.0, 1.0)
    hrt.hrt_kspace_gradient_noalloc(x, n, 100.0, 1.0, f, 3, x)  # first call on the device: the set-up
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            with pytest.raises(hrt.HRTError) as e:
                hrt.hrt_kspace_gradient_noalloc(x, n, 100.0, 1.0, f, 3, x, stream=s)
        finally:
            g.capture_end()
    assert e.value.status == 4 and "captured" in str(e.value)
    torch.cuda.synchronize()
