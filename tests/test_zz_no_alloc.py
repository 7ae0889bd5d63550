"""jfnk_budgets_static: the allocation-free budgets entry point, through the C ABI.

It exists for callers that cannot call cudaMalloc (and so cannot create a
handle); its scratch is a fixed device array inside the library.  Checked
against the handle-based jfnk_budgets on two calls in a row with different
states: the second call reuses the scratch (partial sums and counter) the
first one left behind, so stale partials or a counter that is not reset
would show up as wrong values.  Also checked: a grid of exactly
JFNK_BUDGETS_STATIC_MAX_POINTS points runs, and a NaN in the state makes the
extrema NaN.  (The rejection of one point more is an argument check that
runs before any CUDA call: tests/test_abi.py covers it on the CPU.)
This file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2007_10411_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _static(lib, jfnk, c, u, stream):
    grid = jfnk.structs_from_case(c)[0]
    out = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.jfnk_budgets_static(ctypes.byref(grid), ctypes.c_void_p(u.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), stream)
    assert st == jfnk.JFNK_OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _check(got, ref, U, c):
    m_abs = float(np.max(np.abs(U[:2])))
    scale = 1e-12 * m_abs * c["grid"]["lz"] * c["grid"]["nx"]
    for i, k in enumerate(("E_k", "E_p", "sum_theta")):
        assert got[i] == pytest.approx(ref[k], rel=1e-12)
    assert abs(got[3] - ref["sum_div"]) <= scale + 1e-12 * m_abs
    assert list(got[4:8]) == ref["max"]
    assert list(got[8:12]) == ref["min"]


def test_budgets_static_matches_handle_budgets_twice():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2007_10411_gb300 import jfnk
    torch.cuda.set_device(0)
    c = synth.case("tiny_130x70")
    c["sgs"]["mode"] = synth.SGS_SMAGORINSKY
    c["grid"]["bc_bottom"] = synth.NOSLIP
    lib = jfnk.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    s = jfnk.Solver(c)
    # two different states, the second with larger extremes in every field
    for seed, amp in ((41, (0.5, 0.3, 0.002)), (42, (2.0, 1.1, 0.009))):
        U = synth.random_state(c, seed, amp=amp)
        u = torch.from_numpy(U).cuda()
        ref = s.budgets(u)
        _check(_static(lib, jfnk, c, u, stream), ref, U, c)
    s.close()


def test_budgets_static_largest_grid_and_nan():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2007_10411_gb300 import jfnk
    torch.cuda.set_device(0)
    lib = jfnk.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    nmax = jfnk.BUDGETS_STATIC_MAX_POINTS
    c = synth.with_options(synth.case("tiny_64x32"), nx=4096, nz=nmax // 4096)
    assert c["grid"]["nx"] * c["grid"]["nz"] == nmax
    g = torch.Generator(device="cuda").manual_seed(3)
    u = torch.randn(4 * nmax, device="cuda", dtype=torch.float64, generator=g)
    got = _static(lib, jfnk, c, u, stream)
    U = u.view(4, -1)
    assert np.allclose(got[4:8], U.max(dim=1).values.cpu().numpy(), rtol=0, atol=0)
    assert np.allclose(got[8:12], U.min(dim=1).values.cpu().numpy(), rtol=0, atol=0)
    assert got[2] == pytest.approx(float(U[2].sum()) * (c["grid"]["lx"] / 4096) * (c["grid"]["lz"] / (nmax // 4096)),
                                   rel=1e-9, abs=1e-6)
    # a NaN in theta: its max and min are NaN, the other fields' extrema stay finite
    small = synth.case("tiny_64x32")
    U = synth.random_state(small, 5)
    U[2, 7, 11] = np.nan
    got = _static(lib, jfnk, small, torch.from_numpy(U).cuda(), stream)
    assert np.isnan(got[6]) and np.isnan(got[10])
    assert np.all(np.isfinite(got[[4, 5, 7, 8, 9, 11]]))
    del u
    torch.cuda.empty_cache()
