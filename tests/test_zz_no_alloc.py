"""jfnk_budgets_static: the allocation-free budgets entry point, through the C ABI.

It exists for callers that cannot call cudaMalloc (and so cannot create a
handle); its scratch is a fixed device array inside the library.  Checked
against the handle-based jfnk_budgets on the same state, on two calls in a
row (the second call reuses the scratch the first one left behind).
This file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2007_10411_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_budgets_static_matches_handle_budgets_twice():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2007_10411_gb300 import jfnk
    torch.cuda.set_device(0)
    c = synth.case("tiny_130x70")
    c["sgs"]["mode"] = synth.SGS_SMAGORINSKY
    c["grid"]["bc_bottom"] = synth.NOSLIP
    U = synth.random_state(c, 41, amp=(0.5, 0.3, 0.002))
    u = torch.from_numpy(U).cuda()
    s = jfnk.Solver(c)
    ref = s.budgets(u)
    lib = jfnk.load_library()
    grid = jfnk.structs_from_case(c)[0]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    scale = 1e-12 * (m_abs := float(np.max(np.abs(U[:2])))) * c["grid"]["lz"] * c["grid"]["nx"]
    for _ in range(2):
        out = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.jfnk_budgets_static(ctypes.byref(grid), ctypes.c_void_p(u.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), stream)
        assert st == jfnk.JFNK_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for i, k in enumerate(("E_k", "E_p", "sum_theta")):
            assert got[i] == pytest.approx(ref[k], rel=1e-12)
        assert abs(got[3] - ref["sum_div"]) <= scale + 1e-12 * m_abs
        assert list(got[4:8]) == ref["max"]
        assert list(got[8:12]) == ref["min"]
    # sizes beyond the static scratch are rejected before anything runs
    big = jfnk.structs_from_case(synth.with_options(c, nx=8192, nz=2048))[0]
    assert lib.jfnk_budgets_static(ctypes.byref(big), ctypes.c_void_p(u.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), stream) == jfnk.JFNK_ERR_INVALID_ARG
    s.close()
