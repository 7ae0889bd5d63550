"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every symbol declared in include/jfnk.h, and argument validation
rejects bad input before any CUDA call."""
import ctypes
import os
import re

import pytest

from paper_2007_10411_gb300 import build, jfnk, synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "jfnk.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return jfnk.load_library()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:jfnk_status|const char\*)\s+(jfnk_\w+)\s*\(", text, re.M)))


def test_header_and_binding_agree():
    assert sorted(jfnk.EXPORTS) == declared_functions()


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_status_strings(lib):
    for code in range(0, 9):
        assert lib.jfnk_status_str(code)
    assert lib.jfnk_status_str(1).decode() == "invalid argument"


def _create(lib, c):
    g, s, q, o = jfnk.structs_from_case(c)
    h = ctypes.c_void_p()
    st = lib.jfnk_create(ctypes.byref(g), ctypes.byref(s), ctypes.byref(q), ctypes.byref(o), None,
                         ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("key,val", [
    ("nx", 0), ("nz", 2), ("lx", -1.0), ("lz", float("nan")), ("bc_bottom", 7),
    ("theta0", 0.0), ("Pr", 0.0), ("K_M", -1.0), ("mode", 5),
    ("precision", 3), ("krylov_m", 0), ("krylov_m", 33), ("precond", 5), ("precond", 9), ("pc_sweeps", 0), ("pc_sweeps", 65),
    ("newton_rtol", 0.0), ("eta", 1.0), ("max_newton", -1), ("max_newton", 33), ("dt", 0.0),
    ("scale_p", 0.0),
])
def test_create_rejects_invalid_arguments(lib, key, val):
    c = synth.with_options(synth.case("tiny_16x8"), **{key: val})
    st, h = _create(lib, c)
    assert st == jfnk.JFNK_ERR_INVALID_ARG
    assert not h.value


def test_create_reports_unsupported(lib):
    c = synth.with_options(synth.case("tiny_16x8"), wavelet_p=3)
    assert _create(lib, c)[0] == jfnk.JFNK_ERR_UNSUPPORTED


def test_null_handle_calls_are_rejected(lib):
    P = ctypes.c_void_p
    assert lib.jfnk_rhs(None, P(1), P(1)) == jfnk.JFNK_ERR_INVALID_ARG
    assert lib.jfnk_residual(None, P(1), P(1), P(1)) == jfnk.JFNK_ERR_INVALID_ARG
    assert lib.jfnk_step(None, P(1), None) == jfnk.JFNK_ERR_INVALID_ARG
    assert lib.jfnk_jv(None, P(1), None, P(1), 0.0, P(1), None) == jfnk.JFNK_ERR_INVALID_ARG
    assert lib.jfnk_set_cycle_graph(None, 1) == jfnk.JFNK_ERR_INVALID_ARG
    assert lib.jfnk_kernel_timing(None, 1) == jfnk.JFNK_ERR_INVALID_ARG
    assert lib.jfnk_kernel_timing_sampled(None, 1, 5) == jfnk.JFNK_ERR_INVALID_ARG
    assert lib.jfnk_destroy(None) == jfnk.JFNK_OK


def test_budgets_static_size_limit(lib):
    """jfnk_budgets_static rejects a grid past JFNK_BUDGETS_STATIC_MAX_POINTS before any CUDA call."""
    m = re.search(r"#define\s+JFNK_BUDGETS_STATIC_MAX_POINTS\s+(\d+)", open(HEADER).read())
    nmax = int(m.group(1))
    assert jfnk.BUDGETS_STATIC_MAX_POINTS == nmax
    P = ctypes.c_void_p
    # the smallest grid with nz >= 4 and more points than the limit: nz = 4, nx = nmax / 4 + 1
    c = synth.with_options(synth.case("tiny_16x8"), nx=nmax // 4 + 1, nz=4)
    g = jfnk.structs_from_case(c)[0]
    assert lib.jfnk_budgets_static(ctypes.byref(g), P(16), P(16), None) == jfnk.JFNK_ERR_INVALID_ARG
    # malformed grids and null pointers are rejected the same way
    c = synth.with_options(synth.case("tiny_16x8"), nz=3)
    g = jfnk.structs_from_case(c)[0]
    assert lib.jfnk_budgets_static(ctypes.byref(g), P(16), P(16), None) == jfnk.JFNK_ERR_INVALID_ARG
    g = jfnk.structs_from_case(synth.case("tiny_16x8"))[0]
    assert lib.jfnk_budgets_static(ctypes.byref(g), None, P(16), None) == jfnk.JFNK_ERR_INVALID_ARG


@pytest.mark.parametrize("name,prec", [
    ("thermal3d_32x48x8", synth.PREC_MIXED),     # ny not a multiple of 64
    ("thermal3d_48x64x8", synth.PREC_MIXED),     # nx not a multiple of 32
    ("thermal3d_32x64x6", synth.PREC_MIXED),     # nz not a multiple of 4
    ("thermal3d_32x64x8", synth.PREC_FP64),      # the network runs on the float32 basis only
    ("tiny_48x32", synth.PREC_MIXED),            # 2-D: nx not a multiple of 32
])
def test_learned_preconditioner_grid_rules(lib, name, prec):
    """The learned preconditioner's grid rules (2-D: nx, nz multiples of 32; 3-D: nx of 32,
    ny of 64, nz of 4; mixed precision) are checked before any CUDA call."""
    c = synth.with_options(synth.case(name), precision=prec, precond=jfnk.PC_UNET)
    st, h = _create(lib, c)
    assert st == jfnk.JFNK_ERR_UNSUPPORTED, st
    assert not h.value
