"""Acoustic Schur-complement preconditioner on the GPU against the float64 oracle.

Per-call parity (FP64 1e-12, mixed 1e-5 relative L2 per field, the bounds
of the other preconditioner tests), whole implicit steps (FP64: equal Newton
counts, Krylov counts within one, state 1e-10), and the Krylov-count
reduction over the field-block preconditioner that motivates it.
"""
import numpy as np
import pytest

from oracle.newton import implicit_step
from oracle.operators import Model
from paper_2007_10411_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def jf():
    from paper_2007_10411_gb300 import jfnk
    return jfnk


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_per_field(got, ref):
    return np.array([np.linalg.norm(got[f] - ref[f]) / max(np.linalg.norm(ref[f]), 1e-300)
                     for f in range(ref.shape[0])])


def schur_case(nx, nz, prec, sweeps=8, smag=True, bc=synth.FREESLIP):
    c = synth.case("tiny_%dx%d" % (nx, nz))
    c["opts"]["precision"] = prec
    c["opts"]["precond"] = synth.PC_SCHUR
    c["opts"]["pc_sweeps"] = sweeps
    c["grid"]["bc_bottom"] = bc
    if smag:
        c["sgs"]["mode"] = synth.SGS_SMAGORINSKY
    return c


@pytest.mark.parametrize("grid", [(16, 8), (100, 37), (130, 70)])
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
@pytest.mark.parametrize("sweeps,bc", [(2, synth.FREESLIP), (8, synth.NOSLIP), (16, synth.FREESLIP)])
def test_schur_precond_parity(grid, prec, sweeps, bc):
    c = schur_case(*grid, prec, sweeps=sweeps, bc=bc)
    U = synth.random_state(c, 5, amp=(0.5, 0.3, 0.002))
    m = Model(c)
    s = jf().Solver(c)
    r = np.random.Generator(np.random.PCG64(23)).standard_normal(U.shape)
    ref = m.schur_precond(U, r, sweeps)
    z = torch.empty_like(dev(U))
    s.precond_apply(dev(U), dev(r), z)
    err = rel_per_field(host(z), ref)
    assert np.all(err < (1e-12 if prec == synth.PREC_FP64 else 1e-5)), err
    s.close()


@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_schur_step_parity(prec):
    c = schur_case(64, 32, prec, sweeps=8)
    c["opts"]["krylov_m"] = 12
    # Two states that both pass the Newton test ||W R|| <= rtol ||W R_0|| may
    # differ by ~||J^-1|| rtol ||W R_0||, a few 1e-10 of the state here; with
    # tight inner and outer tolerances both sides converge to the same root and
    # the comparison measures the arithmetic, not the stopping point.
    c["opts"]["eta"] = 1e-8
    c["opts"]["newton_rtol"] = 1e-11
    U = synth.random_state(c, 31, amp=(0.3, 0.1, 0.001))
    m = Model(c)
    st_ref = {}
    ref = implicit_step(m, U, c["opts"], st_ref)
    s = jf().Solver(c)
    u = dev(U)
    st = s.step(u)
    got = host(u)
    assert st["converged"] and st_ref["converged"]
    if prec == synth.PREC_FP64:
        assert st["newton_iters"] == st_ref["newton_iters"]
        assert np.all(np.abs(np.array(st["gmres_per_newton"]) - np.array(st_ref["gmres_iters"])) <= 1)
        err = np.linalg.norm(m.scale(got - ref)) / np.linalg.norm(m.scale(ref))
        assert err < 1e-10, err
    else:
        assert np.all(rel_per_field(got - U, ref - U) < 1e-4)
    R = m.residual(got, m.rhs_f(U))
    assert np.linalg.norm(m.scale(R)) <= st["tol"] * 1.01
    s.close()


def test_schur_cuts_krylov_iterations():
    """256x128 stable thermal (acoustic Courant number 4.4): two steps from the
    initial state need at most a quarter of the field-block preconditioner's
    Krylov iterations, and both reach the Newton tolerance."""
    c = synth.case("thermal_stable_256x128")
    U0 = synth.initial_state(c).reshape(-1)
    counts = {}
    for pc in (synth.PC_BLOCK, synth.PC_SCHUR):
        c2 = synth.with_options(c, precond=pc, pc_sweeps=8)
        s = jf().Solver(c2)
        u = dev(U0)
        st = [s.step(u) for _ in range(2)]
        assert all(x["converged"] for x in st)
        counts[pc] = sum(x["gmres_iters"] for x in st)
        s.close()
    assert counts[synth.PC_SCHUR] <= 0.25 * counts[synth.PC_BLOCK], counts


def test_schur_rejected_for_one_sweep():
    c = schur_case(16, 8, synth.PREC_FP64, sweeps=1)
    with pytest.raises(jf().JfnkError) as e:
        jf().Solver(c)
    assert e.value.code == jf().JFNK_ERR_UNSUPPORTED


def schur_case3d(nx, ny, nz, prec, sweeps=8):
    c = synth.case("tiny3d_%dx%dx%d" % (nx, ny, nz))
    c["opts"]["precision"] = prec
    c["opts"]["precond"] = synth.PC_SCHUR
    c["opts"]["pc_sweeps"] = sweeps
    c["sgs"]["mode"] = synth.SGS_SMAGORINSKY
    return c


@pytest.mark.parametrize("grid", [(16, 12, 8), (20, 18, 11)])
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
@pytest.mark.parametrize("sweeps", [2, 9])
def test_schur3d_precond_parity(grid, prec, sweeps):
    c = schur_case3d(*grid, prec, sweeps=sweeps)
    U = synth.random_state(c, 5, amp=(0.5, 0.3, 0.002))
    m = Model(c)
    s = jf().Solver(c)
    r = np.random.Generator(np.random.PCG64(29)).standard_normal(U.shape)
    ref = m.schur_precond(U, r, sweeps)
    z = torch.empty_like(dev(U))
    s.precond_apply(dev(U), dev(r), z)
    err = rel_per_field(host(z), ref)
    assert np.all(err < (1e-12 if prec == synth.PREC_FP64 else 1e-5)), err
    s.close()


def test_schur3d_step_parity_and_reduction():
    """FP64 step against the oracle (tight tolerances, as in 2-D), and fewer
    Krylov iterations than the field-block preconditioner on the same step."""
    c = schur_case3d(16, 12, 8, synth.PREC_FP64, sweeps=8)
    c["opts"]["eta"] = 1e-8
    c["opts"]["newton_rtol"] = 1e-11
    U = synth.random_state(c, 41, amp=(0.3, 0.1, 0.001))
    m = Model(c)
    st_ref = {}
    ref = implicit_step(m, U, c["opts"], st_ref)
    s = jf().Solver(c)
    u = dev(U)
    st = s.step(u)
    got = host(u)
    assert st["converged"] and st_ref["converged"]
    assert st["newton_iters"] == st_ref["newton_iters"]
    err = np.linalg.norm(m.scale(got - ref)) / np.linalg.norm(m.scale(ref))
    assert err < 1e-10, err
    s.close()
    cb = synth.with_options(c, precond=synth.PC_BLOCK, pc_sweeps=4)
    sb = jf().Solver(cb)
    ub = dev(U)
    stb = sb.step(ub)
    assert stb["converged"]
    assert st["gmres_iters"] < stb["gmres_iters"], (st["gmres_iters"], stb["gmres_iters"])
    sb.close()
