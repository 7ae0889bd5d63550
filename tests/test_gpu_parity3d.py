"""GPU parity of the 3-D kernels (fields u, v, w, theta, p) against the FP64 oracle.

Same tolerances as the 2-D file: FP64 per-call 1e-12 (FD Jv: the derived
roundoff bound), mixed per-call 1e-4 (preconditioner 1e-5), FP64 step 1e-10
on the scaled state, mixed step 1e-4 per field.
"""
import numpy as np
import pytest

from oracle.newton import implicit_step
from oracle.operators import Model
from paper_2007_10411_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -52


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


def make3(nx, ny, nz, smag=False, bc=synth.FREESLIP, prec=synth.PREC_FP64, heat=False, beta=3.058e-3,
          dear=False):
    c = synth.case("tiny3d_%dx%dx%d" % (nx, ny, nz))
    c["grid"]["bc_bottom"] = bc
    c["strat"]["beta"] = beta
    c["opts"]["precision"] = prec
    if smag:
        c["sgs"]["mode"] = synth.SGS_SMAGORINSKY
    if dear:
        # anisotropic closure on anisotropic cells (dy = 0.8 dx, dz = 0.6 dx)
        c["sgs"]["mode"] = synth.SGS_DEARDORFF
        c["grid"]["ly"] *= 0.8
        c["grid"]["lz"] *= 0.6
    if heat:
        c["init"] = {"kind": "rest", "H0": 200.0, "patch_halfwidth": c["grid"]["lx"] / 5, "xi": 0.1, "l": 1.5}
    return c


def setup(c, seed=5):
    U = synth.random_state(c, seed, amp=(0.5, 0.3, 0.002))
    m = Model(c)
    s = jf().Solver(c)
    if c["init"]["kind"] == "rest":
        H = synth.heat_flux(c)
        m.set_heat_flux(H)
        s.set_surface_flux(dev(H))
    return U, m, s


# one tile; ragged; several plane tiles (32 x 8) in x and y and slab tiles (16 / 8 planes) in z, ragged
GRIDS3 = [(16, 8, 8), (21, 13, 9), (40, 18, 21)]
VARS3 = [dict(), dict(smag=True), dict(smag=True, bc=synth.NOSLIP, heat=True),
         dict(dear=True, bc=synth.NOSLIP, heat=True)]


@pytest.mark.parametrize("grid", GRIDS3)
@pytest.mark.parametrize("var", range(len(VARS3)))
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_rhs_parity_3d(grid, var, prec):
    c = make3(*grid, prec=prec, **VARS3[var])
    U, m, s = setup(c)
    F = torch.empty_like(dev(U))
    s.rhs(dev(U), F)
    err = rel_per_field(host(F), m.F(U))
    assert np.all(err < (1e-12 if prec == synth.PREC_FP64 else 1e-4)), err


@pytest.mark.parametrize("grid", GRIDS3)
@pytest.mark.parametrize("var", range(len(VARS3)))
def test_residual_parity_3d(grid, var):
    c = make3(*grid, **VARS3[var])
    U, m, s = setup(c)
    Un = synth.random_state(c, 9, amp=(0.5, 0.3, 0.002))
    R = torch.empty_like(dev(U))
    s.residual(dev(Un), dev(U), R)
    err = rel_per_field(host(R), m.residual(U, m.rhs_f(Un)))
    assert np.all(err < 1e-12), err


@pytest.mark.parametrize("grid", GRIDS3[1:])
@pytest.mark.parametrize("var", range(len(VARS3)))
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_jv_parity_3d(grid, var, prec):
    c = make3(*grid, prec=prec, **VARS3[var])
    U, m, s = setup(c)
    V = np.random.Generator(np.random.PCG64(17)).standard_normal(U.shape)
    V = m.unscale(m.scale(V) / np.linalg.norm(m.scale(V)))
    eps = 1e-4
    FU = m.F(U)
    ref = m.jv(U, FU, V, eps)
    out = torch.empty_like(dev(U))
    s.jv(dev(U), dev(V), out, eps=eps)
    got = host(out)
    if prec == synth.PREC_FP64:
        bound = 1e-12 + 50 * EPS64 * np.linalg.norm(m.scale(FU)) / (eps * np.linalg.norm(m.scale(ref)))
        assert np.linalg.norm(m.scale(got - ref)) / np.linalg.norm(m.scale(ref)) < bound
    else:
        assert np.all(rel_per_field(got, ref) < 1e-4), rel_per_field(got, ref)


@pytest.mark.parametrize("grid", GRIDS3[1:])
@pytest.mark.parametrize("var", range(len(VARS3)))
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
@pytest.mark.parametrize("sweeps", [1, 2, 4])
def test_precond_parity_3d(grid, var, prec, sweeps):
    c = make3(*grid, prec=prec, **VARS3[var])
    c["opts"]["pc_sweeps"] = sweeps
    if not VARS3[var].get("smag"):
        c["sgs"]["K_M"], c["sgs"]["K_H"] = 5.0e3, 7.0e3
    U, m, s = setup(c)
    r = np.random.Generator(np.random.PCG64(23)).standard_normal(U.shape)
    z = torch.empty_like(dev(U))
    s.precond_apply(dev(U), dev(r), z)
    err = rel_per_field(host(z), m.precond(U, r, sweeps))
    assert np.all(err < (1e-12 if prec == synth.PREC_FP64 else 1e-5)), err


def test_budgets_parity_3d():
    c = make3(21, 13, 9, smag=True)
    U, m, s = setup(c)
    ref = m.budgets(U)
    got = s.budgets(dev(U))
    for k in ("E_k", "E_p", "sum_theta"):
        assert got[k] == pytest.approx(ref[k], rel=1e-12)
    bound = 1e-12 * m.dy * m.dz * m.nx * m.ny * m.nz * np.max(np.abs(U[:3]))
    assert abs(got["sum_div"]) < bound and abs(ref["sum_div"]) < bound
    assert got["max"] == ref["max"] and got["min"] == ref["min"]


@pytest.mark.parametrize("var", [dict(), dict(smag=True), dict(smag=True, bc=synth.NOSLIP, heat=True),
                                 dict(dear=True)])
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_step_parity_3d(var, prec):
    c = make3(16, 12, 8, prec=prec, **var)
    c["opts"]["krylov_m"] = 10
    U, m, s = setup(c, seed=31)
    U = synth.random_state(c, 31, amp=(0.3, 0.1, 0.001))
    st_ref = {}
    ref = implicit_step(m, U, c["opts"], st_ref)
    u = dev(U)
    st = s.step(u)
    got = host(u)
    assert st["converged"] and st_ref["converged"]
    if prec == synth.PREC_FP64:
        assert st["newton_iters"] == st_ref["newton_iters"]
        err = np.linalg.norm(m.scale(got - ref)) / np.linalg.norm(m.scale(ref))
        assert err < 1e-10, err
    else:
        assert np.all(rel_per_field(got, ref) < 1e-4), rel_per_field(got, ref)
    R = m.residual(got, m.rhs_f(U))
    assert np.linalg.norm(m.scale(R)) <= st["tol"] * 1.01


def test_full_size_3d_operators_and_step():
    """The config-4 grid (256x256x128 stable thermal, the 3-D bench workload):
    F and the mixed Jacobian product elementwise against the oracle, then one
    mixed step whose state the oracle checks against Eq. ns (property at full size)."""
    c = synth.case("thermal3d_256x256x128")
    m = Model(c)
    s = jf().Solver(c)
    U0 = synth.initial_state(c)
    U = U0 + synth.random_state(c, 2, amp=(0.5, 0.3, 0.001)) - synth.initial_state(synth.with_options(c, noise=0.0))
    F = torch.empty_like(dev(U))
    s.rhs(dev(U), F)
    FU = m.F(U)
    assert np.all(rel_per_field(host(F), FU) < 1e-4), rel_per_field(host(F), FU)
    V = np.random.Generator(np.random.PCG64(3)).standard_normal(U.shape)
    V = m.unscale(m.scale(V) / np.linalg.norm(m.scale(V)))
    out = torch.empty_like(F)
    s.jv(dev(U), dev(V), out, eps=1e-3)
    ref = m.jv(U, FU, V, 1e-3)
    err = np.linalg.norm(m.scale(host(out) - ref)) / np.linalg.norm(m.scale(ref))
    assert err < 1e-4, err
    del F, out, FU, ref
    u = dev(U0)
    st = s.step(u)
    got = host(u)
    assert st["converged"], st
    R = m.residual(got, m.rhs_f(U0))
    assert np.linalg.norm(m.scale(R)) <= st["tol"] * 1.01
    b = s.budgets(u)
    assert abs(b["sum_div"]) < 1e-9 * np.max(np.abs(got[:3])) * m.nx * m.ny * m.nz * m.dx
    s.close()
