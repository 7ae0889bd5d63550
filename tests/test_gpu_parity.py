"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on seeded inputs.

Tolerances (relative L2, per field unless stated):
* FP64 per-call operators (F, R, preconditioner, budgets): 1e-12.
* FP64 Jacobian-vector product with an explicit step eps: the forward
  difference divides rounding noise of F by eps, so the bound is
  1e-12 + 50 eps_mach ||W F|| / (eps ||W Jv||)  (derived from the arithmetic).
* MIXED per-call operators: 1e-4 (float32 stencils).
* One implicit step: 1e-10 on the scaled state for FP64, 1e-4 per field for MIXED.
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
    assert torch.cuda.is_available()
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
    out = []
    for f in range(ref.shape[0]):
        den = np.linalg.norm(ref[f])
        out.append(np.linalg.norm(got[f] - ref[f]) / (den if den > 0 else 1.0))
    return np.array(out)


def make_case(nx, nz, smag=False, bc=synth.FREESLIP, beta=3.058e-3, prec=synth.PREC_FP64, heat=False,
              precond=synth.PC_BLOCK, dear=False):
    c = synth.case("tiny_%dx%d" % (nx, nz))
    c["grid"]["bc_bottom"] = bc
    c["strat"]["beta"] = beta
    c["opts"]["precision"] = prec
    c["opts"]["precond"] = precond
    if smag:
        c["sgs"]["mode"] = synth.SGS_SMAGORINSKY
    if dear:
        # anisotropic cells (dz = 0.6 dx), so that K_m != K_M and K_h != K_H
        c["sgs"]["mode"] = synth.SGS_DEARDORFF
        c["grid"]["lz"] *= 0.6
    if heat:
        c["init"] = {"kind": "rest", "H0": 200.0, "patch_halfwidth": c["grid"]["lx"] / 5, "xi": 0.1, "l": 1.5}
    return c


GRIDS = [(16, 8), (100, 37), (130, 70)]          # one tile, ragged multi-tile, ragged in x and z
VARIANTS = [dict(), dict(smag=True), dict(smag=True, bc=synth.NOSLIP, heat=True),
            dict(dear=True, bc=synth.NOSLIP, heat=True)]


def _setup(c, seed=5):
    U = synth.random_state(c, seed, amp=(0.5, 0.3, 0.002))
    m = Model(c)
    s = jf().Solver(c)
    if c["init"]["kind"] == "rest":
        H = synth.heat_flux(c)
        m.set_heat_flux(H)
        s.set_surface_flux(dev(H))
    return U, m, s


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("var", range(len(VARIANTS)))
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_rhs_parity(grid, var, prec):
    c = make_case(*grid, prec=prec, **VARIANTS[var])
    U, m, s = _setup(c)
    ref = m.F(U)
    F = torch.empty_like(dev(U))
    s.rhs(dev(U), F)
    err = rel_per_field(host(F), ref)
    assert np.all(err < (1e-12 if prec == synth.PREC_FP64 else 1e-4)), err


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("var", range(len(VARIANTS)))
def test_residual_parity(grid, var):
    c = make_case(*grid, **VARIANTS[var])
    U, m, s = _setup(c)
    Un = synth.random_state(c, 9, amp=(0.5, 0.3, 0.002))
    ref = m.residual(U, m.rhs_f(Un))
    R = torch.empty_like(dev(U))
    s.residual(dev(Un), dev(U), R)
    err = rel_per_field(host(R), ref)
    assert np.all(err < 1e-12), err


@pytest.mark.parametrize("grid", [(16, 8), (100, 37)])
@pytest.mark.parametrize("var", range(len(VARIANTS)))
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_jv_parity_explicit_eps(grid, var, prec):
    c = make_case(*grid, prec=prec, **VARIANTS[var])
    U, m, s = _setup(c)
    V = np.random.Generator(np.random.PCG64(17)).standard_normal(U.shape)
    V = m.unscale(m.scale(V) / np.linalg.norm(m.scale(V)))     # ||W v|| = 1
    eps = 1e-4
    FU = m.F(U)
    ref = m.jv(U, FU, V, eps)
    out = torch.empty_like(dev(U))
    e_used = s.jv(dev(U), dev(V), out, eps=eps)
    assert e_used == eps
    got = host(out)
    if prec == synth.PREC_FP64:
        bound = 1e-12 + 50 * EPS64 * np.linalg.norm(m.scale(FU)) / (eps * np.linalg.norm(m.scale(ref)))
        assert np.linalg.norm(m.scale(got - ref)) / np.linalg.norm(m.scale(ref)) < bound
    else:
        assert np.all(rel_per_field(got, ref) < 1e-4), rel_per_field(got, ref)


@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_jv_default_eps_rule(prec):
    c = make_case(100, 37, smag=True, prec=prec)
    U, m, s = _setup(c)
    V = np.random.Generator(np.random.PCG64(19)).standard_normal(U.shape)
    out = torch.empty_like(dev(U))
    e_used = s.jv(dev(U), dev(V), out, eps=0.0)
    e_ref = m.fd_epsilon(U, m.scale(V), eps_mach=EPS64)     # same rule for both precisions
    assert e_used == pytest.approx(e_ref, rel=1e-12)
    ref = m.jv(U, m.F(U), V, e_ref)
    got = host(out)
    if prec == synth.PREC_FP64:
        bound = 1e-12 + 50 * EPS64 * np.linalg.norm(m.scale(m.F(U))) / (e_ref * np.linalg.norm(m.scale(ref)))
        assert np.linalg.norm(m.scale(got - ref)) / np.linalg.norm(m.scale(ref)) < bound
    else:
        assert np.all(rel_per_field(got, ref) < 1e-4), rel_per_field(got, ref)


@pytest.mark.parametrize("grid", [(16, 8), (100, 37)])
@pytest.mark.parametrize("var", range(len(VARIANTS)))
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
@pytest.mark.parametrize("sweeps", [1, 2, 4])
def test_precond_parity(grid, var, prec, sweeps):
    c = make_case(*grid, prec=prec, **VARIANTS[var])
    c["opts"]["pc_sweeps"] = sweeps
    if not VARIANTS[var].get("smag"):
        c["sgs"]["K_M"], c["sgs"]["K_H"] = 5.0e3, 7.0e3      # make the blocks non-trivial
    U, m, s = _setup(c)
    r = np.random.Generator(np.random.PCG64(23)).standard_normal(U.shape)
    ref = m.precond(U, r, sweeps)
    z = torch.empty_like(dev(U))
    s.precond_apply(dev(U), dev(r), z)
    err = rel_per_field(host(z), ref)
    assert np.all(err < (1e-12 if prec == synth.PREC_FP64 else 1e-5)), err


@pytest.mark.parametrize("grid", [(16, 8), (100, 37)])
def test_budgets_parity(grid):
    c = make_case(*grid, smag=True)
    U, m, s = _setup(c)
    ref = m.budgets(U)
    got = s.budgets(dev(U))
    for k in ("E_k", "E_p", "sum_theta"):
        assert got[k] == pytest.approx(ref[k], rel=1e-12)
    bound = 1e-12 * m.dx * m.dz * m.nx * m.nz * np.max(np.abs(U[:2])) / m.dx
    assert abs(got["sum_div"]) < bound and abs(ref["sum_div"]) < bound
    assert got["max"] == ref["max"] and got["min"] == ref["min"]


STEP_CASES = [
    ("const_k", dict()),
    ("smag", dict(smag=True)),
    ("noslip_heat", dict(smag=True, bc=synth.NOSLIP, heat=True)),
    ("no_pc", dict(precond=synth.PC_NONE)),
    ("deardorff", dict(dear=True)),
]


@pytest.mark.parametrize("name,var", STEP_CASES)
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_step_parity(name, var, prec):
    c = make_case(64, 32, prec=prec, **var)
    c["opts"]["krylov_m"] = 12                       # force restarts
    U, m, s = _setup(c, seed=31)
    if c["init"]["kind"] == "bubble":
        U = synth.random_state(c, 31, amp=(0.3, 0.1, 0.001))
    st_ref = {}
    ref = implicit_step(m, U, c["opts"], st_ref)
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
        err = rel_per_field(got - U, ref - U)                 # error on the increment per field
        assert np.all(rel_per_field(got, ref) < 1e-4), rel_per_field(got, ref)
        assert np.all(err < 1e-4), err
    # the GPU state satisfies Eq. ns to the Newton tolerance, checked by the oracle
    R = m.residual(got, m.rhs_f(U))
    assert np.linalg.norm(m.scale(R)) <= st["tol"] * 1.01


def test_rest_state_stays_at_rest():
    c = make_case(64, 32, smag=True)
    s = jf().Solver(c)
    u = torch.zeros(synth.shape(c), dtype=torch.float64, device="cuda")
    for _ in range(10):
        st = s.step(u)
        assert st["newton_iters"] == 0
    assert torch.count_nonzero(u).item() == 0


def test_step_host_matches_device_step():
    c = make_case(64, 32, smag=True, prec=synth.PREC_MIXED)
    U = synth.random_state(c, 4, amp=(0.3, 0.1, 0.001))
    s = jf().Solver(c)
    u = dev(U)
    s.step(u)
    uh = torch.from_numpy(U.copy()).pin_memory()
    s.step_host(uh)
    assert torch.equal(uh, u.cpu())
    assert s.launch_count() > 0


@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_full_size_stable_thermal_operators(prec):
    """The 1024x512 stable-thermal workload: F and Jv elementwise against the oracle."""
    c = synth.case("thermal_stable_1024x512")
    c["opts"]["precision"] = prec
    m = Model(c)
    s = jf().Solver(c)
    U = synth.initial_state(c)
    U = U + synth.random_state(c, 2, amp=(0.5, 0.0, 0.001)) - synth.initial_state(synth.with_options(c, noise=0.0))
    F = torch.empty_like(dev(U))
    s.rhs(dev(U), F)
    assert np.all(rel_per_field(host(F), m.F(U)) < (1e-12 if prec == synth.PREC_FP64 else 1e-4))
    V = np.random.Generator(np.random.PCG64(3)).standard_normal(U.shape)
    V = m.unscale(m.scale(V) / np.linalg.norm(m.scale(V)))
    out = torch.empty_like(F)
    s.jv(dev(U), dev(V), out, eps=1e-3)
    ref = m.jv(U, m.F(U), V, 1e-3)
    err = np.linalg.norm(m.scale(host(out) - ref)) / np.linalg.norm(m.scale(ref))
    if prec == synth.PREC_FP64:
        bound = 1e-12 + 50 * EPS64 * np.linalg.norm(m.scale(m.F(U))) / (1e-3 * np.linalg.norm(m.scale(ref)))
        assert err < bound, (err, bound)
    else:
        assert err < 1e-4, err


def test_full_size_step_satisfies_trapezoid_equation():
    """One mixed-precision step of the 1024x512 workload (the benchmark configuration):
    the oracle evaluates Eq. ns at the GPU's state (property check at full size)."""
    c = synth.case("thermal_stable_1024x512")
    m = Model(c)
    s = jf().Solver(c)
    U0 = synth.initial_state(c)
    u = dev(U0)
    st = s.step(u)
    got = host(u)
    assert st["converged"], st
    # the oracle's first step takes 3 Newton corrections (156 + 174 + 230 Krylov iterations)
    assert st["newton_iters"] <= 4, st
    R = m.residual(got, m.rhs_f(U0))
    assert np.linalg.norm(m.scale(R)) <= st["tol"] * 1.01
    b = s.budgets(u)
    assert abs(b["sum_div"]) < 1e-9 * np.max(np.abs(got[:2])) * m.nx * m.nz * m.dx


@pytest.mark.parametrize("smag", [False, True, "deardorff"])
@pytest.mark.parametrize("grid", [(130, 70), (70, 33)])
def test_tile_shapes_give_identical_results(smag, grid):
    """Every tile shape of the float32 Jv and preconditioner kernels computes the same values
    (bitwise), on grids with ragged tiles in x and z (nz = 33: the top tile holds one row, so
    the flux rows above it are ghost rows whose eddy coefficient comes from the rows below);
    autotune picks a valid shape."""
    c = make_case(*grid, smag=smag is True, dear=smag == "deardorff", prec=synth.PREC_MIXED, bc=synth.NOSLIP)
    U, m, s = _setup(c)
    V = np.random.Generator(np.random.PCG64(29)).standard_normal(U.shape)
    outs_jv, outs_pc = [], []
    for t in range(4):
        s.set_tiles(t, t)
        jv = torch.empty_like(dev(U))
        s.jv(dev(U), dev(V), jv, eps=1e-5)
        z = torch.empty_like(dev(U))
        s.precond_apply(dev(U), dev(V), z)
        outs_jv.append(host(jv))
        outs_pc.append(host(z))
    for t in range(1, 4):
        assert np.array_equal(outs_jv[t], outs_jv[0]), t
        assert np.array_equal(outs_pc[t], outs_pc[0]), t
    tiles = s.autotune(dev(U))
    assert all(0 <= t < 4 for t in tiles)
    jv = torch.empty_like(dev(U))
    s.jv(dev(U), dev(V), jv, eps=1e-5)
    assert np.array_equal(host(jv), outs_jv[0])
