"""Pins of the oracle's discrete operators against invariants, closed forms and brute force.

Section 2.2 (skew-symmetric convection), Section 2.1 (Eqs. ch2_28-ch2_30),
Section 2.4 (eddy viscosity), Section 2.5 (Eq. fd), Section 3.1.3 (budgets).
"""
import math

import numpy as np
import pytest

from oracle.operators import Model, chebyshev
from paper_2007_10411_gb300 import synth


def small_case(nx=16, nz=12, dim=2, ny=1, bc_bottom=synth.FREESLIP, smag=False, beta=0.0, K=(10.0, 14.1)):
    c = synth.case("tiny_%dx%d" % (nx, nz))
    c["grid"]["bc_bottom"] = bc_bottom
    c["strat"]["beta"] = beta
    c["sgs"]["K_M"], c["sgs"]["K_H"] = K
    if smag:
        c["sgs"]["mode"] = synth.SGS_SMAGORINSKY
    if dim == 3:
        c["grid"].update(dim=3, ny=ny, ly=c["grid"]["lx"] * ny / nx)
    return c


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def deriv_matrix(m, parity):
    """Assemble the 1-D z-derivative for a mirror parity by applying it to unit vectors."""
    nz = m.nz
    D = np.zeros((nz, nz))
    for k in range(nz):
        e = np.zeros((nz, 1))
        e[k, 0] = 1.0
        dz = m.deriv(m.extend(e, m.H, parity), 0, m.dz)     # rows: halo r in z
        D[:, k] = dz[m.r:m.r + nz, m.H]
    return D


@pytest.mark.parametrize("pb,pt", [(1, 1), (-1, -1), (-1, 1), (1, -1)])
def test_mirror_derivative_pairing(pb, pt):
    """D_s = -D_{-s}^T for mirror ghosts of parity s (what makes the discrete forms skew)."""
    m = Model(small_case(nx=8, nz=10))
    Dp = deriv_matrix(m, (pb, pt))
    Dm = deriv_matrix(m, (-pb, -pt))
    assert np.allclose(Dp, -Dm.T, atol=1e-15 / m.dz)
    # even data: derivative of a constant vanishes
    if pb == pt == 1:
        assert np.allclose(Dp @ np.ones(m.nz), 0.0, atol=1e-15)


def _conv(m, U, phi, parity):
    Pv = [m.extend(U[i], m.H, m.parity[i]) for i in m.vel]
    Pp = m.extend(phi, m.H, parity)
    return m.convection(Pv, Pp, m.grad_halo(Pp))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("bc", [synth.FREESLIP, synth.NOSLIP])
def test_convection_skew(dim, bc):
    """<phi, C(u) phi> = 0 for every parity of phi (Section 2.2), to 1e-12 relative."""
    c = small_case(nx=12, nz=10, dim=dim, ny=8, bc_bottom=bc)
    m = Model(c)
    r = rng(11)
    U = r.standard_normal(synth.shape(c))
    for f in range(m.nf):
        phi = r.standard_normal(U[f].shape)
        C = _conv(m, U, phi, m.parity[f])
        scale = np.sum(phi * phi) * np.max(np.abs(U)) / min(m.spacing)
        assert abs(np.sum(phi * C)) <= 1e-12 * scale
        # a plain advective form is not skew: the pin is sensitive
        P = m.extend(phi, m.H, m.parity[f])
        adv = sum(m.crop(m.extend(U[i], m.H, m.parity[i]), m.H) * m.crop(g, m.r)
                  for i, g in zip(m.vel, m.grad_halo(P)))
        assert abs(np.sum(phi * adv)) > 1e-6 * scale


def test_flux_form_conserves():
    """sum_k D_j(u_j phi)_k = 0: the flux half of C(u) conserves theta and p.

    (Fields whose wall-normal flux w*phi is even at a wall, like w itself,
    exchange momentum with the wall and are not conserved.)
    """
    c = small_case(nx=12, nz=10, bc_bottom=synth.NOSLIP)
    m = Model(c)
    r = rng(3)
    U = r.standard_normal(synth.shape(c))
    for f in (m.ith, m.ip):
        Pv = [m.extend(U[i], m.H, m.parity[i]) for i in m.vel]
        Pf = m.extend(U[f], m.H, m.parity[f])
        fl = m.div_halo([m.crop(v * Pf, m.r) for v in Pv])
        assert abs(np.sum(fl)) < 1e-12 * np.sum(np.abs(fl))


def diffusion_matrix(m, K_r, parity):
    n = m.nz * m.nx
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        P = m.extend(e.reshape(m.nz, m.nx), m.H, parity)
        A[:, k] = m.diffusion(K_r, m.grad_halo(P)).ravel()
    return A


@pytest.mark.parametrize("parity", [(1, 1), (-1, -1), (-1, 1)])
@pytest.mark.parametrize("smag", [False, True])
def test_diffusion_symmetric_nsd(parity, smag):
    """sum_j D_j(K D_j .) on an 8x8 grid is symmetric and negative semi-definite (Section 2.4)."""
    c = small_case(nx=8, nz=8, smag=smag)
    m = Model(c)
    if smag:
        U = rng(5).standard_normal(synth.shape(c))
        K_r, _ = m.eddy(U)
        assert np.min(K_r) >= 0.0
    else:
        K_r = 10.0
    A = diffusion_matrix(m, K_r, parity)
    scale = np.max(np.abs(A))
    assert np.max(np.abs(A - A.T)) <= 1e-14 * scale
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert np.max(ev) <= 1e-12 * scale
    if parity == (1, 1):
        assert np.max(np.abs(A @ np.ones(A.shape[0]))) <= 1e-12 * scale


def test_global_mass_conservation():
    """sum_k div(u)_k = 0 to roundoff on periodic-x / mirror-z grids (north wall w odd)."""
    for bc in (synth.FREESLIP, synth.NOSLIP):
        c = small_case(nx=32, nz=16, bc_bottom=bc)
        m = Model(c)
        U = rng(7).standard_normal(synth.shape(c))
        b = m.budgets(U)
        dV = m.dx * m.dz
        assert abs(b["sum_div"]) <= 1e-13 * dV * m.nx * m.nz * np.max(np.abs(U)) / m.dx


def test_rest_state_is_exact_equilibrium():
    """u = w = theta = p = 0 is a discrete steady state for any stratification: F(0) = 0 exactly."""
    for smag in (False, True):
        c = small_case(beta=3.058e-3, smag=smag)
        m = Model(c)
        Z = np.zeros(synth.shape(c))
        assert np.all(m.F(Z) == 0.0)
        assert np.all(m.residual(Z, m.rhs_f(Z)) == 0.0)


def test_gravity_coupling_pointwise():
    """F_w = g theta/theta0 and F_theta = -beta w where the other terms vanish (Eqs. ch2_29-30)."""
    c = small_case(beta=3.058e-3, K=(0.0, 0.0))
    m = Model(c)
    r = rng(9)
    U = np.zeros(synth.shape(c))
    U[m.ith] = r.standard_normal(U[m.ith].shape)
    F = m.F(U)
    assert np.allclose(F[m.iw], m.g * U[m.ith] / m.theta0, rtol=0, atol=1e-16)
    assert np.all(F[m.iu] == 0.0) and np.all(F[m.ith] == 0.0) and np.all(F[m.ip] == 0.0)
    U = np.zeros(synth.shape(c))
    U[m.iw] = 1e-3 * r.standard_normal(U[m.iw].shape)
    F = m.F(U)
    conv = _conv(m, U, np.zeros_like(U[m.ith]), (1, 1))
    assert np.all(conv == 0.0)
    assert np.allclose(F[m.ith], -m.beta * U[m.iw], rtol=0, atol=1e-18)


def _acoustic_mode(m, a, kx_i, kz_i):
    """p ~ cos(kx x) cos(kz z), u ~ sin cos, w ~ cos sin: exact eigenfunctions of the mirror grid."""
    x = -0.5 * m.nx * m.dx + np.arange(m.nx) * m.dx
    z = (np.arange(m.nz) + 0.5) * m.dz
    kx = 2 * math.pi * kx_i / (m.nx * m.dx)
    kz = math.pi * kz_i / (m.nz * m.dz)
    X, Z = np.meshgrid(x, z, indexing="xy")
    modes = [np.sin(kx * X) * np.cos(kz * Z), np.cos(kx * X) * np.sin(kz * Z),
             np.cos(kx * X) * np.sin(kz * Z), np.cos(kx * X) * np.cos(kz * Z)]
    U = np.stack([a[f] * modes[f] for f in range(4)])
    return U, modes, kx, kz


def _ktil(k, h):
    """Symbol of the textbook fourth-order central difference (independent of the oracle weights)."""
    return (8 * math.sin(k * h) - math.sin(2 * k * h)) / (6 * h)


def test_acoustic_linear_operator_closed_form():
    """About rest with K = 0, beta = 0 the Jacobian on a Fourier mode is the closed-form 3x3 map.

    du/dt = -theta0 kx~ P,  dw/dt = theta0 kz~ P,  dP/dt = gamma pbar (-kx~ U + kz~ W)
    for u = U sin cos, w = W cos sin, p = P cos cos  (kx~, kz~ the discrete symbols).
    """
    c = small_case(nx=32, nz=16, K=(0.0, 0.0))
    m = Model(c)
    amp = 1e-7
    a = [0.3, -0.2, 0.0, 0.5]
    U, modes, kx, kz = _acoustic_mode(m, [amp * v for v in a], 3, 2)
    F = m.F(U)
    kxt, kzt = _ktil(kx, m.dx), _ktil(kz, m.dz)
    gp = m.gamma_p * m.pbar
    expect_u = -m.theta0 * (-kxt) * amp * a[3]       # D_x cos = -kxt sin
    expect_w = -m.theta0 * (-kzt) * amp * a[3]       # D_z cos = -kzt sin
    expect_p = -gp * (kxt * amp * a[0] + kzt * amp * a[1])  # D_x sin = kxt cos, D_z sin = kzt cos
    scale = abs(gp * kxt * amp)
    assert np.allclose(F[0], expect_u * modes[0], atol=1e-6 * scale)
    assert np.allclose(F[1], expect_w * modes[1], atol=1e-6 * scale)
    assert np.allclose(F[3], expect_p * modes[3], atol=1e-6 * scale)
    assert np.max(np.abs(F[2])) < 1e-6 * scale


def test_jv_matches_assembled_jacobian_8x8():
    """Forward-difference Jv (Eq. fd) vs the brute-force Jacobian of R on an 8x8 grid.

    With constant K, F is a quadratic polynomial, so central differences of F
    assemble J_F exactly (up to roundoff) and the forward difference obeys
    Jv_fd = J v - eps B(v,v) with B(v,v) = F(v) - J_F(0) v.
    """
    c = small_case(nx=8, nz=8, beta=3.058e-3)
    m = Model(c)
    r = rng(21)
    U = synth.random_state(c, 4)
    n = U.size
    h = 1e-3

    def jac(at):
        J = np.zeros((n, n))
        for k in range(n):
            e = np.zeros(n)
            e[k] = h
            J[:, k] = ((m.F(at + e.reshape(at.shape)) - m.F(at - e.reshape(at.shape))) / (2 * h)).ravel()
        return J

    JF = jac(U)
    JF0 = jac(np.zeros_like(U))
    V = r.standard_normal(U.shape)
    eps = 1e-4
    jv = m.jv(U, m.F(U), V, eps)
    B = m.F(V) - (JF0 @ V.ravel()).reshape(V.shape)
    exact = 2.0 * V / m.dt - (JF @ V.ravel()).reshape(V.shape)
    err = np.linalg.norm((jv + eps * B - exact).ravel()) / np.linalg.norm(exact.ravel())
    assert err < 1e-9
    # scaled product with the default epsilon rule: same identity in W units
    Vhat = m.scale(V)
    Vhat = Vhat / np.linalg.norm(Vhat.ravel())          # unit vector, as a Krylov basis vector
    V = m.unscale(Vhat)
    B = m.F(V) - (JF0 @ V.ravel()).reshape(V.shape)
    exact = 2.0 * V / m.dt - (JF @ V.ravel()).reshape(V.shape)
    jvs = m.jv_scaled(U, m.F(U), Vhat)
    e2 = m.fd_epsilon(U, Vhat)
    assert e2 > 0.0
    ex_s = m.scale(exact)
    err = np.linalg.norm((jvs + e2 * m.scale(B) - ex_s).ravel()) / np.linalg.norm(ex_s.ravel())
    # what remains is cancellation in F(u + eps v) - F(u): ~ eps_mach ||W F|| / eps
    bound = 20 * 2.0 ** -52 * np.linalg.norm(m.scale(m.F(U)).ravel()) / e2 / np.linalg.norm(ex_s.ravel())
    assert err < bound
    assert err < 1e-4


def test_jv_smagorinsky_central_difference():
    c = small_case(nx=8, nz=8, smag=True)
    m = Model(c)
    U = synth.random_state(c, 8)
    V = rng(2).standard_normal(U.shape)
    h = 1e-6
    cd = 2 * V / m.dt - (m.F(U + h * V) - m.F(U - h * V)) / (2 * h)
    jv = m.jv(U, m.F(U), V, 1e-7)
    assert np.linalg.norm((jv - cd).ravel()) / np.linalg.norm(cd.ravel()) < 1e-6


def test_mirror_symmetry_about_x0():
    """F commutes with x -> -x (u odd; w, theta, p even) on the symmetric node set."""
    c = synth.case("tiny_32x16")
    c["sgs"]["mode"] = synth.SGS_SMAGORINSKY
    m = Model(c)
    U = synth.random_state(c, 1)

    def reflect(A):
        B = np.roll(A[..., ::-1], 1, axis=-1)            # x_i -> x_{(nx - i) mod nx}
        B[0] = -B[0]
        return B

    Us = 0.5 * (U + reflect(U))
    F = m.F(Us)
    assert np.allclose(F, reflect(F), atol=1e-13 * np.max(np.abs(F)))


def test_chebyshev_block_preconditioner():
    """Chebyshev with many sweeps inverts each SPD block; with 4 sweeps it is a fixed linear map."""
    c = small_case(nx=8, nz=8, smag=True)
    m = Model(c)
    U = synth.random_state(c, 3)
    K_M, K_H = m.eddy(U)
    r = rng(4).standard_normal(U.shape)
    for f in range(m.nf):
        K = K_H if f == m.ith else K_M
        kmax = 0.0 if f == m.ip else float(np.max(K))
        lo, hi = m.gershgorin_bounds(kmax)
        A = np.zeros((64, 64))
        for k in range(64):
            e = np.zeros(64)
            e[k] = 1.0
            A[:, k] = m.block_operator(K, e.reshape(8, 8), f).ravel()
        ev = np.linalg.eigvalsh(0.5 * (A + A.T))
        assert ev.min() >= lo * (1 - 1e-12) and ev.max() <= hi * (1 + 1e-12)
        x = chebyshev(lambda q: m.block_operator(K, q, f), r[f], lo, hi, 60)
        assert np.allclose(x.ravel(), np.linalg.solve(A, r[f].ravel()), rtol=1e-10, atol=1e-14)
    z1 = m.precond(U, r, 4)
    z2 = m.precond(U, 2.0 * r, 4)
    assert np.allclose(z2, 2.0 * z1, rtol=1e-13, atol=0)


def test_budgets_closed_forms():
    c = small_case(nx=16, nz=8)
    m = Model(c)
    U = np.zeros(synth.shape(c))
    U[m.iu] = 2.0
    U[m.iw] = 0.0
    U[m.ith] = 0.5
    b = m.budgets(U)
    area = m.nx * m.dx * m.nz * m.dz
    assert b["E_k"] == pytest.approx(0.5 * 4.0 * area, rel=1e-14)
    # midpoint rule is exact for the linear weight (lz - z)
    assert b["E_p"] == pytest.approx(0.5 * m.lz * m.lz * m.nx * m.dx * 0.5, rel=1e-13)
    assert b["sum_theta"] == pytest.approx(0.5 * area, rel=1e-14)
    assert b["max"][m.iu] == 2.0 and b["min"][m.ith] == 0.5


def test_schur_preconditioner_inverts_the_acoustic_jacobian_at_rest():
    """At rest with K = 0 and beta = 0 the linearised F holds only the pressure
    gradient and divergence couplings (plus buoyancy, inactive for theta-free
    inputs), so the acoustic Schur preconditioner with a converged Helmholtz
    solve is the exact inverse: J_hat P v = v.  J_hat is the central difference
    of F at u = 0 (exact there: F is linear plus a quadratic convection)."""
    from oracle.operators import Model
    from paper_2007_10411_gb300 import synth
    c = synth.case("thermal_stable_64x32")
    c["strat"]["beta"] = 0.0
    c["sgs"] = {"mode": synth.SGS_CONST, "K_M": 0.0, "K_H": 0.0, "Cs": 0.0, "Pr": 1.0}
    m = Model(c)
    Z0 = np.zeros((4, 32, 64))

    def J_hat(vhat):
        V = m.unscale(vhat)
        h = 1e-3
        JF = (m.F(Z0 + h * V) - m.F(Z0 - h * V)) / (2 * h)
        return m.scale(2.0 * V / m.dt - JF)

    rng = np.random.default_rng(17)
    v = rng.standard_normal((4, 32, 64))
    v[2] = 0.0
    z = m.schur_precond(Z0, v, 40)
    res = J_hat(z) - v
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(v), np.linalg.norm(res) / np.linalg.norm(v)
    # fewer Helmholtz sweeps: an approximate inverse, error shrinking with the sweep count
    errs = [np.linalg.norm(J_hat(m.schur_precond(Z0, v, s)) - v) for s in (2, 4, 8)]
    assert errs[0] > errs[1] > errs[2]
    # the Helmholtz operator is H = J's pressure block after eliminating the velocities
    p = rng.standard_normal((32, 64))
    lo, hi = m.helmholtz_bounds()
    q = m.helmholtz(p)
    assert lo * np.sum(p * p) * (1 - 1e-12) <= np.sum(p * q) <= hi * np.sum(p * p) * (1 + 1e-12)


def test_schur_preconditioner_inverts_the_acoustic_jacobian_at_rest_3d():
    """3-D form of the exact-inverse pin: three velocity components eliminated."""
    from oracle.operators import Model
    from paper_2007_10411_gb300 import synth
    c = synth.case("tiny3d_16x12x8")
    c["strat"]["beta"] = 0.0
    c["sgs"] = {"mode": synth.SGS_CONST, "K_M": 0.0, "K_H": 0.0, "Cs": 0.0, "Pr": 1.0}
    m = Model(c)
    shape = (5, 8, 12, 16)
    Z0 = np.zeros(shape)

    def J_hat(vhat):
        V = m.unscale(vhat)
        h = 1e-3
        JF = (m.F(Z0 + h * V) - m.F(Z0 - h * V)) / (2 * h)
        return m.scale(2.0 * V / m.dt - JF)

    rng = np.random.default_rng(19)
    v = rng.standard_normal(shape)
    v[3] = 0.0
    z = m.schur_precond(Z0, v, 60)
    res = J_hat(z) - v
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(v), np.linalg.norm(res) / np.linalg.norm(v)
