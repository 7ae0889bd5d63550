"""Pins of the oracle's GMRES (Section 2.5.1, Saad & Schultz) and Newton loop (Eq. jv, Eq. ns)."""
import math

import numpy as np
import pytest

from oracle.krylov import cgs2, givens, gmres
from oracle.newton import implicit_step
from oracle.operators import Model
from paper_2007_10411_gb300 import synth


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_givens_zeroes_second_entry():
    for a, b in [(3.0, 4.0), (-1.0, 2.0), (0.0, 1.0), (2.0, 0.0)]:
        c, s = givens(a, b)
        assert c * c + s * s == pytest.approx(1.0)
        assert -s * a + c * b == pytest.approx(0.0, abs=1e-15)


def test_gmres_full_dimension_solves_dense_system():
    """With m >= n and no restart GMRES returns numpy.linalg.solve's answer."""
    n = 40
    r = rng(1)
    A = np.eye(n) * 4 + r.standard_normal((n, n))
    b = r.standard_normal(n)
    rec = {}
    x = gmres(lambda v: A @ v, b, m=n, eta=1e-14, max_restarts=0, record=rec)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
    V = np.stack(rec["V"][:-1])
    k = V.shape[0]
    # Arnoldi relation A V_k = V_{k+1} Hbar and orthonormality (CGS2)
    Vk1 = np.stack(rec["V"])
    assert np.max(np.abs(A @ V.T - Vk1.T @ rec["Hbar"])) < 1e-12
    assert np.max(np.abs(V @ V.T - np.eye(k))) < 1e-14


def test_gmres_restarted_reaches_eta_true_residual():
    n = 300
    r = rng(2)
    A = np.diag(np.linspace(1, 10, n)) + 0.3 * r.standard_normal((n, n)) / math.sqrt(n)
    b = r.standard_normal(n)
    rec = {}
    x = gmres(lambda v: A @ v, b, m=10, eta=1e-6, max_restarts=200, record=rec)
    assert rec["converged"] and rec["restarts"] > 0
    # the stopping test is on the rotated estimate; the true residual agrees to roundoff
    assert np.linalg.norm(b - A @ x) <= 1.01e-6 * np.linalg.norm(b)


def test_flexible_equals_right_preconditioned_for_linear_pc():
    n = 60
    r = rng(3)
    A = np.eye(n) * 3 + r.standard_normal((n, n)) / 3
    Mi = np.diag(1.0 / np.diag(A)) + 0.01 * r.standard_normal((n, n))
    b = r.standard_normal(n)
    x1 = gmres(lambda v: A @ v, b, 15, 1e-10, 50, precond=lambda v: Mi @ v)
    x2 = gmres(lambda v: A @ v, b, 15, 1e-10, 50, precond=lambda v: Mi @ v, flexible=True)
    assert np.allclose(x1, x2, rtol=1e-8, atol=1e-10)
    assert np.linalg.norm(b - A @ x1) <= 1.01e-10 * np.linalg.norm(b)


def test_cgs2_orthogonality_on_ill_conditioned_input():
    n = 200
    r = rng(4)
    V = [v for v in np.linalg.qr(r.standard_normal((n, 20)))[0].T]
    w = V[3] * (1 - 1e-10) + 1e-12 * r.standard_normal(n)     # almost dependent
    h, hn, vn = cgs2(V, w)
    assert abs(np.linalg.norm(vn) - 1.0) < 1e-12
    assert np.max(np.abs(np.stack(V) @ vn)) < 1e-12


def _jacobian_of_R(m, U):
    n = U.size
    J = np.zeros((n, n))
    h = 1e-3
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        E = e.reshape(U.shape)
        J[:, k] = (4 * E / m.dt - m.F(U + E) + m.F(U - E)).ravel() / (2 * h)   # (R(u+e) - R(u-e)) / 2h
    return J


def test_gmres_on_assembled_jacobian_8x8():
    """GMRES(256) with the FD product solves the Newton system of the 8x8 grid like numpy.linalg.solve."""
    c = synth.case("tiny_8x8")
    c["strat"]["beta"] = 3.058e-3
    m = Model(c)
    U = synth.random_state(c, 6, amp=(0.1, 0.05, 0.0005))
    Jhat = np.diag(1 / np.repeat(m.scales, 64)) @ _jacobian_of_R(m, U) @ np.diag(np.repeat(m.scales, 64))
    b = rng(7).standard_normal(U.shape)
    FU = m.F(U)
    x = gmres(lambda v: m.jv_scaled(U, FU, v), b, 256, 1e-12, 0)
    ref = np.linalg.solve(Jhat, b.ravel())
    assert np.linalg.norm(x.ravel() - ref) / np.linalg.norm(ref) < 1e-6


def test_rest_stays_at_rest_ten_steps():
    c = synth.case("tiny_16x8")
    c["strat"]["beta"] = 3.058e-3
    c["sgs"]["mode"] = synth.SGS_SMAGORINSKY
    m = Model(c)
    U = np.zeros(synth.shape(c))
    for _ in range(10):
        st = {}
        U = implicit_step(m, U, c["opts"], st)
        assert st["newton_iters"] == 0
    assert np.all(U == 0.0)


def _energy(m, U):
    n2 = m.g * m.beta / m.theta0
    return 0.5 * (np.sum(U[m.iu] ** 2) + np.sum(U[m.iw] ** 2)) + \
        0.5 * m.g * m.g / (m.theta0 ** 2 * n2) * np.sum(U[m.ith] ** 2) + \
        0.5 * m.theta0 / (m.gamma_p * m.pbar) * np.sum(U[m.ip] ** 2)


def test_linear_trapezoid_step_conserves_weighted_energy():
    """About rest with K = 0 the linear operator is skew in the energy inner product
    E = (u^2+w^2)/2 + g^2 theta^2 / (2 theta0^2 N^2) + theta0 p^2 / (2 gamma pbar),
    so one trapezoidal step (Eq. ns, solved by Newton-GMRES) conserves E."""
    c = synth.case("tiny_16x12")
    c["strat"]["beta"] = 3.058e-3
    c["sgs"]["K_M"] = c["sgs"]["K_H"] = 0.0
    c["opts"]["newton_rtol"] = 1e-12
    c["opts"]["eta"] = 1e-10
    c["opts"]["precond"] = 0
    m = Model(c)
    amp = 1e-6
    U = synth.random_state(c, 12, amp=(amp, amp, amp * 1e-2))
    U -= synth.initial_state(c) * 1.0                    # drop the bubble: pure small noise
    e0 = _energy(m, U)
    st = {}
    U1 = implicit_step(m, U, c["opts"], st)
    assert st["converged"]
    assert abs(_energy(m, U1) - e0) / e0 < 1e-7
    assert np.max(np.abs(U1 - U)) > 1e-3 * np.max(np.abs(U))  # the state did move


def test_acoustic_mode_cayley_amplification():
    """One implicit step multiplies an acoustic eigenmode by the Cayley transform
    (I - dt A/2)^{-1} (I + dt A/2) of the closed-form 3x3 symbol (trapezoid, Eq. ns)."""
    c = synth.case("tiny_32x16")
    c["sgs"]["K_M"] = c["sgs"]["K_H"] = 0.0
    c["opts"]["newton_rtol"] = 1e-12
    c["opts"]["eta"] = 1e-10
    c["opts"]["dt"] = 5.0
    m = Model(c)
    kx = 2 * math.pi * 3 / (m.nx * m.dx)
    kz = math.pi * 2 / (m.nz * m.dz)
    kxt = (8 * math.sin(kx * m.dx) - math.sin(2 * kx * m.dx)) / (6 * m.dx)
    kzt = (8 * math.sin(kz * m.dz) - math.sin(2 * kz * m.dz)) / (6 * m.dz)
    gp = m.gamma_p * m.pbar
    # amplitudes (U, W, P) of u = U sin cos, w = W cos sin, p = P cos cos
    A = np.array([[0.0, 0.0, m.theta0 * kxt],
                  [0.0, 0.0, m.theta0 * kzt],
                  [-gp * kxt, -gp * kzt, 0.0]])
    a0 = np.array([0.3, -0.2, 0.5e-3]) * 1e-6
    x = -0.5 * m.nx * m.dx + np.arange(m.nx) * m.dx
    z = (np.arange(m.nz) + 0.5) * m.dz
    X, Z = np.meshgrid(x, z, indexing="xy")
    modes = [np.sin(kx * X) * np.cos(kz * Z), np.cos(kx * X) * np.sin(kz * Z),
             np.cos(kx * X) * np.cos(kz * Z)]

    def state(a):
        return np.stack([a[0] * modes[0], a[1] * modes[1], np.zeros_like(X), a[2] * modes[2]])

    I = np.eye(3)
    dt = m.dt
    a1 = np.linalg.solve(I - 0.5 * dt * A, (I + 0.5 * dt * A) @ a0)
    U1 = implicit_step(m, state(a0), c["opts"])
    ref = state(a1)
    assert np.linalg.norm(m.scale(U1 - ref)) / np.linalg.norm(m.scale(ref)) < 1e-6


def test_newton_converges_thermal_128x64():
    c = synth.case("thermal_neutral_128x64")
    m = Model(c)
    U0 = synth.initial_state(c)
    st = {}
    U1 = implicit_step(m, U0, c["opts"], st)
    assert st["converged"] and 1 <= st["newton_iters"] <= 4
    h = st["residual_history"]
    assert all(h[i + 1] < 1e-2 * h[i] for i in range(len(h) - 1))
    # the returned state satisfies Eq. ns independently of the solver internals
    R = 2 * U1 / m.dt - m.F(U1) - 2 * U0 / m.dt - m.F(U0)
    assert np.linalg.norm(m.scale(R)) <= st["tol"] * 1.0000001
    # buoyancy accelerates the bubble upward
    assert U1[m.iw].max() > 0.05
