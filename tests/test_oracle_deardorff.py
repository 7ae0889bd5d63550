"""Pins of the oracle's anisotropic Deardorff closure (Section 2.4, Eq. KmM).

Section 2.4 gives K_m = Cs^(4/3) eps^(1/3) (Dx Dy)^(2/3), K_M = Cs^(4/3) eps^(1/3) Dz^(4/3)
with eps = nu_tau S_ij S_ij, nu_tau = (Delta Cs)^2 sqrt(2 S_ij S_ij), and the heat
coefficients K_h = (1 + 2l/sqrt(Dx Dy)) K_m, K_H = (1 + 2l/Dz) K_M.  What fixes the
oracle here are consequences of those definitions worked out by hand, on strains
known in closed form (single Fourier modes, textbook fourth-order symbol k~):

* isotropic cells (Dx = Dz = Delta): eps^(1/3) = (Cs Delta)^(2/3) s / 2^(1/3) with
  s = sqrt(2 S:S), so K_m = K_M = 2^(-1/3) nu_tau, and with l capped at Delta,
  K_h = K_H = 3 K_m;
* anisotropic cells: K_m / K_M = (Dx / Dz)^(4/3) in 2-D (Dy read as Dx), and
  ((Dx Dy)^(1/2) / Dz)^(4/3) in 3-D;
* homogeneity: every coefficient is linear in the strain where l = Delta, and
  scales with Cs^2;
* stable stratification (N > 0): below the cap, l = 0.75 sqrt(e)/N with
  sqrt(e) = nu_tau / (0.1 Delta) (reading recorded in the oracle), so
  K_h / K_m - 1 = 2 l / Dx grows linearly with the strain until l reaches Delta;
* the anisotropic diffusion operator is symmetric negative semi-definite, and the
  forward-difference Jv matches central differences.
"""
import math

import numpy as np
import pytest

from oracle.operators import SGS_DEARDORFF, Model
from paper_2007_10411_gb300 import synth


def ktil(k, h):
    return (8 * math.sin(k * h) - math.sin(2 * k * h)) / (6 * h)


def dd_case(nx=16, nz=12, dz_ratio=1.0, beta=0.0, cs=0.18, dim=2, ny=10):
    c = synth.case("tiny_%dx%d" % (nx, nz))
    c["sgs"]["mode"] = SGS_DEARDORFF
    c["sgs"]["Cs"] = cs
    c["strat"]["beta"] = beta
    c["grid"]["lz"] *= dz_ratio
    if dim == 3:
        c["grid"].update(dim=3, ny=ny, ly=c["grid"]["lx"] * ny / nx)
    return c


def shear_state(c, A, mode=1):
    """u = A cos(kz z) (w = theta = p = 0): s = A kz~ |sin(kz z)| at every column."""
    g = c["grid"]
    dz = g["lz"] / g["nz"]
    z = (np.arange(g["nz"]) + 0.5) * dz
    kz = math.pi * mode / g["lz"]
    U = np.zeros(synth.shape(c))
    prof = A * np.cos(kz * z)
    U[0] = prof.reshape((-1,) + (1,) * (U.ndim - 2)) * np.ones(U.shape[1:])
    s = A * ktil(kz, dz) * np.abs(np.sin(kz * z))
    return U, s.reshape((-1,) + (1,) * (U.ndim - 2)) * np.ones(U.shape[1:])


def interior(m, K):
    return [m.crop(k, m.r) for k in K]


def test_isotropic_limit():
    c = dd_case()
    m = Model(c)
    assert m.dx == pytest.approx(m.dz)
    U, s = shear_state(c, 0.9)
    (Kmx, KMz), (Khx, KHz) = (interior(m, K) for K in m.eddy(U))
    nu = (0.18 * m.dx) ** 2 * s
    assert np.allclose(Kmx, 2.0 ** (-1.0 / 3.0) * nu, rtol=1e-12, atol=1e-14 * nu.max())
    assert np.allclose(KMz, Kmx, rtol=1e-13, atol=0)
    assert np.allclose(Khx, 3.0 * Kmx, rtol=1e-13, atol=0)     # neutral: l = Delta = Dx = Dz
    assert np.allclose(KHz, Khx, rtol=1e-13, atol=0)


def test_isotropic_limit_3d():
    c = dd_case(dim=3, ny=16)
    m = Model(c)
    assert m.dx == pytest.approx(m.dy) and m.dx == pytest.approx(m.dz)
    U, s = shear_state(c, 0.6)
    (Kx, Ky, Kz), (Hx, Hy, Hz) = (interior(m, K) for K in m.eddy(U))
    nu = (0.18 * m.dx) ** 2 * s
    for K in (Kx, Ky, Kz):
        assert np.allclose(K, 2.0 ** (-1.0 / 3.0) * nu, rtol=1e-12, atol=1e-14 * nu.max())
    for H in (Hx, Hy, Hz):
        assert np.allclose(H, 3.0 * Kx, rtol=1e-12, atol=0)


@pytest.mark.parametrize("ratio", [0.6, 1.7])
def test_anisotropic_ratio(ratio):
    c = dd_case(dz_ratio=ratio)
    m = Model(c)
    U, s = shear_state(c, 0.8, mode=2)
    (Kmx, KMz), _ = (interior(m, K) for K in m.eddy(U))
    mask = s > 1e-3 * s.max()
    assert np.allclose(Kmx[mask] / KMz[mask], (m.dx / m.dz) ** (4.0 / 3.0), rtol=1e-12)
    # absolute value: 2^(-1/3) (Cs^2 Delta^(2/3) s) Dx^(4/3) with Delta = (Dx Dz)^(1/2)
    delta = math.sqrt(m.dx * m.dz)
    expect = 2.0 ** (-1.0 / 3.0) * 0.18 ** 2 * delta ** (2.0 / 3.0) * m.dx ** (4.0 / 3.0) * s
    assert np.allclose(Kmx, expect, rtol=1e-12, atol=1e-14 * expect.max())


def test_anisotropic_ratio_3d():
    c = dd_case(dim=3, ny=10, dz_ratio=0.5)
    m = Model(c)
    U, s = shear_state(c, 0.8)
    (Kx, Ky, Kz), _ = (interior(m, K) for K in m.eddy(U))
    mask = s > 1e-3 * s.max()
    assert np.allclose(Kx, Ky, rtol=1e-14, atol=0)
    assert np.allclose(Kx[mask] / Kz[mask], (math.sqrt(m.dx * m.dy) / m.dz) ** (4.0 / 3.0), rtol=1e-12)


def test_linear_in_strain_and_quadratic_in_cs():
    c = dd_case(dz_ratio=0.7)
    m = Model(c)
    U, _ = shear_state(c, 0.5)
    U = U + 0.2 * synth.random_state(c, 9, amp=(1.0, 0.0, 0.0))
    K1 = [interior(m, K) for K in m.eddy(U)]
    K2 = [interior(m, K) for K in m.eddy(3.0 * U)]
    for a, b in zip(K1, K2):
        for x, y in zip(a, b):
            assert np.allclose(y, 3.0 * x, rtol=1e-12, atol=0)
    m2 = Model(dd_case(dz_ratio=0.7, cs=0.36))
    K3 = [interior(m2, K) for K in m2.eddy(U)]
    for a, b in zip(K1, K3):
        for x, y in zip(a, b):
            assert np.allclose(y, 4.0 * x, rtol=1e-12, atol=0)


def test_stable_mixing_length_regimes():
    N = 0.01
    c = dd_case(beta=synth.brunt_beta(N))
    m = Model(c)
    # the cap l = Delta is reached where nu_tau = 0.1 Delta^2 N / 0.75
    delta = m.delta_les
    s_cap = 0.1 * delta ** 2 * N / 0.75 / (0.18 * delta) ** 2
    U, s = shear_state(c, 1.0)
    U *= 4.0 * s_cap / s.max()
    s *= 4.0 * s_cap / s.max()
    (Kmx, KMz), (Khx, KHz) = (interior(m, K) for K in m.eddy(U))
    nu = (0.18 * delta) ** 2 * s
    l = np.minimum(delta, 0.75 * (nu / (0.1 * delta)) / N)
    below, above = s < 0.9 * s_cap, s > 1.1 * s_cap
    assert below.any() and above.any()
    ok = s > 1e-6 * s.max()
    assert np.allclose(Khx[ok] / Kmx[ok], 1.0 + 2.0 * l[ok] / m.dx, rtol=1e-12)
    assert np.allclose(KHz[ok] / KMz[ok], 1.0 + 2.0 * l[ok] / m.dz, rtol=1e-12)
    assert np.allclose(Khx[above] / Kmx[above], 1.0 + 2.0 * delta / m.dx, rtol=1e-12)
    # below the cap the excess ratio is proportional to the strain
    r = (Khx[below & ok] / Kmx[below & ok] - 1.0) / s[below & ok]
    assert np.allclose(r, r[0], rtol=1e-10)


@pytest.mark.parametrize("parity", [(1, 1), (-1, -1), (-1, 1)])
def test_anisotropic_diffusion_symmetric_nsd(parity):
    c = dd_case(nx=8, nz=8, dz_ratio=0.6, beta=synth.brunt_beta(0.01))
    m = Model(c)
    U = np.random.Generator(np.random.PCG64(5)).standard_normal(synth.shape(c))
    K_mom, K_heat = m.eddy(U)
    for K in (K_mom, K_heat):
        n = m.nz * m.nx
        A = np.zeros((n, n))
        for k in range(n):
            e = np.zeros(n)
            e[k] = 1.0
            P = m.extend(e.reshape(m.nz, m.nx), m.H, parity)
            A[:, k] = m.diffusion(K, m.grad_halo(P)).ravel()
        assert np.allclose(A, A.T, rtol=0, atol=1e-14 * np.max(np.abs(A)))
        assert np.max(np.linalg.eigvalsh(0.5 * (A + A.T))) <= 1e-12 * np.max(np.abs(A))


def test_rest_state_and_jv_central_difference():
    c = dd_case(nx=8, nz=8, beta=synth.brunt_beta(0.01))
    m = Model(c)
    Z = np.zeros(synth.shape(c))
    assert np.all(m.F(Z) == 0.0)
    U = synth.random_state(c, 8)
    V = np.random.Generator(np.random.PCG64(2)).standard_normal(U.shape)
    h = 1e-6
    cd = 2 * V / m.dt - (m.F(U + h * V) - m.F(U - h * V)) / (2 * h)
    jv = m.jv(U, m.F(U), V, 1e-7)
    assert np.linalg.norm((jv - cd).ravel()) / np.linalg.norm(cd.ravel()) < 1e-6


def test_block_preconditioner_bounds_cover_the_anisotropic_blocks():
    c = dd_case(nx=8, nz=8, dz_ratio=0.6, beta=synth.brunt_beta(0.01))
    m = Model(c)
    U = synth.random_state(c, 3)
    K_mom, K_heat = m.eddy(U)
    for f, K in ((0, K_mom), (m.ith, K_heat)):
        lo, hi = m.gershgorin_bounds(m.kmax_of(K))
        A = np.zeros((64, 64))
        for k in range(64):
            e = np.zeros(64)
            e[k] = 1.0
            A[:, k] = m.block_operator(K, e.reshape(8, 8), f).ravel()
        ev = np.linalg.eigvalsh(0.5 * (A + A.T))
        assert ev.min() >= lo * (1 - 1e-12) and ev.max() <= hi * (1 + 1e-12)
