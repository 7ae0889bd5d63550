"""The pins are sensitive: plausible mistakes planted in (copies of) the oracle make them fail.

Every mutation is applied to a throw-away Model instance on the CPU.
"""
import math

import numpy as np

from oracle.newton import implicit_step
from oracle.operators import Model
from paper_2007_10411_gb300 import synth


def _mode_state(m, a):
    kx = 2 * math.pi * 3 / (m.nx * m.dx)
    kz = math.pi * 2 / (m.nz * m.dz)
    x = -0.5 * m.nx * m.dx + np.arange(m.nx) * m.dx
    z = (np.arange(m.nz) + 0.5) * m.dz
    X, Z = np.meshgrid(x, z, indexing="xy")
    U = np.stack([a[0] * np.sin(kx * X) * np.cos(kz * Z), a[1] * np.cos(kx * X) * np.sin(kz * Z),
                  np.zeros_like(X), a[2] * np.cos(kx * X) * np.cos(kz * Z)])
    kxt = (8 * math.sin(kx * m.dx) - math.sin(2 * kx * m.dx)) / (6 * m.dx)
    kzt = (8 * math.sin(kz * m.dz) - math.sin(2 * kz * m.dz)) / (6 * m.dz)
    return U, X, Z, kx, kz, kxt, kzt


def _acoustic_pin_error(m):
    a = np.array([0.3, -0.2, 0.5e-3]) * 1e-7
    U, X, Z, kx, kz, kxt, kzt = _mode_state(m, a)
    F = m.F(U)
    ref_p = -m.gamma_p * m.pbar * (kxt * a[0] + kzt * a[1]) * np.cos(kx * X) * np.cos(kz * Z)
    ref_u = m.theta0 * kxt * a[2] * np.sin(kx * X) * np.cos(kz * Z)
    return max(np.max(np.abs(F[3] - ref_p)) / np.max(np.abs(ref_p)),
               np.max(np.abs(F[0] - ref_u)) / np.max(np.abs(ref_u)))


def _fresh(K=0.0):
    c = synth.case("tiny_32x16")
    c["sgs"]["K_M"] = c["sgs"]["K_H"] = K
    return Model(c)


def test_unmutated_passes():
    assert _acoustic_pin_error(_fresh()) < 1e-6


def test_transposed_stencil_is_caught():
    m = _fresh()
    m.d = {-l: v for l, v in m.d.items()}            # D u_j = sum d_l u_{j+l}: sign flip
    assert _acoustic_pin_error(m) > 0.5


def test_dropped_stencil_term_is_caught():
    m = _fresh()
    m.d = {l: v for l, v in m.d.items() if abs(l) == 1}  # second-order stencil by mistake
    assert _acoustic_pin_error(m) > 1e-3


def test_wrong_pressure_coefficient_is_caught():
    m = _fresh()
    m.gamma_p = 1004.0 / 717.0                         # c_p/c_v instead of R/c_v
    assert _acoustic_pin_error(_fresh()) < 1e-6
    m2 = _fresh()
    # the closed form is built from the reading gamma_p = R/c_v; the mutated model disagrees
    a = np.array([0.3, -0.2, 0.5e-3]) * 1e-7
    U, X, Z, kx, kz, kxt, kzt = _mode_state(m2, a)
    ref_p = -m2.gamma_p * m2.pbar * (kxt * a[0] + kzt * a[1]) * np.cos(kx * X) * np.cos(kz * Z)
    assert np.max(np.abs(m.F(U)[3] - ref_p)) > 0.5 * np.max(np.abs(ref_p))


def test_non_skew_convection_is_caught():
    c = synth.case("tiny_16x12")
    m = Model(c)
    orig = m.convection

    def flux_only(vel_pad, phi_pad, grad_phi_r):
        r = m.r
        return m.div_halo([m.crop(uj * phi_pad, r) for uj in vel_pad])
    r = np.random.Generator(np.random.PCG64(5))
    U = r.standard_normal(synth.shape(c))
    phi = r.standard_normal(U[0].shape)
    Pv = [m.extend(U[i], m.H, m.parity[i]) for i in m.vel]
    Pp = m.extend(phi, m.H, (1, 1))
    good = orig(Pv, Pp, m.grad_halo(Pp))
    bad = flux_only(Pv, Pp, m.grad_halo(Pp))
    assert abs(np.sum(phi * good)) < 1e-12 * np.sum(np.abs(phi * good))
    assert abs(np.sum(phi * bad)) > 1e-3 * np.sum(np.abs(phi * bad))


def test_wrong_stratification_sign_breaks_energy_conservation():
    c = synth.case("tiny_16x12")
    c["strat"]["beta"] = 3.058e-3
    c["sgs"]["K_M"] = c["sgs"]["K_H"] = 0.0
    c["opts"].update(newton_rtol=1e-12, eta=1e-10, precond=0)
    m = Model(c)
    beta = m.beta

    def energy(U):
        n2 = m.g * beta / m.theta0
        return 0.5 * (np.sum(U[0] ** 2) + np.sum(U[1] ** 2)) + \
            0.5 * m.g ** 2 / (m.theta0 ** 2 * n2) * np.sum(U[2] ** 2) + \
            0.5 * m.theta0 / (m.gamma_p * m.pbar) * np.sum(U[3] ** 2)
    U = synth.random_state(c, 12, amp=(1e-6, 1e-6, 1e-8)) - synth.initial_state(c)
    m.beta = -beta                                     # planted: +beta w instead of -beta w
    m.dt = 20.0
    U1 = implicit_step(m, U, c["opts"] | {"dt": 20.0})
    assert abs(energy(U1) - energy(U)) / energy(U) > 1e-4
