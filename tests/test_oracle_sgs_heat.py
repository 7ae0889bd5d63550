"""Pins of the oracle's eddy viscosity (Section 2.4) and surface heat source (Section 3.2).

Both are fixed by closed forms that use neither the oracle's derivative
weights nor its extension code:

* Smagorinsky nu = (Cs Delta)^2 sqrt(2 S_ij S_ij), Delta = (dx dz)^(1/2) in 2-D
  and (dx dy dz)^(1/3) in 3-D.  On single Fourier modes whose mirror images
  are the same analytic functions, the collocation derivative returns the
  textbook fourth-order symbol k~ (8 sin kh - sin 2kh) / (6h) times the exact
  derivative's mode, so nu has a closed form:
    shear     u = A cos(kz z):  S_13 = S_31 = -A kz~ sin(kz z)/2   ->  nu = (Cs Delta)^2 A kz~ |sin(kz z)|
    stretch   u = A sin(kx x):  S_11 = A kx~ cos(kx x)             ->  nu = (Cs Delta)^2 sqrt(2) A kx~ |cos(kx x)|
  The two differ by the sqrt(2) between diagonal and off-diagonal strain,
  and dx != dz on the test grids, so a dropped factor 2, a wrong Delta or an
  unsquared Cs each fail.
* The surface flux H(x) [W/m^2] heats the bottom row of theta at the rate
  H / (rho0 cp dz), rho0 = p0 / (R theta0): with the fluid at rest, F is zero
  everywhere else, and one implicit step raises the heat content
  sum(theta) dV by mean(H) Lx dt / (rho0 cp).
"""
import math

import numpy as np
import pytest

from oracle.newton import implicit_step
from oracle.operators import Model
from paper_2007_10411_gb300 import synth

# the constants of Section 2.1 written out here (not taken from the case)
P0, R_GAS, CP, THETA0 = 1.0e5, 287.0, 1004.0, 300.0
RHO0 = P0 / (R_GAS * THETA0)


def ktil(k, h):
    """Symbol of the textbook fourth-order central difference."""
    return (8 * math.sin(k * h) - math.sin(2 * k * h)) / (6 * h)


def smag_case(nx=16, nz=12, dim=2, ny=10, cs=0.18):
    c = synth.case("tiny_%dx%d" % (nx, nz))
    c["sgs"]["mode"] = synth.SGS_SMAGORINSKY
    c["sgs"]["Cs"] = cs
    c["grid"]["lz"] *= 0.6                  # dz = 0.6 dx
    if dim == 3:
        c["grid"].update(dim=3, ny=ny, ly=c["grid"]["lx"] * ny / nx * 0.7)
    return c


def interior_nu(m, U):
    nu_r, kh_r = m.eddy(U)
    r = m.r
    return m.crop(nu_r, r), m.crop(kh_r, r)


def grid_xyz(c):
    g = c["grid"]
    dx, dz = g["lx"] / g["nx"], g["lz"] / g["nz"]
    x = -0.5 * g["lx"] + np.arange(g["nx"]) * dx
    z = (np.arange(g["nz"]) + 0.5) * dz
    return x, z, dx, dz


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_smagorinsky_shear_mode_closed_form(mode):
    c = smag_case()
    m = Model(c)
    x, z, dx, dz = grid_xyz(c)
    assert abs(dx - dz) > 0.1 * dx          # Delta = dx or dz would be caught
    A = 0.7
    kz = math.pi * mode / c["grid"]["lz"]   # cos(kz z) is even about both walls: free slip
    U = np.zeros(synth.shape(c))
    U[0] = A * np.cos(kz * z)[:, None] * np.ones_like(x)[None, :]
    nu, kh = interior_nu(m, U)
    delta = math.sqrt(dx * dz)
    expect = (0.18 * delta) ** 2 * A * ktil(kz, dz) * np.abs(np.sin(kz * z))[:, None] * np.ones_like(x)
    assert np.allclose(nu, expect, rtol=1e-12, atol=1e-14 * np.max(expect))
    # K_H = nu / Pr (Section 2.4, Pr = 0.71)
    assert np.allclose(kh, expect / 0.71, rtol=1e-12, atol=1e-14 * np.max(expect))


@pytest.mark.parametrize("mode", [1, 3])
def test_smagorinsky_stretching_mode_closed_form(mode):
    c = smag_case()
    m = Model(c)
    x, z, dx, dz = grid_xyz(c)
    A = 0.4
    kx = 2 * math.pi * mode / c["grid"]["lx"]
    U = np.zeros(synth.shape(c))
    U[0] = np.ones_like(z)[:, None] * (A * np.sin(kx * x))[None, :]
    nu, _ = interior_nu(m, U)
    delta = math.sqrt(dx * dz)
    expect = (0.18 * delta) ** 2 * math.sqrt(2.0) * A * ktil(kx, dx) * np.abs(np.cos(kx * x))[None, :] \
        * np.ones_like(z)[:, None]
    assert np.allclose(nu, expect, rtol=1e-12, atol=1e-14 * np.max(expect))


def test_smagorinsky_shear_mode_closed_form_3d():
    c = smag_case(dim=3)
    m = Model(c)
    g = c["grid"]
    dx, dy, dz = g["lx"] / g["nx"], g["ly"] / g["ny"], g["lz"] / g["nz"]
    z = (np.arange(g["nz"]) + 0.5) * dz
    A = 0.5
    kz = 2 * math.pi / g["lz"]
    U = np.zeros(synth.shape(c))
    U[1] = A * np.cos(kz * z)[:, None, None] * np.ones((1, g["ny"], g["nx"]))   # v = A cos(kz z)
    nu, _ = interior_nu(m, U)
    delta = (dx * dy * dz) ** (1.0 / 3.0)
    expect = (0.18 * delta) ** 2 * A * ktil(kz, dz) * np.abs(np.sin(kz * z))[:, None, None] \
        * np.ones((1, g["ny"], g["nx"]))
    assert np.allclose(nu, expect, rtol=1e-12, atol=1e-14 * np.max(expect))


def heat_case(nx=32, nz=16):
    c = synth.case("tiny_%dx%d" % (nx, nz))
    c["strat"]["beta"] = 0.0
    return c


def test_surface_heat_source_at_rest_is_pointwise():
    c = heat_case()
    m = Model(c)
    x, z, dx, dz = grid_xyz(c)
    H = 50.0 + 40.0 * np.cos(2 * math.pi * x / c["grid"]["lx"]) ** 2
    m.set_heat_flux(H)
    F = m.F(np.zeros(synth.shape(c)))
    expect = H / (RHO0 * CP * dz)
    assert np.allclose(F[m.ith][0], expect, rtol=1e-14, atol=0)
    F[m.ith][0] = 0.0
    assert np.all(F == 0.0)


def test_surface_heat_source_heat_content_after_one_step():
    c = heat_case()
    c["opts"]["newton_rtol"] = 1e-11
    m = Model(c)
    x, z, dx, dz = grid_xyz(c)
    H = np.where(np.abs(x) < 0.25 * c["grid"]["lx"], 120.0, 10.0)
    m.set_heat_flux(H)
    U0 = np.zeros(synth.shape(c))
    st = {}
    U1 = implicit_step(m, U0, c["opts"], st)
    assert st["converged"]
    dV = dx * dz
    gained = np.sum(U1[m.ith] - U0[m.ith]) * dV
    dt = c["opts"]["dt"]
    expect = np.mean(H) * c["grid"]["lx"] * dt / (RHO0 * CP)
    # what is left is the O(dt^3) convective exchange started by the buoyancy of the heated row
    assert gained == pytest.approx(expect, rel=1e-7)
