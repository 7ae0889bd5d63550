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


# ---------------------------------------------------------------- nonlinear preconditioning
def _diffusive_pair(K=1e4):
    import copy
    c = synth.case("thermal_stable_64x32")
    c["sgs"] = {"mode": synth.SGS_CONST, "K_M": K, "K_H": K, "Cs": 0.0, "Pr": 1.0}
    m = Model(copy.deepcopy(c))
    U = synth.random_state(c, 31, amp=(0.3, 0.1, 0.001))
    return m, U, m.rhs_f(U - 0.01)


def _nl_pin_error(m, U, f):
    a = m.nonlinear_pc_residual(U, f, 16)
    b = m.left_pc_residual(U, f, 16)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_nonlinear_pc_pin_unmutated():
    assert _nl_pin_error(*_diffusive_pair()) < 1e-12


def test_nonlinear_pc_pin_catches_a_wrong_block_operator():
    m, U, f = _diffusive_pair()
    good = m.block_operator
    m.block_operator = lambda K, x, fld: good(K, x, fld) * (1.0 if fld != 2 else 1.01)   # theta block 1 % off
    # precond keeps inverting the correct operator, so the planted error only
    # shows where block_apply is used: the paper's form carries (I - M^{-1} P) u
    m.precond = lambda Uf, R, sw: _precond_with(m, good, Uf, R, sw)
    assert _nl_pin_error(m, U, f) > 1e-6


def _precond_with(m, block_operator, U_frozen, Rhat, sweeps):
    """The field-block inverse built on a given block operator (the correct one)."""
    from oracle.operators import chebyshev
    K_M, K_H = m.frozen_eddy(U_frozen)
    Z = np.zeros_like(Rhat)
    for fld in range(m.nf):
        K = K_H if fld == m.ith else K_M
        kmax = float(np.max(K)) if not np.isscalar(K) else float(K)
        lo, hi = m.gershgorin_bounds(0.0 if fld == m.ip else kmax)
        Z[fld] = chebyshev(lambda x: block_operator(K, x, fld), Rhat[fld], lo, hi, sweeps)
    return Z


def test_nonlinear_pc_pin_catches_a_sign_error():
    m, U, f = _diffusive_pair()
    good = m.left_pc_residual
    m.left_pc_residual = lambda Uu, ff, sw: -good(Uu, ff, sw)          # b = +M^{-1} W R by mistake
    assert _nl_pin_error(m, U, f) > 1.0


def test_left_gmres_step_catches_a_right_hand_side_left_unpreconditioned():
    """Newton with GMRES on M^{-1} J but an unpreconditioned right-hand side
    converges to a wrong correction: the step no longer reaches the root in
    the same Newton count, or the state differs from the correct left step."""
    import copy
    c = synth.case("thermal_stable_64x32")
    c["sgs"] = {"mode": synth.SGS_CONST, "K_M": 1e4, "K_H": 1e4, "Cs": 0.0, "Pr": 1.0}
    c["opts"].update(krylov_m=12, eta=1e-8, newton_rtol=1e-11, max_newton=3, precond=4, pc_sweeps=2)
    U = synth.random_state(c, 31, amp=(0.3, 0.1, 0.001))
    st_good = {}
    good = implicit_step(Model(copy.deepcopy(c)), U, c["opts"], st_good)
    m = Model(copy.deepcopy(c))
    orig = m.precond
    calls = {"n": 0}

    def precond_skipping_rhs(Uf, R, sw):
        # the first application of the step is the one on the first right-hand side
        calls["n"] += 1
        return R if calls["n"] == 1 else orig(Uf, R, sw)
    m.precond = precond_skipping_rhs
    st_bad = {}
    bad = implicit_step(m, U, c["opts"], st_bad)
    err = float(np.linalg.norm(m.scale(bad - good)) / np.linalg.norm(m.scale(good)))
    assert (not st_bad["converged"]) or st_bad["newton_iters"] != st_good["newton_iters"] or err > 1e-9


# ------------------------------------------------- eddy viscosity and heat source
# Mistakes planted in copies of the oracle's Smagorinsky coefficient (Section 2.4)
# and surface heat source (Section 3.2) make the closed-form pins of
# test_oracle_sgs_heat fail.
import test_oracle_sgs_heat as sh    # noqa: E402


def _shear_nu_error(m, c):
    x, z, dx, dz = sh.grid_xyz(c)
    kz = math.pi * 2 / c["grid"]["lz"]
    U = np.zeros(synth.shape(c))
    U[0] = 0.7 * np.cos(kz * z)[:, None] * np.ones_like(x)[None, :]
    nu, _ = sh.interior_nu(m, U)
    expect = (0.18 * math.sqrt(dx * dz)) ** 2 * 0.7 * sh.ktil(kz, dz) * np.abs(np.sin(kz * z))[:, None]
    return np.max(np.abs(nu - expect)) / np.max(expect)


def test_smagorinsky_pin_unmutated():
    c = sh.smag_case()
    assert _shear_nu_error(Model(c), c) < 1e-12


def test_smagorinsky_without_the_factor_two_is_caught():
    c = sh.smag_case()
    m = Model(c)
    plain = m.smagorinsky_nu
    m.smagorinsky_nu = lambda g: plain(g) / math.sqrt(2.0)     # sqrt(S:S) instead of sqrt(2 S:S)
    assert _shear_nu_error(m, c) > 0.2


def test_smagorinsky_with_delta_dx_is_caught():
    c = sh.smag_case()
    m = Model(c)
    m.delta_les = m.dx
    assert _shear_nu_error(m, c) > 0.2


def test_smagorinsky_with_unsquared_cs_is_caught():
    c = sh.smag_case()
    m = Model(c)
    m.Cs = math.sqrt(m.Cs)            # (Cs Delta)^2 -> Cs Delta^2
    assert _shear_nu_error(m, c) > 0.2


class _HeatWithoutDz(Model):
    """Oracle copy whose surface source forgets the 1/dz of the bottom row."""

    def F(self, U):
        H = self.heat
        self.heat = None
        out = super().F(U)
        self.heat = H
        if H is not None:
            out[self.ith][0] += H / (self.rho0 * self.cp)
        return out


def _heat_pin_error(m, c):
    x, z, dx, dz = sh.grid_xyz(c)
    H = 50.0 + 40.0 * np.cos(2 * math.pi * x / c["grid"]["lx"]) ** 2
    m.set_heat_flux(H)
    F = m.F(np.zeros(synth.shape(c)))
    expect = H / (sh.RHO0 * sh.CP * dz)
    return np.max(np.abs(F[m.ith][0] - expect)) / np.max(expect)


def test_heat_source_pin_unmutated():
    c = sh.heat_case()
    assert _heat_pin_error(Model(c), c) < 1e-14


def test_heat_source_without_dz_is_caught():
    c = sh.heat_case()
    assert _heat_pin_error(_HeatWithoutDz(c), c) > 0.5


def test_heat_source_with_wrong_density_is_caught():
    c = sh.heat_case()
    m = Model(c)
    m.rho0 = 1.0e5 / (287.0 * 288.15)     # density at a standard 288 K, not theta0
    assert _heat_pin_error(m, c) > 1e-2


# ------------------------------------------------------------- Deardorff closure
import test_oracle_deardorff as tdd    # noqa: E402
from oracle.operators import SGS_DEARDORFF  # noqa: E402


class _DDMutant(Model):
    """Oracle copy whose Deardorff coefficients carry one planted mistake."""

    def __init__(self, case, mistake):
        super().__init__(case)
        self.mistake = mistake

    def deardorff(self, s):
        nu = (self.Cs * self.delta_les) ** 2 * s
        eps = nu * s * s / 2.0
        if self.mistake == "eps_2SS":
            eps = nu * s * s                       # nu 2 S_ij S_ij instead of nu S_ij S_ij
        c = self.Cs ** (4.0 / 3.0) * np.cbrt(eps)
        Km = c * (self.dx * self.dy_h) ** (2.0 / 3.0)
        KM = c * self.dz ** (2.0 / 3.0 if self.mistake == "dz_exponent" else 4.0 / 3.0)
        sqrt_e = nu / (0.1 * self.delta_les)
        if self.N2 > 0.0:
            l = 0.75 * sqrt_e / math.sqrt(self.N2)
            if self.mistake != "no_cap":
                l = np.minimum(self.delta_les, l)
        else:
            l = self.delta_les * np.ones_like(s)
        hh = self.dz if self.mistake == "ratio_dz" else math.sqrt(self.dx * self.dy_h)
        return Km, KM, (1.0 + 2.0 * l / hh) * Km, (1.0 + 2.0 * l / self.dz) * KM


def _dd_isotropic_error(m, c):
    U, s = tdd.shear_state(c, 0.9)
    (Kmx, KMz), (Khx, KHz) = (tdd.interior(m, K) for K in m.eddy(U))
    nu = (0.18 * m.dx) ** 2 * s
    return np.max(np.abs(Kmx - 2.0 ** (-1.0 / 3.0) * nu)) / nu.max()


def _dd_ratio_error(m):
    U, s = tdd.shear_state(m.case, 0.8, mode=2)
    (Kmx, KMz), (Khx, KHz) = (tdd.interior(m, K) for K in m.eddy(U))
    mask = s > 1e-3 * s.max()
    return max(np.max(np.abs(Kmx[mask] / KMz[mask] / (m.dx / m.dz) ** (4.0 / 3.0) - 1.0)),
               np.max(np.abs(Khx[mask] / Kmx[mask] - (1.0 + 2.0 * m.delta_les / m.dx))))


def _dd_cap_error(m, c):
    N = 0.01
    delta = m.delta_les
    s_cap = 0.1 * delta ** 2 * N / 0.75 / (0.18 * delta) ** 2
    U, s = tdd.shear_state(c, 1.0)
    U *= 4.0 * s_cap / s.max()
    s *= 4.0 * s_cap / s.max()
    (Kmx, _), (Khx, _) = (tdd.interior(m, K) for K in m.eddy(U))
    above = s > 1.1 * s_cap
    return np.max(np.abs(Khx[above] / Kmx[above] - (1.0 + 2.0 * delta / m.dx)))


def _mutant(case, mistake):
    m = _DDMutant(case, mistake) if mistake else Model(case)
    m.case = case
    return m


def test_deardorff_pins_unmutated():
    c = tdd.dd_case()
    assert _dd_isotropic_error(_mutant(c, None), c) < 1e-12
    assert _dd_ratio_error(_mutant(tdd.dd_case(dz_ratio=0.6), None)) < 1e-12
    cs = tdd.dd_case(beta=synth.brunt_beta(0.01))
    assert _dd_cap_error(_mutant(cs, None), cs) < 1e-12


def test_deardorff_dissipation_with_2SS_is_caught():
    c = tdd.dd_case()
    assert _dd_isotropic_error(_mutant(c, "eps_2SS"), c) > 0.1


def test_deardorff_vertical_exponent_is_caught():
    assert _dd_ratio_error(_mutant(tdd.dd_case(dz_ratio=0.6), "dz_exponent")) > 0.1


def test_deardorff_heat_ratio_length_is_caught():
    assert _dd_ratio_error(_mutant(tdd.dd_case(dz_ratio=0.6), "ratio_dz")) > 0.1


def test_deardorff_uncapped_mixing_length_is_caught():
    cs = tdd.dd_case(beta=synth.brunt_beta(0.01))
    assert _dd_cap_error(_mutant(cs, "no_cap"), cs) > 0.1


# ------------------------------------------------- 3-D network (oracle/unet.py)
def _expect_pin_failure(pin, monkeypatch, name, fake):
    from oracle import unet
    monkeypatch.setattr(unet, name, fake)
    try:
        pin()
    except AssertionError:
        return
    raise AssertionError("pin %s passed with a mutated %s" % (pin.__name__, name))


def test_3d_pool_that_subsamples_z_is_caught(monkeypatch):
    from oracle import unet
    from tests import test_oracle_unet as pins
    orig = unet.pool2

    def pool_even_plane(x):          # averages (y, x) but takes every other z plane
        if x.ndim == 3:
            return orig(x)
        return orig(x[:, 0::2].repeat(2, axis=1))
    _expect_pin_failure(pins.test_coarse_path_is_4x4x4_block_mean, monkeypatch, "pool2", pool_even_plane)


def test_3d_conv_over_the_wrong_planes_is_caught(monkeypatch):
    from oracle import unet
    from tests import test_oracle_unet as pins

    def conv_xz_planes(x, w):        # 3x3 over (z, x) for every y instead of (y, x) for every z
        if x.ndim == 3:
            return unet.conv(x, w)
        return np.stack([unet.conv(x[:, :, y], w) for y in range(x.shape[2])], axis=2)
    _expect_pin_failure(pins.test_conv_planes_matches_scipy_3d_correlate, monkeypatch, "conv_planes",
                        conv_xz_planes)


def test_3d_balance_on_the_2d_field_indices_is_caught(monkeypatch):
    from oracle import unet
    from tests import test_oracle_unet as pins
    orig = unet.balance

    def balance_2d_indices(case):    # theta / p factors on fields 2 and 3 (w, theta) in 3-D
        b = orig(case)
        if b.size == 5:
            b = np.array([1.0, 1.0, b[3], b[4], 1.0])
        return b
    _expect_pin_failure(pins.test_balance_3d_makes_the_couplings_skew, monkeypatch, "balance",
                        balance_2d_indices)


def test_3d_upsampling_that_skips_z_adjoint_is_caught(monkeypatch):
    from oracle import unet
    from tests import test_oracle_unet as pins
    orig = unet.up2_adjoint

    def adjoint_first_plane(d):      # sums the (y, x) children but reads only even z planes, twice
        if d.ndim == 3:
            return orig(d)
        return orig(d[:, 0::2].repeat(2, axis=1))
    _expect_pin_failure(pins.test_gradient_3d_with_balance_matches_central_differences, monkeypatch,
                        "up2_adjoint", adjoint_first_plane)
