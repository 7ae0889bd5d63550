"""Pins of the oracle's nonlinear preconditioning (Section 2.5.2).

The paper's preconditioned residual R~(u) = u - P^{-1}[f - L(u) + P u] equals
P^{-1} R(u) when P^{-1} is the exact inverse of the field-block operator P;
the oracle solves with M^{-1} R (M^{-1} the Chebyshev field-block inverse),
which keeps the root of R for any M.  Checked here: the two agree to rounding
once the Chebyshev inverse has converged and differ visibly when it has not
(the reason for the reading); left-preconditioned GMRES reproduces the
brute-force minimiser of ||M^{-1}(b - A x)|| over the Krylov space; a Newton
step with the nonlinear preconditioner reaches the same root as the right-
preconditioned one.
"""
import copy

import numpy as np

from oracle.krylov import gmres
from oracle.newton import implicit_step
from oracle.operators import Model
from paper_2007_10411_gb300 import synth


def _diffusive_case(K):
    c = synth.case("thermal_stable_64x32")
    c["sgs"] = {"mode": synth.SGS_CONST, "K_M": K, "K_H": K, "Cs": 0.0, "Pr": 1.0}
    return c


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_paper_formula_is_left_preconditioned_residual_for_exact_inverse():
    c = _diffusive_case(1e4)                  # K dt / dx^2 ~ 0.1: the block inverse is not trivial
    m = Model(c)
    U = synth.random_state(c, 31, amp=(0.3, 0.1, 0.001))
    f = m.rhs_f(U - 0.01)
    # converged Chebyshev inverse: u - P^{-1}(P u - W R) = P^{-1} W R to rounding
    assert _rel(m.nonlinear_pc_residual(U, f, 16), m.left_pc_residual(U, f, 16)) < 1e-12
    # two sweeps: the approximate inverse leaves (I - M^{-1} P) u in the paper's form
    assert _rel(m.nonlinear_pc_residual(U, f, 2), m.left_pc_residual(U, f, 2)) > 1e-6


def test_block_apply_is_the_operator_precond_inverts():
    c = _diffusive_case(1e4)
    m = Model(c)
    U = synth.random_state(c, 7, amp=(0.3, 0.1, 0.001))
    X = np.random.default_rng(3).standard_normal(U.shape)
    # M^{-1} P x -> x as the sweeps grow (Chebyshev on the Gershgorin interval of P)
    e2 = _rel(m.precond(U, m.block_apply(U, X), 2), X)
    e16 = _rel(m.precond(U, m.block_apply(U, X), 16), X)
    assert e16 < 1e-12 and e2 > 1e-6 and e16 < e2


def test_left_preconditioned_gmres_matches_brute_force():
    rng = np.random.default_rng(11)
    n = 10
    A = np.eye(n) * 3.0 + rng.standard_normal((n, n))
    Minv = np.eye(n) + 0.3 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    bt = Minv @ b
    for k in range(1, 6):
        x = gmres(lambda v: Minv @ (A @ v), bt, k, 0.0, 0)
        # Krylov space span{r, (M A) r, ..., (M A)^{k-1} r}, r = M b
        K = np.empty((n, k))
        v = bt.copy()
        for i in range(k):
            K[:, i] = v
            v = Minv @ (A @ v)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(Minv @ A @ Q, bt, rcond=None)
        np.testing.assert_allclose(x, Q @ y, rtol=1e-9, atol=1e-11)


def test_nonlinear_pc_step_reaches_the_same_root():
    c = _diffusive_case(1e4)
    c["opts"]["krylov_m"] = 12
    c["opts"]["eta"] = 1e-8
    c["opts"]["newton_rtol"] = 1e-11
    U = synth.random_state(c, 31, amp=(0.3, 0.1, 0.001))
    out = {}
    for pc in (1, 4):
        c2 = copy.deepcopy(c)
        c2["opts"]["precond"] = pc
        st = {}
        out[pc] = implicit_step(Model(c2), U, c2["opts"], st)
        assert st["converged"]
        m = Model(c2)
        R = m.residual(out[pc], m.rhs_f(U))
        assert np.linalg.norm(m.scale(R)) <= st["tol"]
    m = Model(c)
    assert _rel(m.scale(out[4]), m.scale(out[1])) < 1e-10
