"""Inexact Newton outer loop of one trapezoidal step (Section 2.5.1), float64 numpy.

TEST INFRASTRUCTURE (oracle only).

u^{n+1,0} = u^n;  u^{n+1,k+1} = u^{n+1,k} + du^k  with  J du^k = -R(u^{n+1,k})
solved by GMRES (Eq. jv), J applied matrix-free by the forward difference of
Eq. fd.  Everything Krylov-side lives in scaled units W = diag(1/U,..,1/Theta,1/P):
the solve is J_hat dhat = -W R with J_hat = W J W^{-1}, du = W^{-1} dhat.
Stopping rule: ||W R(u^k)|| <= max(rtol ||W R(u^0)||, atol_factor ||W 2u^n/dt||),
at most max_newton corrections.
"""
from __future__ import annotations

import numpy as np

from .krylov import gmres
from .operators import Model


def norm(a: np.ndarray) -> float:
    return float(np.sqrt(np.sum(a * a)))


def implicit_step(model: Model, Un: np.ndarray, opts: dict, stats: dict | None = None) -> np.ndarray:
    """One trapezoidal step u^n -> u^{n+1} (Eq. ns) by Newton-GMRES.

    precond 1: field block on the right; 3: acoustic Schur complement on the
    right; 4: nonlinear preconditioning (Section 2.5.2), Newton on the
    preconditioned residual M^{-1} W R with GMRES on M^{-1} J_hat; 0: none.
    The Newton test is on ||W R|| in every case."""
    f = model.rhs_f(Un)
    U = Un.copy()
    R = model.residual(U, f)
    r0 = norm(model.scale(R))
    tol = max(opts["newton_rtol"] * r0,
              opts["newton_atol_factor"] * norm(model.scale(2.0 * Un / model.dt)))
    hist = [r0]
    gm_iters = []
    k = 0
    while hist[-1] > tol and k < opts["max_newton"]:
        FU = model.F(U)
        b = -model.scale(R)
        pc = None
        apply_J = (lambda v, Uk=U, FUk=FU: model.jv_scaled(Uk, FUk, v))
        if opts["precond"] == 1:
            pc = (lambda v, Uk=U: model.precond(Uk, v, opts["pc_sweeps"]))
        elif opts["precond"] == 3:
            pc = (lambda v, Uk=U: model.schur_precond(Uk, v, opts["pc_sweeps"]))
        elif opts["precond"] == 4:
            # nonlinear preconditioning: Newton on M^{-1} W R, i.e. GMRES on
            # M^{-1} J_hat (left) with the field block M frozen at u^k
            ML = (lambda v, Uk=U: model.precond(Uk, v, opts["pc_sweeps"]))
            b = ML(b)
            apply_J = (lambda v, Jk=apply_J, MLk=ML: MLk(Jk(v)))
        rec = {}
        dhat = gmres(apply_J, b, opts["krylov_m"], opts["eta"], opts["max_restarts"], precond=pc,
                     flexible=bool(opts["flexible"]) and pc is not None, record=rec)
        gm_iters.append(rec["iters"])
        U = U + model.unscale(dhat)
        R = model.residual(U, f)
        hist.append(norm(model.scale(R)))
        k += 1
    if stats is not None:
        stats.update(newton_iters=k, residual_history=hist, gmres_iters=gm_iters,
                     converged=hist[-1] <= tol, tol=tol)
    return U
