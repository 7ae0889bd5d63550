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
    """One trapezoidal step u^n -> u^{n+1} (Eq. ns) by Newton-GMRES with the field-block PC."""
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
        if opts["precond"] == 1:
            pc = (lambda v, Uk=U: model.precond(Uk, v, opts["pc_sweeps"]))
        elif opts["precond"] == 3:
            pc = (lambda v, Uk=U: model.schur_precond(Uk, v, opts["pc_sweeps"]))
        else:
            pc = None
        rec = {}
        dhat = gmres(lambda v: model.jv_scaled(U, FU, v), b, opts["krylov_m"], opts["eta"],
                     opts["max_restarts"], precond=pc, flexible=bool(opts["flexible"]), record=rec)
        gm_iters.append(rec["iters"])
        U = U + model.unscale(dhat)
        R = model.residual(U, f)
        hist.append(norm(model.scale(R)))
        k += 1
    if stats is not None:
        stats.update(newton_iters=k, residual_history=hist, gmres_iters=gm_iters,
                     converged=hist[-1] <= tol, tol=tol)
    return U
