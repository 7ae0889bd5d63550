"""Restarted, right-preconditioned GMRES(m) (Saad & Schultz 1986), float64 numpy.

TEST INFRASTRUCTURE (oracle only).  This is the Krylov solver of the inner
Newton loop (Section 2.5.1, Eq. jv): it minimises ||b - A x|| over the Krylov
space, with
* Arnoldi by classical Gram-Schmidt applied twice (CGS2),
* the Hessenberg least-squares problem reduced by Givens rotations,
* right preconditioning x = M^{-1} (V y) for a fixed linear M, or the flexible
  variant x = Z y with z_j = M^{-1} v_j stored (FGMRES, Saad 1993),
* zero initial guess, restart after m steps with the true residual b - A x,
* stopping when the rotated residual |g_{j+1}| <= eta ||b||, on a "lucky"
  breakdown h_{j+1,j} = 0, or after max_restarts restarts.
"""
from __future__ import annotations

import numpy as np


def givens(a: float, b: float):
    """Rotation (c, s) with [c s; -s c] [a; b] = [rho; 0]."""
    if b == 0.0:
        return 1.0, 0.0
    rho = float(np.hypot(a, b))
    return a / rho, b / rho


def cgs2(V: list, w: np.ndarray):
    """Orthogonalise w against the orthonormal v_0..v_j twice (classical Gram-Schmidt).

    Returns (h, h_next, v_next): h = h1 + h2 has j+1 entries, h_next = ||w'||
    and v_next = w'/h_next (w' the twice-projected vector).
    """
    Vm = np.stack([v.ravel() for v in V])
    wf = w.ravel().copy()
    h1 = Vm @ wf
    wf = wf - Vm.T @ h1
    h2 = Vm @ wf
    wf = wf - Vm.T @ h2
    hn = float(np.sqrt(wf @ wf))
    vnext = (wf / hn if hn > 0.0 else wf).reshape(w.shape)
    return h1 + h2, hn, vnext


def gmres(apply_A, b: np.ndarray, m: int, eta: float, max_restarts: int,
          precond=None, flexible: bool = False, record: dict | None = None):
    """Solve A x ~= b to ||b - A x|| <= eta ||b|| (right preconditioned, zero initial guess).

    ``apply_A`` and ``precond`` act on arrays shaped like ``b``.  ``record``
    (optional dict) receives the iteration count, the restart count, the
    rotated-residual history and, for the last cycle, the basis and the
    Hessenberg matrix.
    """
    M = precond if precond is not None else (lambda v: v)
    x = np.zeros_like(b)
    beta0 = float(np.sqrt(np.sum(b * b)))
    target = eta * beta0
    total, cycles = 0, 0
    history = []
    converged = beta0 == 0.0
    r = b
    while not converged and cycles <= max_restarts:
        beta = float(np.sqrt(np.sum(r * r)))
        V, Z = [r / beta], []
        Hbar = np.zeros((m + 1, m))      # Hessenberg as built by Arnoldi
        Rt = np.zeros((m, m))            # its rotated upper-triangular factor
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k, breakdown = 0, False
        for j in range(m):
            z = M(V[j])
            if flexible:
                Z.append(z)
            h, hn, vnext = cgs2(V, apply_A(z))
            Hbar[: j + 1, j] = h
            Hbar[j + 1, j] = hn
            col = Hbar[: j + 2, j].copy()
            for i in range(j):                       # apply the previous rotations
                t = cs[i] * col[i] + sn[i] * col[i + 1]
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1]
                col[i] = t
            cs[j], sn[j] = givens(col[j], col[j + 1])
            Rt[: j + 1, j] = col[: j + 1]
            Rt[j, j] = cs[j] * col[j] + sn[j] * col[j + 1]
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            total += 1
            history.append(abs(g[j + 1]))
            V.append(vnext)
            breakdown = hn == 0.0
            if abs(g[j + 1]) <= target or breakdown:
                break
        y = np.linalg.solve(np.triu(Rt[:k, :k]), g[:k])
        if flexible:
            dx = sum(yi * zi for yi, zi in zip(y, Z))
        else:
            dx = M(sum(yi * vi for yi, vi in zip(y, V[:k])))
        x = x + dx
        if record is not None:
            record["V"] = V
            record["Hbar"] = Hbar[: k + 1, :k]
        if history[-1] <= target or breakdown:
            converged = True
            break
        cycles += 1
        if cycles > max_restarts:
            break
        r = b - apply_A(x)
    if record is not None:
        record.update(iters=total, restarts=cycles, history=history, converged=converged)
    return x
