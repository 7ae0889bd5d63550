"""Deslauriers-Dubuc interpolating wavelets: refinement mask and derivative weights.

Section 2.3 of the paper: the collocation derivative of the interpolant
u^N(x) = sum_k u_k psi_k(x) at node x_j is sum_k u_k psi_k'(x_j), where
psi_k(x) = phi(x/dx - k) and phi is the Deslauriers-Dubuc fundamental
function of order p (support [-(2p-1), 2p-1], exact for polynomials of degree
2p-1).  So the weights are phi'(l) at the integers l.

phi is the fixed point of the two-scale relation phi(x) = sum_k h_k phi(2x-k)
whose mask h comes from midpoint Lagrange interpolation on 2p neighbouring
nodes.  Differentiating the relation and evaluating at integers gives the
eigen-problem  phi'(l) = 2 sum_k h_k phi'(2l-k)  with normalisation
sum_l l phi'(l) = -1 (derivative of the reproduction identity
sum_k k phi(x-k) = x).  We solve it directly with numpy (SVD null space).
"""
from __future__ import annotations

import numpy as np


def dd_mask(p: int) -> dict:
    """Refinement mask {k: h_k} of the order-p Deslauriers-Dubuc scheme.

    h_0 = 1, h_{2n} = 0 for n != 0, and h_{2n+1} is the weight that midpoint
    interpolation at x = 1/2 from nodes m = -p+1..p gives to node m = -n.
    """
    nodes = np.arange(-p + 1, p + 1, dtype=float)
    h = {0: 1.0}
    for m in nodes:
        others = nodes[nodes != m]
        w = np.prod((0.5 - others) / (m - others))  # Lagrange basis of node m at 1/2
        n = -int(m)
        h[2 * n + 1] = float(w)
    return h


def derivative_weights(p: int) -> dict:
    """Weights {l: d_l} with (D u)_j = (1/dx) sum_l d_l u_{j-l},  d_l = phi'(l).

    Only non-zero entries are returned (|l| <= 2p-2).
    """
    h = dd_mask(p)
    L = 2 * p - 1                         # phi' vanishes outside (-L, L)
    idx = np.arange(-L, L + 1)
    A = np.zeros((idx.size, idx.size))
    for a, l in enumerate(idx):
        for b, m in enumerate(idx):
            A[a, b] = 2.0 * h.get(int(2 * l - m), 0.0)
    # phi' is the eigenvector of A for eigenvalue 1 (i.e. null vector of A - I)
    _, s, vt = np.linalg.svd(A - np.eye(idx.size))
    v = vt[-1]
    v = v / -(idx @ v)                    # normalisation sum_l l phi'(l) = -1
    d = {int(l): float(val) for l, val in zip(idx, v) if abs(val) > 1e-13}
    return d


def radius(p: int) -> int:
    """Half-width of the derivative stencil (largest |l| with d_l != 0)."""
    return max(abs(l) for l in derivative_weights(p))
