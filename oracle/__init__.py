"""Plain FP64 CPU oracle of the symmetry-preserving JFNK hot path (TEST INFRASTRUCTURE).

This package is the independent checker of the CUDA library.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the product path never does.  It shares no code with the CUDA
path: the only common inputs are the seeded fields and parameter sets of
``paper_2007_10411_gb300.synth`` (which contains no method arithmetic).

Everything is written as whole-array numpy in float64, following the paper's
statement of the method, with no blocking, fusion or reordering:

* ``wavelet``    Deslauriers-Dubuc refinement mask and the collocation
                 first-derivative weights phi'(l) (Section 2.3).
* ``operators``  ghost extension, derivatives, skew-symmetric convection
                 (Section 2.2), Smagorinsky eddy viscosity (Section 2.4),
                 the semi-discrete right-hand side F (Eqs. ch2_28-ch2_30, Eq. ds),
                 the trapezoidal residual R (Eq. ns), the finite-difference
                 Jacobian-vector product (Eq. fd), the field-block
                 preconditioner (Section 2.5.2), the acoustic Schur-complement
                 preconditioner (the semi-implicit elimination Section 2.5
                 follows) and the energy budgets (Section 3.1.3).
* ``krylov``     restarted right-preconditioned GMRES(m) with classical
                 Gram-Schmidt applied twice and Givens rotations (Section 2.5.1).
* ``newton``     the inexact Newton outer loop of one implicit step (Section 2.5.1),
                 with the field block or the acoustic Schur complement on the
                 right, or the nonlinear preconditioning of Section 2.5.2
                 (Newton on M^{-1} W R, GMRES on M^{-1} J_hat).

Parity status: every function is pinned by the tests in ``tests/test_oracle_*.py``
(closed forms, invariants, brute force); none is "parity unpinned" except the
long-time physical trajectory, which the paper reports only as figures.
"""
