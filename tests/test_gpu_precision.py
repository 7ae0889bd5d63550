"""Per-field error of the mixed-precision path on the stable-thermal workload.

The mixed path runs the stencils, the preconditioner and the Krylov basis
in float32 and keeps float64 for the Newton residual, the difference
quotient's scaling, the Hessenberg / Givens solve and the Newton update.
Both sides stop at the same Newton test on the float64 residual
(||W R|| <= 1e-8 ||W R0||), so the two states are two roots of Eq. ns to
that tolerance: the per-field bound 1e-4 (relative L2) is the mixed-path
tolerance, checked on the state and on the step's increment.

* 256 x 128, same physics as the 1024 x 512 benchmark (stable thermal,
  Smagorinsky, bubble plus noise): GPU mixed step against the float64
  oracle's step (about 3 s of oracle time).
* 1024 x 512, the benchmark workload itself: a whole oracle step takes
  minutes, so the mixed step is compared with the GPU's float64 step from
  the same state, whose parity with the oracle is fixed at 1e-10 on the
  smaller grids of test_gpu_parity.
"""
import numpy as np
import pytest

from oracle.newton import implicit_step
from oracle.operators import Model
from paper_2007_10411_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def rel_per_field(got, ref):
    out = []
    for f in range(ref.shape[0]):
        den = np.linalg.norm(ref[f])
        out.append(np.linalg.norm(got[f] - ref[f]) / (den if den > 0 else 1.0))
    return np.array(out)


def gpu_step(c, U0):
    from paper_2007_10411_gb300 import jfnk
    s = jfnk.Solver(c)
    u = torch.from_numpy(U0.copy()).cuda()
    st = s.step(u)
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    s.close()
    return got, st


def test_mixed_step_per_field_error_against_oracle_256x128():
    c = synth.case("thermal_stable_256x128")
    assert c["opts"]["precision"] == synth.PREC_MIXED
    m = Model(c)
    U0 = synth.initial_state(c)
    st_ref = {}
    ref = implicit_step(m, U0, c["opts"], st_ref)
    got, st = gpu_step(c, U0)
    assert st["converged"] and st_ref["converged"]
    e_state = rel_per_field(got, ref)
    e_inc = rel_per_field(got - U0, ref - U0)
    print("per-field relative L2 (u, w, theta, p): state", e_state, "increment", e_inc)
    assert np.all(e_state < 1e-4), e_state
    assert np.all(e_inc < 1e-4), e_inc


def test_mixed_step_per_field_error_against_fp64_1024x512():
    c = synth.case("thermal_stable_1024x512")
    U0 = synth.initial_state(c)
    got, st = gpu_step(c, U0)
    ref, st64 = gpu_step(synth.with_options(c, precision=synth.PREC_FP64), U0)
    assert st["converged"] and st64["converged"]
    e_state = rel_per_field(got, ref)
    e_inc = rel_per_field(got - U0, ref - U0)
    print("per-field relative L2 (u, w, theta, p): state", e_state, "increment", e_inc)
    assert np.all(e_state < 1e-4), e_state
    assert np.all(e_inc < 1e-4), e_inc
