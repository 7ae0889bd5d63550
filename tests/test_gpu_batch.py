"""Batched heat-island instances (uneven grids, log-spaced surface heat flux):
a batch step equals the instances' individual steps, and one small instance
matches the FP64 oracle."""
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


def test_batch_step_equals_individual_steps():
    from paper_2007_10411_gb300 import jfnk
    cases = synth.uhi_batch(n=6, nx0=64, nz0=16)
    fluxes = [torch.from_numpy(synth.heat_flux(c)).cuda() for c in cases]
    b = jfnk.Batch(cases)
    for i, H in enumerate(fluxes):
        b.set_surface_flux(i, H)
    states = [torch.from_numpy(synth.random_state(c, 50 + i, amp=(0.2, 0.05, 0.001))).cuda()
              for i, c in enumerate(cases)]
    ref = [u.clone() for u in states]
    for _ in range(2):
        stats = b.step(states)
        assert all(s["converged"] for s in stats)
    torch.cuda.synchronize()
    for i, c in enumerate(cases):
        s = jfnk.Solver(c)
        s.set_surface_flux(fluxes[i])
        for _ in range(2):
            s.step(ref[i])
        torch.cuda.synchronize()
        assert torch.equal(states[i], ref[i]), i
        s.close()
    b.close()


def test_batch_instance_matches_oracle():
    from paper_2007_10411_gb300 import jfnk
    cases = synth.uhi_batch(n=2, nx0=48, nz0=16)
    for c in cases:
        c["opts"]["precision"] = synth.PREC_FP64
    b = jfnk.Batch(cases)
    Hs = [synth.heat_flux(c) for c in cases]
    for i, H in enumerate(Hs):
        b.set_surface_flux(i, torch.from_numpy(H).cuda())
    U0 = [synth.random_state(c, 7 + i, amp=(0.2, 0.05, 0.001)) for i, c in enumerate(cases)]
    states = [torch.from_numpy(u).cuda() for u in U0]
    b.step(states)
    torch.cuda.synchronize()
    for i, c in enumerate(cases):
        m = Model(c)
        m.set_heat_flux(Hs[i])
        ref = implicit_step(m, U0[i], c["opts"])
        got = states[i].cpu().numpy()
        err = np.linalg.norm(m.scale(got - ref)) / np.linalg.norm(m.scale(ref))
        assert err < 1e-10, (i, err)
    b.close()
