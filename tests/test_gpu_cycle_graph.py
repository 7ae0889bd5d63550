"""GMRES cycles launched as captured CUDA graphs against stream launches.

Every kernel of a fused Krylov step returns at entry once the device has
ended the cycle, so a graph that launches all m steps of a cycle (or
segments of them) must leave the same state, bit for bit, and the same
Krylov and Newton counts as stream launches polled after every step; the
segments are captured again after a change of tiles, surface flux or
preconditioner.  The stream path itself is checked against the float64
oracle by the parity tests.
"""
import numpy as np
import pytest

from paper_2007_10411_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def jf():
    from paper_2007_10411_gb300 import jfnk
    return jfnk


def stable_case(nx, nz, prec, m=20, precond=synth.PC_BLOCK, sweeps=2):
    c = synth.case("tiny_%dx%d" % (nx, nz))
    c["strat"]["beta"] = synth.brunt_beta(0.01)
    c["sgs"]["mode"] = synth.SGS_SMAGORINSKY
    c["opts"]["precision"] = prec
    c["opts"]["krylov_m"] = m
    c["opts"]["precond"] = precond
    c["opts"]["pc_sweeps"] = sweeps
    return c


def run(c, U, segment, steps=2):
    s = jf().Solver(c)
    s.set_cycle_graph(segment)
    u = torch.from_numpy(U.copy()).cuda()
    stats = [s.step(u) for _ in range(steps)]
    torch.cuda.synchronize()
    out = u.cpu().numpy()
    n = s.launch_count()
    s.close()
    return out, stats, n


def counts(stats):
    return [(st["newton_iters"], tuple(st["gmres_per_newton"][:st["newton_iters"]]), st["restarts"])
            for st in stats]


CASES = [
    ("thermal_neutral_128x64", None),                       # float64, GMRES(30), four sweeps
    ("stable_mixed_256x128", (256, 128, synth.PREC_MIXED, 20)),
    ("stable_fp64_100x37", (100, 37, synth.PREC_FP64, 8)),   # ragged tiles, restarts
    # three-pass cycles: acoustic Schur complement, nonlinear (left), none
    ("schur_mixed_130x70", (130, 70, synth.PREC_MIXED, 20, synth.PC_SCHUR, 8)),
    ("schur_fp64_64x32", (64, 32, synth.PREC_FP64, 4, synth.PC_SCHUR, 4)),
    ("nonlinear_mixed_128x64", (128, 64, synth.PREC_MIXED, 12, synth.PC_NONLINEAR, 2)),
    ("none_fp64_64x32", (64, 32, synth.PREC_FP64, 10, synth.PC_NONE, 2)),
]


@pytest.mark.parametrize("name,spec", CASES)
@pytest.mark.parametrize("segment", [1, 7, 32])
def test_graph_cycle_matches_stream_launches(name, spec, segment):
    c = synth.case(name) if spec is None else stable_case(*spec)
    U = synth.initial_state(c) if spec is None else synth.random_state(c, 11, amp=(0.5, 0.3, 0.002))
    ref, st_ref, n_ref = run(c, U, 0)
    got, st, n = run(c, U, segment)
    assert all(x["converged"] for x in st_ref)
    assert counts(st) == counts(st_ref)
    assert np.array_equal(got, ref)
    if segment == 32 and st_ref[0]["gmres_per_newton"][0] < c["opts"]["krylov_m"] - 2:
        # whole-cycle graphs launch every step of a cycle (those past its end return at once)
        assert n > n_ref


def test_graph_recaptured_after_tiles_flux_and_preconditioner_change():
    # also switches between the fused and three-pass cycles on one handle
    c = stable_case(128, 64, synth.PREC_MIXED, m=16)
    c["init"] = {"kind": "rest", "H0": 200.0, "patch_halfwidth": c["grid"]["lx"] / 5, "xi": 0.1, "l": 1.5}
    U = synth.random_state(c, 3, amp=(0.3, 0.1, 0.001))
    H = synth.heat_flux(c)
    results = []
    for segment in (0, 16):
        s = jf().Solver(c)
        s.set_cycle_graph(segment)
        s.set_surface_flux(torch.from_numpy(H).cuda())
        u = torch.from_numpy(U.copy()).cuda()
        seq = [s.step(u)]
        s.set_tiles(2, 3)
        seq.append(s.step(u))
        s.set_surface_flux(torch.from_numpy(2.0 * H).cuda())
        seq.append(s.step(u))
        s.set_precond(synth.PC_NONE)
        seq.append(s.step(u))
        s.set_precond(synth.PC_BLOCK)
        seq.append(s.step(u))
        s.set_precond(synth.PC_NONLINEAR)
        seq.append(s.step(u))
        seq.append(s.step(u))
        s.set_precond(synth.PC_BLOCK)
        seq.append(s.step(u))
        torch.cuda.synchronize()
        results.append((u.cpu().numpy(), counts(seq)))
        s.close()
    assert results[0][1] == results[1][1]
    assert np.array_equal(results[0][0], results[1][0])


def test_set_cycle_graph_argument_rules():
    c = stable_case(64, 32, synth.PREC_FP64)
    s = jf().Solver(c)
    with pytest.raises(jf().JfnkError):
        s.set_cycle_graph(-2)
    s.set_cycle_graph(-1)            # the default rule
    s.set_cycle_graph(1000)          # taken as m
    s.close()


@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
@pytest.mark.parametrize("every", [1, 3])
def test_kernel_timing_counts_only_launches_that_did_work(prec, every):
    # Event timing inside captured cycles and around stream launches counts
    # the same launches and bytes: one pass B per Hessenberg column, and the
    # steps enqueued past a cycle's end are left out in both modes.
    c = stable_case(128, 64, prec, m=12)
    U = synth.random_state(c, 7, amp=(0.5, 0.3, 0.002))
    out = []
    for segment in (0, 5):
        s = jf().Solver(c)
        s.set_cycle_graph(segment)
        u = torch.from_numpy(U.copy()).cuda()
        s.step(u)                                # the first cycles run before any capture
        s.kernel_timing(every=every)
        st = [s.step(u) for _ in range(2)]
        kt = s.kernel_timing_read()
        out.append((kt, sum(x["gmres_iters"] for x in st), u.cpu().numpy()))
        s.close()
    (k0, it0, u0), (k1, it1, u1) = out
    assert it0 == it1 and np.array_equal(u0, u1)
    if every == 1:
        assert k0["arnoldi_b"]["launches"] == it0 == k1["arnoldi_b"]["launches"]
    else:
        assert 0 < k0["arnoldi_b"]["launches"] < it0
    for fam in ("arnoldi_a", "arnoldi_b", "jv", "precond", "residual"):
        assert k0[fam]["launches"] == k1[fam]["launches"], fam
        assert k0[fam]["bytes"] == pytest.approx(k1[fam]["bytes"], rel=1e-12), fam
        assert k1[fam]["ms"] > 0.0, fam


def test_learned_cycles_in_graphs_match_stream_launches():
    # The learned correction's launches are captured with the cycle; a weight
    # change between steps changes the network's version and forces a new
    # capture, so graph and stream launches stay bit-identical.
    c = stable_case(256, 128, synth.PREC_MIXED, m=20, precond=synth.PC_UNET)
    U = synth.random_state(c, 21, amp=(0.3, 0.1, 0.001))
    results = []
    for segment in (0, 8):
        s = jf().Solver(c)
        s.set_cycle_graph(segment)
        s.unet_init(11)
        rng = np.random.default_rng(5)
        nw = s.unet_num_weights()
        s.unet_set_weights((0.01 * rng.standard_normal(nw)).astype(np.float32))
        u = torch.from_numpy(U.copy()).cuda()
        seq = [s.step(u) for _ in range(2)]
        s.unet_set_weights((0.02 * rng.standard_normal(nw)).astype(np.float32))
        seq += [s.step(u) for _ in range(2)]
        torch.cuda.synchronize()
        results.append((u.cpu().numpy(), counts(seq), [x["pc_switches"] for x in seq]))
        s.close()
    assert results[0][1] == results[1][1] and results[0][2] == results[1][2]
    assert np.array_equal(results[0][0], results[1][0])
