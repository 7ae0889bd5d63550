"""Learned right preconditioner on the GPU: the tensor-core network against the
float64 oracle (forward and gradient), the training pairs the solver records,
training, and the gain over the field-block preconditioner alone.

Tolerances.  The GPU network rounds its input and every activation to
bfloat16 (unit roundoff u = 2^-9) and accumulates in float32; weights are
chosen bfloat16-representable so that both sides use the same ones.  The
deepest path rounds 12 times, so the expected relative error of the output
is about sqrt(12) u ~ 7e-3 for well-scaled weights; the forward bound is
2e-2.  Gradients add the rounding of the output gradient and of the
back-propagated activations (about twice as many roundings) and a float32
sum over every pixel: the expected per-layer error is about sqrt(24) u ~ 1e-2
at most; the bound is 1e-2 per layer (relative L2 of the layer's gradient
block), the tolerance set for the bfloat16 network (measured: 6e-4 .. 6e-3).
"""
import numpy as np
import pytest

from oracle import unet as ou
from oracle.operators import Model
from paper_2007_10411_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def random_weights(seed: int, nf: int = 4) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for (name, ci, co, k) in ou.LAYERS:
        fan = k * k * (nf if name == "L0a" else ci)
        w = rng.standard_normal((k * k, co, ci)) / np.sqrt(fan)
        if name == "L0a":
            w[:, :, nf:] = 0.0           # padded input channels carry zeros
        parts.append(w.reshape(-1))
    return bf16_round(np.concatenate(parts).astype(np.float32))


def learned_case(name: str) -> dict:
    c = synth.case(name)
    c["opts"]["precision"] = synth.PREC_MIXED
    c["opts"]["precond"] = 2
    return c


def rel(a, b) -> float:
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / np.linalg.norm(np.asarray(b, float)))


ENGINES = [0, 1]     # jfnk.UNET_TCGEN05 (default), jfnk.UNET_MMA_SYNC


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("name", ["tiny_64x32", "tiny_96x64"])
def test_forward_matches_oracle(name, engine):
    from paper_2007_10411_gb300 import jfnk
    c = learned_case(name)
    s = jfnk.Solver(c)
    s.unet_init(1)
    s.unet_set_engine(engine)
    w = random_weights(11)
    assert s.unet_num_weights() == w.size == ou.num_weights()
    s.unet_set_weights(w)
    np.testing.assert_array_equal(s.unet_get_weights(), w)
    nz, nx = c["grid"]["nz"], c["grid"]["nx"]
    X = np.random.default_rng(3).standard_normal((4, nz, nx)).astype(np.float32)
    xd = torch.from_numpy(X).cuda().reshape(-1)
    yd = torch.empty_like(xd)
    s.unet_forward(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy().reshape(4, nz, nx)
    ref = ou.apply(w.astype(np.float64), X.astype(np.float64), ou.balance(c))
    e = rel(y, ref)
    assert e < 2e-2, e
    # per field as well (no field may be badly off while the total is fine)
    for f in range(4):
        assert rel(y[f], ref[f]) < 3e-2, (f, rel(y[f], ref[f]))
    s.unet_status()
    s.close()


def test_zero_init_network_is_zero_and_block_pc_unchanged():
    from paper_2007_10411_gb300 import jfnk
    c = learned_case("tiny_64x32")
    s = jfnk.Solver(c)
    s.unet_init(5)
    nz, nx = c["grid"]["nz"], c["grid"]["nx"]
    xd = torch.randn(4 * nz * nx, device="cuda", dtype=torch.float32)
    yd = torch.full_like(xd, 7.0)
    s.unet_forward(xd, yd)
    torch.cuda.synchronize()
    assert torch.count_nonzero(yd).item() == 0
    s.close()


@pytest.mark.parametrize("engine", ENGINES)
def test_gradient_matches_oracle(engine):
    from paper_2007_10411_gb300 import jfnk
    c = learned_case("tiny_64x32")
    s = jfnk.Solver(c)
    s.unet_init(2)
    s.unet_set_engine(engine)
    w = random_weights(12)
    s.unet_set_weights(w)
    nz, nx = c["grid"]["nz"], c["grid"]["nx"]
    rng = np.random.default_rng(4)
    X = rng.standard_normal((4, nz, nx)).astype(np.float32)
    T = rng.standard_normal((4, nz, nx)).astype(np.float32)
    loss, g = s.unet_loss_grad(torch.from_numpy(X).cuda().reshape(-1), torch.from_numpy(T).cuda().reshape(-1))
    L_ref, g_ref = ou.loss_grad(w.astype(np.float64), X.astype(np.float64), T.astype(np.float64), ou.balance(c))
    assert abs(loss - L_ref) <= 2e-2 * L_ref, (loss, L_ref)
    offs = np.concatenate([[0], np.cumsum(ou.layer_sizes())])
    errs = {}
    for li, (name, ci, co, k) in enumerate(ou.LAYERS):
        a, b = g[offs[li]:offs[li + 1]], g_ref[offs[li]:offs[li + 1]]
        if name == "L0a":   # padded input channels: both zero
            a = a.reshape(k * k, co, ci)[:, :, :4]
            b = b.reshape(k * k, co, ci)[:, :, :4]
        errs[name] = rel(a, b)
    print("per-layer gradient relative L2:", {k: "%.2e" % v for k, v in errs.items()})
    for name, e in errs.items():
        assert e < 1e-2, (name, e)
    s.close()


def _pc_state(c, seed):
    return synth.random_state(c, seed, amp=(0.5, 0.1, 0.002))


@pytest.mark.parametrize("kinds", [1, 2])
def test_recorded_pairs_follow_definition(kinds):
    """Newton pairs: X = -W R / ||W R|| at u^n.  Both kinds: J_hat (M^-1 X + T) = X.

    The bound 1e-3 covers the GMRES tolerance eta = 1e-4 (Newton pairs), the
    float32 Jacobian product of the mixed path against the float64 oracle
    (relative 1e-4) and the float32 storage of the pair.
    """
    from paper_2007_10411_gb300 import jfnk
    c = synth.case("thermal_stable_64x32")
    c["opts"]["precision"] = synth.PREC_MIXED
    s = jfnk.Solver(c)
    s.unet_capture(4, kinds)
    U0 = _pc_state(c, 21)
    u = torch.from_numpy(U0.reshape(-1).copy()).cuda()
    st = s.step(u)
    assert st["converged"]
    expect = min(4, st["newton_iters"] if kinds == 1 else st["gmres_iters"])
    assert s.unet_pair_count() == expect
    n = U0.size
    Xd = torch.empty(n, device="cuda", dtype=torch.float32)
    Td = torch.empty_like(Xd)
    s.unet_get_pair(0, Xd, Td)
    torch.cuda.synchronize()
    X = Xd.cpu().numpy().astype(np.float64).reshape(U0.shape)
    T = Td.cpu().numpy().astype(np.float64).reshape(U0.shape)
    m = Model(c)
    if kinds == 1:
        b = -m.scale(m.residual(U0, m.rhs_f(U0)))
        assert rel(X, b / np.linalg.norm(b)) < 1e-6
    assert abs(np.linalg.norm(X) - 1.0) < 1e-5
    Y = T + m.precond(U0, X, c["opts"]["pc_sweeps"])
    res = np.linalg.norm(X - m.jv_scaled(U0, m.F(U0), Y))
    assert res <= 10 * c["opts"]["eta"], res
    s.unet_capture(0, 0)
    assert s.unet_pair_count() == 0
    s.close()


def test_training_reduces_loss_and_checkpoint_round_trip():
    from paper_2007_10411_gb300 import jfnk
    c = synth.case("thermal_stable_128x64")
    c["opts"]["precision"] = synth.PREC_MIXED
    c["opts"]["precond"] = 2
    s = jfnk.Solver(c)
    s.unet_init(7)
    s.unet_capture(64, jfnk.PAIRS_ARNOLDI)
    u = torch.from_numpy(_pc_state(c, 31).reshape(-1).copy()).cuda()
    for _ in range(3):
        s.step(u)
    assert s.unet_pair_count() >= 32
    hist = s.unet_train(20, 3e-4)
    assert hist[-1] < 0.3 * hist[0], hist
    w = s.unet_get_weights()
    assert np.all(np.isfinite(w))
    # checkpoint round trip: a second handle with the same weights gives the same output
    s2 = jfnk.Solver(c)
    s2.unet_init(99)
    s2.unet_set_weights(w)
    x = torch.randn(u.numel(), device="cuda", dtype=torch.float32)
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    s.unet_forward(x, y1)
    s2.unet_forward(x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    s.close()
    s2.close()


def test_unsupported_configurations():
    from paper_2007_10411_gb300 import jfnk
    c = synth.case("tiny_64x32")
    c["opts"]["precision"] = synth.PREC_FP64
    s = jfnk.Solver(c)
    with pytest.raises(jfnk.JfnkError) as e:
        s.unet_init(0)
    assert e.value.code == jfnk.JFNK_ERR_UNSUPPORTED
    with pytest.raises(jfnk.JfnkError) as e:
        s.set_precond(jfnk.PC_UNET)
    assert e.value.code == jfnk.JFNK_ERR_UNSUPPORTED
    s.close()
    c = synth.case("tiny_48x32")
    c["opts"]["precision"] = synth.PREC_MIXED
    c["opts"]["precond"] = 2
    with pytest.raises(jfnk.JfnkError) as e:
        jfnk.Solver(c)
    assert e.value.code == jfnk.JFNK_ERR_UNSUPPORTED


def _run_steps(s, u, mode, k):
    s.set_precond(mode)
    v = u.clone()
    stats = [s.step(v) for _ in range(k)]
    torch.cuda.synchronize()
    return v, stats


def test_untrained_network_matches_block_preconditioner():
    """N = 0 at initialisation, so P = M^-1 and the solver takes the same path."""
    from paper_2007_10411_gb300 import jfnk
    c = learned_case("thermal_stable_128x64")
    s = jfnk.Solver(c)
    s.unet_init(3)
    u = torch.from_numpy(synth.initial_state(c).reshape(-1).copy()).cuda()
    vb, sb = _run_steps(s, u, jfnk.PC_BLOCK, 2)
    vl, sl = _run_steps(s, u, jfnk.PC_UNET, 2)
    for a, b in zip(sb, sl):
        assert a["converged"] and b["converged"]
        assert abs(a["gmres_iters"] - b["gmres_iters"]) <= 2, (a["gmres_iters"], b["gmres_iters"])
    assert float((vb - vl).norm() / vb.norm()) < 1e-6
    s.close()


def test_trained_network_gain_over_block_preconditioner():
    """What the trained network gains on the stable thermal at 256x128.

    Pairs: every Arnoldi step of two plain (field-block preconditioned) steps;
    40 epochs of Adam.  Then two steps from the same state with the field-block
    preconditioner alone and with P = M^-1 + N: both meet the Newton tolerance
    (the states agree to it), and the learned preconditioner needs at most 70%
    of the Krylov iterations (about 50% when measured), with no safeguard
    switching back to the block preconditioner.
    """
    from paper_2007_10411_gb300 import jfnk
    c = learned_case("thermal_stable_256x128")
    s = jfnk.Solver(c)
    s.set_precond(jfnk.PC_BLOCK)
    s.unet_init(7)
    s.unet_capture(256, jfnk.PAIRS_ARNOLDI)
    u = torch.from_numpy(synth.initial_state(c).reshape(-1).copy()).cuda()
    for _ in range(2):
        s.step(u)
    assert s.unet_pair_count() >= 128
    hist = s.unet_train(40, 3e-4)
    assert hist[-1] < 0.05 * hist[0], hist
    s.unet_capture(0, 0)
    vb, sb = _run_steps(s, u, jfnk.PC_BLOCK, 2)
    vl, sl = _run_steps(s, u, jfnk.PC_UNET, 2)
    gb = sum(x["gmres_iters"] for x in sb)
    gl = sum(x["gmres_iters"] for x in sl)
    print("gmres iterations: block %d, learned %d" % (gb, gl))
    assert all(x["converged"] for x in sb + sl)
    assert not any(x["pc_fallback"] for x in sl)
    assert sum(x["pc_switches"] for x in sl) == 0
    assert gl <= 0.7 * gb, (gb, gl)
    assert float((vb - vl).norm() / vb.norm()) < 1e-6
    s.close()


def test_engines_agree_on_the_benchmark_grid():
    """The tcgen05 and mma.sync convolutions compute the same network: on the 1024 x 512
    grid (several persistent tiles per CTA, every layer shape) their outputs differ only
    by the bfloat16 rounding of activations that sit on a rounding boundary."""
    from paper_2007_10411_gb300 import jfnk
    c = learned_case("thermal_stable_1024x512")
    s = jfnk.Solver(c)
    s.unet_init(3)
    w = random_weights(13)
    s.unet_set_weights(w)
    nz, nx = c["grid"]["nz"], c["grid"]["nx"]
    x = torch.randn(4 * nz * nx, device="cuda", dtype=torch.float32, generator=torch.Generator("cuda").manual_seed(9))
    ys = []
    for engine in ENGINES:
        s.unet_set_engine(engine)
        y = torch.empty_like(x)
        s.unet_forward(x, y)
        s.unet_status()
        ys.append(y.cpu().numpy())
    assert rel(ys[0], ys[1]) < 1e-2, rel(ys[0], ys[1])
    s.close()


# ------------------------------------------------------------------ 3-D grids
# thermal3d_<nx>x<ny>x<nz>: stable stratification, so both balance factors are
# non-trivial; 32x64x8 has several 16-row tiles per slice at level 0 and one at
# level 2, 64x128x4 a single slice at level 2 (nz = 4 pools twice).
CASES_3D = ["thermal3d_32x64x8", "thermal3d_64x128x4"]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("name", CASES_3D)
def test_forward_3d_matches_oracle(name, engine):
    from paper_2007_10411_gb300 import jfnk
    c = learned_case(name)
    s = jfnk.Solver(c)
    s.unet_init(1)
    s.unet_set_engine(engine)
    w = random_weights(21, nf=5)
    s.unet_set_weights(w)
    shape = synth.shape(c)
    assert shape[0] == 5
    X = np.random.default_rng(5).standard_normal(shape).astype(np.float32)
    xd = torch.from_numpy(X).cuda().reshape(-1)
    yd = torch.empty_like(xd)
    s.unet_forward(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy().reshape(shape)
    ref = ou.apply(w.astype(np.float64), X.astype(np.float64), ou.balance(c))
    e = rel(y, ref)
    assert e < 2e-2, e
    for f in range(5):
        assert rel(y[f], ref[f]) < 3e-2, (f, rel(y[f], ref[f]))
    s.unet_forward(xd, yd)      # same output again: bitwise reproducible
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy().reshape(shape), y)
    s.unet_status()
    s.close()


@pytest.mark.parametrize("engine", ENGINES)
def test_gradient_3d_matches_oracle(engine):
    from paper_2007_10411_gb300 import jfnk
    c = learned_case("thermal3d_32x64x8")
    s = jfnk.Solver(c)
    s.unet_init(2)
    s.unet_set_engine(engine)
    w = random_weights(22, nf=5)
    s.unet_set_weights(w)
    shape = synth.shape(c)
    rng = np.random.default_rng(6)
    X = rng.standard_normal(shape).astype(np.float32)
    T = rng.standard_normal(shape).astype(np.float32)
    loss, g = s.unet_loss_grad(torch.from_numpy(X).cuda().reshape(-1), torch.from_numpy(T).cuda().reshape(-1))
    L_ref, g_ref = ou.loss_grad(w.astype(np.float64), X.astype(np.float64), T.astype(np.float64), ou.balance(c))
    assert abs(loss - L_ref) <= 2e-2 * L_ref, (loss, L_ref)
    offs = np.concatenate([[0], np.cumsum(ou.layer_sizes())])
    errs = {}
    for li, (name, ci, co, k) in enumerate(ou.LAYERS):
        a, b = g[offs[li]:offs[li + 1]], g_ref[offs[li]:offs[li + 1]]
        if name == "L0a":
            a = a.reshape(k * k, co, ci)[:, :, :5]
            b = b.reshape(k * k, co, ci)[:, :, :5]
        errs[name] = rel(a, b)
    print("3-D per-layer gradient relative L2:", {k: "%.2e" % v for k, v in errs.items()})
    for name, e in errs.items():
        assert e < 1e-2, (name, e)
    s.close()


def test_3d_untrained_network_matches_block_and_trained_network_converges():
    """3-D learned preconditioner on a small stable thermal: with N = 0 the
    solver follows the field-block path; after training on its own Arnoldi
    pairs the learned steps still meet the Newton tolerance (same state)."""
    from paper_2007_10411_gb300 import jfnk
    c = learned_case("thermal3d_64x64x32")
    s = jfnk.Solver(c)
    s.unet_init(3)
    u = torch.from_numpy(synth.initial_state(c).reshape(-1).copy()).cuda()
    vb, sb = _run_steps(s, u, jfnk.PC_BLOCK, 1)
    vl, sl = _run_steps(s, u, jfnk.PC_UNET, 1)
    assert sb[0]["converged"] and sl[0]["converged"]
    assert abs(sb[0]["gmres_iters"] - sl[0]["gmres_iters"]) <= 2
    assert float((vb - vl).norm() / vb.norm()) < 1e-6
    s.set_precond(jfnk.PC_BLOCK)
    s.unet_capture(64, jfnk.PAIRS_ARNOLDI)
    s.step(u.clone())
    assert s.unet_pair_count() >= 16
    hist = s.unet_train(10, 3e-4)
    assert hist[-1] < 0.5 * hist[0], hist
    s.unet_capture(0, 0)
    vl, sl = _run_steps(s, u, jfnk.PC_UNET, 1)
    print("3-D gmres iterations: block %d, learned %d" % (sb[0]["gmres_iters"], sl[0]["gmres_iters"]))
    assert sl[0]["converged"] and not sl[0]["pc_fallback"]
    assert float((vb - vl).norm() / vb.norm()) < 1e-6
    s.close()


def test_3d_unsupported_grids():
    from paper_2007_10411_gb300 import jfnk
    for name in ("thermal3d_32x48x8", "thermal3d_48x64x8", "thermal3d_32x64x6"):
        c = learned_case(name)
        with pytest.raises(jfnk.JfnkError) as e:
            jfnk.Solver(c)
        assert e.value.code == jfnk.JFNK_ERR_UNSUPPORTED, name
