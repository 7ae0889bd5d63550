"""Pins of the float64 U-Net oracle (learned right preconditioner).

Each check ties the oracle to something outside itself: scipy's 2-D and
3-D correlation, closed-form outputs of hand-set networks, the adjoint identities
of the resampling operators, and exact central differences (the loss is
quadratic in every single weight, so a central difference reproduces the
partial derivative up to rounding).
"""
import numpy as np
import pytest

scipy_signal = pytest.importorskip("scipy.signal")

from oracle import unet as U  # noqa: E402


def _rng(seed=7):
    return np.random.default_rng(seed)


def _random_weights(rng, scale=1.0):
    parts = []
    for (_, ci, co, k) in U.LAYERS:
        parts.append(rng.standard_normal(k * k * co * ci) * scale / np.sqrt(k * k * ci))
    return np.concatenate(parts)


@pytest.mark.parametrize("k,ci,co", [(3, 5, 4), (1, 3, 2)])
def test_conv_matches_scipy_correlate(k, ci, co):
    rng = _rng(1)
    x = rng.standard_normal((ci, 9, 11))
    w = rng.standard_normal((k * k, co, ci))
    out = U.conv(x, w)
    ref = np.zeros((co, 9, 11))
    for o in range(co):
        for c in range(ci):
            K = w[:, o, c].reshape(k, k)
            ref[o] += scipy_signal.correlate2d(x[c], K, mode="same", boundary="fill", fillvalue=0.0)
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-13)


def _eye_tap(k, co, ci, shift_in=0):
    w = np.zeros((k * k, co, ci))
    c = (k * k) // 2
    for i in range(min(co, ci - shift_in)):
        w[c, i, i + shift_in] = 1.0
    return w


def test_identity_network_is_identity():
    rng = _rng(2)
    ws = {name: rng.standard_normal((k * k, co, ci)) for (name, ci, co, k) in U.LAYERS}
    ws["L0a"] = _eye_tap(3, 16, 16)
    ws["L0b"] = _eye_tap(3, 16, 16)
    ws["L1c"] = np.zeros_like(ws["L1c"])          # coarse path off
    ws["L0c"] = _eye_tap(3, 16, 48, shift_in=32)  # read s0 only
    ws["L0d"] = _eye_tap(1, 16, 16)
    X = rng.standard_normal((4, 16, 24))
    y = U.apply(U.join_weights(ws), X)
    np.testing.assert_allclose(y, X, rtol=0, atol=1e-14)


def test_coarse_path_is_4x4_block_mean():
    rng = _rng(3)
    ws = {name: np.zeros((k * k, co, ci)) for (name, ci, co, k) in U.LAYERS}
    for name in ("L0a", "L0b", "L1a", "L1b", "L2a", "L2b", "L1c", "L0c"):
        _, ci, co, k = next(l for l in U.LAYERS if l[0] == name)
        ws[name] = _eye_tap(k, co, ci)               # first channels straight through
    ws["L0d"] = _eye_tap(1, 16, 16)
    X = rng.standard_normal((4, 8, 12))
    y = U.apply(U.join_weights(ws), X)
    ref = X.reshape(4, 2, 4, 3, 4).mean(axis=(2, 4))
    ref = np.repeat(np.repeat(ref, 4, axis=1), 4, axis=2)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-14)


def test_resampling_adjoints():
    rng = _rng(4)
    a = rng.standard_normal((3, 8, 6))
    b = rng.standard_normal((3, 4, 3))
    assert abs(np.sum(U.pool2(a) * b) - np.sum(a * U.pool2_adjoint(b))) < 1e-13
    assert abs(np.sum(U.up2(b) * a) - np.sum(b * U.up2_adjoint(a))) < 1e-13
    # pool(up(b)) = b
    np.testing.assert_allclose(U.pool2(U.up2(b)), b, atol=1e-15)


def test_linearity():
    rng = _rng(5)
    w = _random_weights(rng)
    X1 = rng.standard_normal((4, 8, 8))
    X2 = rng.standard_normal((4, 8, 8))
    lhs = U.apply(w, 2.0 * X1 - 3.0 * X2)
    rhs = 2.0 * U.apply(w, X1) - 3.0 * U.apply(w, X2)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_gradient_matches_central_differences():
    rng = _rng(6)
    w = _random_weights(rng)
    X = rng.standard_normal((4, 8, 8))
    T = rng.standard_normal((4, 8, 8))
    L, g = U.loss_grad(w, X, T)
    assert abs(L - U.loss(w, X, T)) < 1e-14 * max(1.0, abs(L))
    sizes = U.layer_sizes()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    for li in range(len(U.LAYERS)):
        for idx in rng.integers(offs[li], offs[li + 1], size=4):
            h = 1e-3
            wp = w.copy(); wp[idx] += h
            wm = w.copy(); wm[idx] -= h
            fd = (U.loss(wp, X, T) - U.loss(wm, X, T)) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-8 * (abs(g[idx]) + np.max(np.abs(g[offs[li]:offs[li + 1]]))), \
                (U.LAYERS[li][0], idx, fd, g[idx])


def test_gradient_zero_at_exact_fit():
    rng = _rng(8)
    w = _random_weights(rng)
    X = rng.standard_normal((4, 8, 8))
    T = U.apply(w, X)
    L, g = U.loss_grad(w, X, T)
    assert L < 1e-28
    assert np.max(np.abs(g)) < 1e-13


def test_identity_network_with_balance_is_identity():
    rng = _rng(9)
    ws = {name: np.zeros((k * k, co, ci)) for (name, ci, co, k) in U.LAYERS}
    ws["L0a"] = _eye_tap(3, 16, 16)
    ws["L0b"] = _eye_tap(3, 16, 16)
    ws["L0c"] = _eye_tap(3, 16, 48, shift_in=32)
    ws["L0d"] = _eye_tap(1, 16, 16)
    X = rng.standard_normal((4, 8, 12))
    B = np.array([1.0, 1.0, 0.3, 8e-4])
    np.testing.assert_allclose(U.apply(U.join_weights(ws), X, B), X, rtol=1e-14, atol=1e-14)
    # the raw network sees B X: a network that only scales by 2 returns 2 X
    ws["L0d"] = 2.0 * ws["L0d"]
    np.testing.assert_allclose(U.apply(U.join_weights(ws), X, B), 2.0 * X, rtol=1e-14, atol=1e-14)


def test_gradient_with_balance_matches_central_differences():
    rng = _rng(10)
    w = _random_weights(rng)
    B = np.array([1.0, 1.0, 0.3, 8e-4])
    X = rng.standard_normal((4, 8, 8))
    T = rng.standard_normal((4, 8, 8))
    L, g = U.loss_grad(w, X, T, B)
    assert abs(L - U.loss(w, X, T, B)) < 1e-14 * max(1.0, L)
    for idx in rng.integers(0, w.size, size=12):
        h = 1e-3
        wp = w.copy(); wp[idx] += h
        wm = w.copy(); wm[idx] -= h
        fd = (U.loss(wp, X, T, B) - U.loss(wm, X, T, B)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-8 * (abs(g[idx]) + np.max(np.abs(g))), (idx, fd, g[idx])


def _linear_rest_model():
    """Stable thermal at rest with no eddy diffusion: F is linear plus quadratic convection."""
    from oracle.operators import Model
    from paper_2007_10411_gb300 import synth
    c = synth.case("thermal_stable_64x32")
    c["sgs"] = {"mode": synth.SGS_CONST, "K_M": 0.0, "K_H": 0.0, "Cs": 0.0, "Pr": 1.0}
    return c, Model(c)


def test_balance_makes_acoustic_and_buoyancy_coupling_skew():
    """In balanced units the field coupling of the linearised F at rest is skew-adjoint.

    J_F e is the central difference of F at u = 0 (exact: F is linear plus a
    quadratic convection there).  For a velocity-only vector a and a
    (theta, p)-only vector c, <c, J a> = -<a, J c> holds in the units B W u
    and fails by orders of magnitude in the units W u.
    """
    c, m = _linear_rest_model()
    shape = (4, 32, 64)
    rng = _rng(11)
    Z = np.zeros(shape)

    def JF(e):
        h = 1e-4
        return (m.F(Z + h * e) - m.F(Z - h * e)) / (2 * h)

    def J_units(D, x):      # D diag per field: variables y = D u
        Dr = D.reshape(4, 1, 1)
        return Dr * JF(x / Dr)

    a = rng.standard_normal(shape); a[2:] = 0.0
    cc = rng.standard_normal(shape); cc[:2] = 0.0
    W = 1.0 / m.scales
    for D, skew in ((U.balance(c) * W, True), (W, False)):
        lhs = float(np.sum(cc * J_units(D, a)))
        rhs = -float(np.sum(a * J_units(D, cc)))
        asym = abs(lhs - rhs) / max(abs(lhs), abs(rhs))
        if skew:
            assert asym < 1e-8, asym
        else:
            assert asym > 0.5, asym


def test_training_pairs_reproduce_the_correction():
    from oracle.krylov import gmres
    from paper_2007_10411_gb300 import synth
    from oracle.operators import Model
    c = synth.case("thermal_stable_64x32")
    m = Model(c)
    sw = c["opts"]["pc_sweeps"]
    Uk = synth.random_state(c, 5, amp=(0.5, 0.1, 0.002))
    FU = m.F(Uk)
    J = lambda v: m.jv_scaled(Uk, FU, v)
    rng = _rng(12)
    # Arnoldi pair: M^-1 X + T = z / ||w|| and J of it gives X back
    z = m.precond(Uk, rng.standard_normal(Uk.shape), sw)
    w = J(z)
    X, T = U.arnoldi_pair(m, Uk, z, w, sw)
    assert abs(np.linalg.norm(X) - 1.0) < 1e-14
    Y = m.precond(Uk, X, sw) + T
    np.testing.assert_allclose(Y, z / np.linalg.norm(w), rtol=0, atol=1e-12 * np.max(np.abs(z)) / np.linalg.norm(w))
    assert np.linalg.norm(J(Y) - X) < 1e-6
    # Newton pair from a tightly solved correction
    f = m.rhs_f(Uk - 0.01)
    R = m.residual(Uk, f)
    b = -m.scale(R)
    xhat = gmres(J, b, 30, 1e-10, 20, precond=lambda v: m.precond(Uk, v, sw), flexible=True)
    X, T = U.newton_pair(m, Uk, R, xhat, sw)
    # J_hat is a finite-difference product whose step depends on the vector,
    # so it is linear only to ~1e-6 here: a wrong sign or scale gives O(1)
    assert np.linalg.norm(J(m.precond(Uk, X, sw) + T) - X) < 1e-4


# ------------------------------------------------------------------- 3-D grids
def test_conv_planes_matches_scipy_3d_correlate():
    """Per-plane 3x3 convolution = scipy's 3-D correlation with a kernel one plane deep."""
    rng = _rng(21)
    ci, co = 3, 2
    x = rng.standard_normal((ci, 4, 7, 9))
    w = rng.standard_normal((9, co, ci))
    out = U.conv_planes(x, w)
    ref = np.zeros((co, 4, 7, 9))
    for o in range(co):
        for c in range(ci):
            K = w[:, o, c].reshape(1, 3, 3)
            ref[o] += scipy_signal.correlate(x[c], K, mode="same", method="direct")
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-13)


def test_identity_network_3d():
    rng = _rng(22)
    ws = {name: rng.standard_normal((k * k, co, ci)) for (name, ci, co, k) in U.LAYERS}
    ws["L0a"] = _eye_tap(3, 16, 16)
    ws["L0b"] = _eye_tap(3, 16, 16)
    ws["L1c"] = np.zeros_like(ws["L1c"])
    ws["L0c"] = _eye_tap(3, 16, 48, shift_in=32)
    ws["L0d"] = _eye_tap(1, 16, 16)
    X = rng.standard_normal((5, 4, 8, 12))
    B = np.array([1.0, 1.0, 1.0, 0.3, 8e-4])
    np.testing.assert_allclose(U.apply(U.join_weights(ws), X, B), X, rtol=1e-14, atol=1e-14)


def test_coarse_path_is_4x4x4_block_mean():
    rng = _rng(23)
    ws = {name: np.zeros((k * k, co, ci)) for (name, ci, co, k) in U.LAYERS}
    for (name, ci, co, k) in U.LAYERS:
        ws[name] = _eye_tap(k, co, ci)
    X = rng.standard_normal((5, 8, 4, 12))
    y = U.apply(U.join_weights(ws), X)
    ref = X.reshape(5, 2, 4, 1, 4, 3, 4).mean(axis=(2, 4, 6))
    for ax in (1, 2, 3):
        ref = np.repeat(ref, 4, axis=ax)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-14)


def test_planes_do_not_couple_without_the_coarse_levels():
    """With the coarse path off, a field in one z plane never leaves that plane."""
    rng = _rng(24)
    w = _random_weights(rng)
    ws = U.split_weights(w)
    ws["L1c"] = np.zeros_like(ws["L1c"])
    w = U.join_weights(ws)
    X = np.zeros((5, 4, 8, 8))
    X[:, 2] = rng.standard_normal((5, 8, 8))
    y = U.apply(w, X)
    assert np.max(np.abs(y[:, 2])) > 1e-3
    assert np.max(np.abs(y[:, [0, 1, 3]])) == 0.0
    # and with it on, the pooled levels carry the plane's content to its pool partner (z = 3)
    y2 = U.apply(_random_weights(rng), X)
    assert np.max(np.abs(y2[:, 3])) > 1e-3


def test_resampling_adjoints_3d():
    rng = _rng(25)
    a = rng.standard_normal((3, 4, 8, 6))
    b = rng.standard_normal((3, 2, 4, 3))
    assert abs(np.sum(U.pool2(a) * b) - np.sum(a * U.pool2_adjoint(b))) < 1e-13
    assert abs(np.sum(U.up2(b) * a) - np.sum(b * U.up2_adjoint(a))) < 1e-13
    np.testing.assert_allclose(U.pool2(U.up2(b)), b, atol=1e-15)
    # pool2 is the mean of the 8 children
    assert U.pool2(a)[1, 1, 2, 0] == pytest.approx(a[1, 2:4, 4:6, 0:2].mean(), rel=1e-14)


def test_gradient_3d_with_balance_matches_central_differences():
    rng = _rng(26)
    w = _random_weights(rng)
    B = np.array([1.0, 1.0, 1.0, 0.3, 8e-4])
    X = rng.standard_normal((5, 4, 8, 8))
    T = rng.standard_normal((5, 4, 8, 8))
    L, g = U.loss_grad(w, X, T, B)
    assert abs(L - U.loss(w, X, T, B)) < 1e-14 * max(1.0, L)
    sizes = U.layer_sizes()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    for li in range(len(U.LAYERS)):
        for idx in rng.integers(offs[li], offs[li + 1], size=3):
            h = 1e-3
            wp = w.copy(); wp[idx] += h
            wm = w.copy(); wm[idx] -= h
            fd = (U.loss(wp, X, T, B) - U.loss(wm, X, T, B)) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-8 * (abs(g[idx]) + np.max(np.abs(g[offs[li]:offs[li + 1]]))), \
                (U.LAYERS[li][0], idx, fd, g[idx])


def test_balance_3d_makes_the_couplings_skew():
    """3-D analogue of the 2-D check: five fields, B = (1, 1, 1, b_theta, b_p)."""
    from oracle.operators import Model
    from paper_2007_10411_gb300 import synth
    c = synth.case("thermal3d_8x8x8")
    c["sgs"] = {"mode": synth.SGS_CONST, "K_M": 0.0, "K_H": 0.0, "Cs": 0.0, "Pr": 1.0}
    m = Model(c)
    shape = synth.shape(c)
    assert shape[0] == 5
    Bal = U.balance(c)
    assert Bal.shape == (5,) and np.all(Bal[:3] == 1.0) and Bal[3] != 1.0 and Bal[4] != 1.0
    rng = _rng(27)
    Z = np.zeros(shape)

    def JF(e):
        h = 1e-4
        return (m.F(Z + h * e) - m.F(Z - h * e)) / (2 * h)

    a = rng.standard_normal(shape); a[3:] = 0.0
    cc = rng.standard_normal(shape); cc[:3] = 0.0
    W = 1.0 / m.scales
    for D, skew in ((Bal * W, True), (W, False)):
        Dr = D.reshape(5, 1, 1, 1)
        lhs = float(np.sum(cc * Dr * JF(a / Dr)))
        rhs = -float(np.sum(a * Dr * JF(cc / Dr)))
        asym = abs(lhs - rhs) / max(abs(lhs), abs(rhs))
        if skew:
            assert asym < 1e-8, asym
        else:
            assert asym > 0.5, asym
