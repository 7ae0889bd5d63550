"""Learned right preconditioner: float64 reference of the 3-level linear U-Net.

TEST INFRASTRUCTURE (oracle only).  The learned preconditioner is not in the
paper (its Section 2.5.2 preconditioner is the physics-based field-block
one); this module fixes what the CUDA network computes so that its forward
pass, its gradients and its training pairs can be checked:

* network (no biases, no activations, zero padding, rows = z, columns = x):
    x (4 field planes; the GPU pads them to 16 channels with zeros)
    L0a 3x3 16->16, L0b 3x3 16->16 = s0, 2x2 average pool
    L1a 3x3 16->32, L1b 3x3 32->32 = s1, 2x2 average pool
    L2a 3x3 32->64, L2b 3x3 64->64, nearest upsampling x2, concat [up, s1] (96)
    L1c 3x3 96->32, nearest upsampling x2, concat [up, s0] (48)
    L0c 3x3 48->16, L0d 1x1 16->16; the first 4 output channels are N(x)
* weights: one flat vector, layers in the order above, each layer stored as
  [tap][cout][cin] with tap = ky * k + kx reading the input at offset
  (ky - k // 2, kx - k // 2);
* field balance: the convolutions act in balanced units, N(x) = B^-1 net(B x)
  with B = diag(1, 1, s_theta / Theta_b, s_p / P_b), s_* the scales of W and
  Theta_b = s_u sqrt(|beta| theta0 / g), P_b = s_u sqrt(gamma_p pbar / theta0):
  the units in which the buoyancy pair (g theta / theta0 in the w equation,
  -beta w in the theta equation) and the acoustic pair (-theta0 grad p, and
  -gamma_p pbar div u, Eqs. ch2_28-ch2_30) have equal coefficients both ways;
* loss of a pair (x, t): L = 1/2 ||B (N(x) - t)||^2 / ||B x||^2, and its
  gradient with respect to the flat weight vector (plain chain rule);
* training pairs (Section 2.5.1, Eq. jv), both giving an input X and the
  correction T that P = M^{-1} + N should add to the field-block
  preconditioner M^{-1} of Section 2.5.2 (frozen at u_k):
  - Arnoldi step: z_j = M^{-1} v_j and w = J_hat z_j, so J_hat^{-1} w = z_j
    exactly: X = w / ||w||, T = (z_j - M^{-1} w) / ||w||;
  - Newton correction: b = -W R(u_k), beta = ||b||, x_hat the scaled
    correction GMRES returned: X = b / beta, T = x_hat / beta - M^{-1} X;
* the preconditioner itself: P v = M^{-1} v + N(v).
* 3-D grids (5 fields u, v, w, theta, p on [z][y][x]): the same graph with
  every 3x3 convolution applied to each horizontal (y, x) plane (zero padding
  at the plane's edges), 2x2x2 average pooling and 2x2x2 nearest upsampling,
  so that the vertical coupling enters through the coarser levels; the
  balance is B = diag(1, 1, 1, s_theta / Theta_b, s_p / P_b).

Everything is whole-array numpy in float64 following these definitions, with
no blocking or fusion.  Pins (tests/test_oracle_unet.py): single layers
against scipy.signal.correlate2d, an identity network (with and without a
balance), a 4x4 block-mean network, the adjoint identities of pooling and
upsampling, the gradient against exact central differences, the balance
making the linearised acoustic and buoyancy couplings symmetric, and the
training-pair identities on a linear system solved exactly; for 3-D grids,
the per-plane convolution against scipy's 3-D correlation with a kernel one
plane deep, the identity network, the 4x4x4 block mean of the coarse path,
planes that stay uncoupled without the coarse levels, the 3-D adjoints, the
gradient with a five-field balance, and the five-field balance making the
couplings skew.
"""
from __future__ import annotations

import numpy as np

# (name, cin, cout, kernel size)
LAYERS = (
    ("L0a", 16, 16, 3), ("L0b", 16, 16, 3),
    ("L1a", 16, 32, 3), ("L1b", 32, 32, 3),
    ("L2a", 32, 64, 3), ("L2b", 64, 64, 3),
    ("L1c", 96, 32, 3), ("L0c", 48, 16, 3), ("L0d", 16, 16, 1),
)
NFIELDS = 4           # 2-D fields (u, w, theta, p); 3-D adds v
IN_CH = 16


def nfields(X: np.ndarray) -> int:
    """Field count of a state of shape (nf, nz, nx) (2-D) or (nf, nz, ny, nx) (3-D)."""
    return 4 if X.ndim == 3 else 5


def layer_sizes():
    return [k * k * co * ci for (_, ci, co, k) in LAYERS]


def num_weights() -> int:
    return int(sum(layer_sizes()))


def split_weights(flat: np.ndarray) -> dict:
    """Flat vector -> {name: array [k*k, cout, cin]}."""
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == num_weights()
    out, o = {}, 0
    for (name, ci, co, k), sz in zip(LAYERS, layer_sizes()):
        out[name] = flat[o:o + sz].reshape(k * k, co, ci)
        o += sz
    return out


def join_weights(ws: dict) -> np.ndarray:
    return np.concatenate([ws[name].reshape(-1) for (name, _, _, _) in LAYERS])


# ------------------------------------------------------------------ layers
def conv(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """out[co, y, x] = sum_tap sum_ci w[tap, co, ci] x[ci, y + dy, x + dx], zero outside."""
    kk, co, ci = w.shape
    k = int(round(np.sqrt(kk)))
    hp = k // 2
    C, H, W = x.shape
    assert C == ci
    xp = np.zeros((C, H + 2 * hp, W + 2 * hp))
    xp[:, hp:hp + H, hp:hp + W] = x
    out = np.zeros((co, H, W))
    for tap in range(kk):
        ky, kx = divmod(tap, k)
        shifted = xp[:, ky:ky + H, kx:kx + W]          # x[ci, y + ky - hp, x + kx - hp]
        out += np.einsum("oc,chw->ohw", w[tap], shifted)
    return out


def conv_grads(x: np.ndarray, w: np.ndarray, dout: np.ndarray):
    """Gradients of <dout, conv(x, w)> w.r.t. x (scatter form) and w."""
    kk, co, ci = w.shape
    k = int(round(np.sqrt(kk)))
    hp = k // 2
    C, H, W = x.shape
    xp = np.zeros((C, H + 2 * hp, W + 2 * hp))
    xp[:, hp:hp + H, hp:hp + W] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for tap in range(kk):
        ky, kx = divmod(tap, k)
        shifted = xp[:, ky:ky + H, kx:kx + W]
        dw[tap] = np.einsum("ohw,chw->oc", dout, shifted)
        dxp[:, ky:ky + H, kx:kx + W] += np.einsum("oc,ohw->chw", w[tap], dout)
    return dxp[:, hp:hp + H, hp:hp + W], dw


def conv_planes(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """conv() on every horizontal plane of x (C, nz, ny, nx) (3-D), or conv() itself (2-D)."""
    if x.ndim == 3:
        return conv(x, w)
    return np.stack([conv(x[:, z], w) for z in range(x.shape[1])], axis=1)


def conv_grads_planes(x: np.ndarray, w: np.ndarray, dout: np.ndarray):
    if x.ndim == 3:
        return conv_grads(x, w, dout)
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for z in range(x.shape[1]):
        dxz, dwz = conv_grads(x[:, z], w, dout[:, z])
        dx[:, z] = dxz
        dw += dwz
    return dx, dw


def pool2(x: np.ndarray) -> np.ndarray:
    """2x2 average (2-D) or 2x2x2 average (3-D)."""
    if x.ndim == 3:
        C, H, W = x.shape
        return x.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))
    C, D, H, W = x.shape
    return x.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def up2(x: np.ndarray) -> np.ndarray:
    """Nearest-neighbour upsampling x2 along every spatial axis."""
    for ax in range(1, x.ndim):
        x = np.repeat(x, 2, axis=ax)
    return x


def pool2_adjoint(d: np.ndarray) -> np.ndarray:
    return up2(d) / 2.0 ** (d.ndim - 1)


def up2_adjoint(d: np.ndarray) -> np.ndarray:
    if d.ndim == 3:
        C, H, W = d.shape
        return d.reshape(C, H // 2, 2, W // 2, 2).sum(axis=(2, 4))
    C, D, H, W = d.shape
    return d.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))


def balance(case: dict) -> np.ndarray:
    """Per-field factors B (velocity components, theta, p) of a 2-D or 3-D case."""
    st, op = case["strat"], case["opts"]
    su = op["scale_u"]
    nf = 4 if case["grid"]["dim"] == 2 else 5
    b = np.ones(nf)
    if st["beta"] != 0.0 and st["g"] > 0.0:
        b[nf - 2] = op["scale_theta"] / (su * np.sqrt(abs(st["beta"]) * st["theta0"] / st["g"]))
    if st["gamma_p"] * st["pbar"] > 0.0:
        b[nf - 1] = op["scale_p"] / (su * np.sqrt(st["gamma_p"] * st["pbar"] / st["theta0"]))
    return b


def _b(B, nf, ndim):
    B = np.ones(nf) if B is None else np.asarray(B, dtype=np.float64)
    return B.reshape((nf,) + (1,) * (ndim - 1))


# ----------------------------------------------------------------- network
def forward(flat: np.ndarray, X: np.ndarray, B=None):
    """N(X) for X of shape (4, nz, nx) (2-D) or (5, nz, ny, nx) (3-D); returns (y, activations).

    The activations hold the raw network run on B X (balanced units); y is
    B^-1 times its first nf output channels.
    """
    w = split_weights(flat)
    nf = nfields(X)
    assert all(n % 4 == 0 for n in X.shape[1:])
    a = {}
    a["x0"] = np.zeros((IN_CH,) + X.shape[1:])
    a["x0"][:nf] = _b(B, nf, X.ndim) * X
    a["h0a"] = conv_planes(a["x0"], w["L0a"])
    a["s0"] = conv_planes(a["h0a"], w["L0b"])
    a["p1"] = pool2(a["s0"])
    a["h1a"] = conv_planes(a["p1"], w["L1a"])
    a["s1"] = conv_planes(a["h1a"], w["L1b"])
    a["p2"] = pool2(a["s1"])
    a["h2a"] = conv_planes(a["p2"], w["L2a"])
    a["h2b"] = conv_planes(a["h2a"], w["L2b"])
    a["cat1"] = np.concatenate([up2(a["h2b"]), a["s1"]])
    a["h1c"] = conv_planes(a["cat1"], w["L1c"])
    a["cat0"] = np.concatenate([up2(a["h1c"]), a["s0"]])
    a["h0c"] = conv_planes(a["cat0"], w["L0c"])
    a["out"] = conv_planes(a["h0c"], w["L0d"])
    return a["out"][:nf] / _b(B, nf, X.ndim), a


def backward(flat: np.ndarray, a: dict, dy: np.ndarray) -> np.ndarray:
    """Flat gradient of <dy, raw output channels 0..nf-1> given the activations of forward()."""
    w = split_weights(flat)
    g = {}
    dout = np.zeros_like(a["out"])
    dout[:dy.shape[0]] = dy
    d_h0c, g["L0d"] = conv_grads_planes(a["h0c"], w["L0d"], dout)
    d_cat0, g["L0c"] = conv_grads_planes(a["cat0"], w["L0c"], d_h0c)
    d_h1c = up2_adjoint(d_cat0[:32])
    d_s0 = d_cat0[32:].copy()
    d_cat1, g["L1c"] = conv_grads_planes(a["cat1"], w["L1c"], d_h1c)
    d_h2b = up2_adjoint(d_cat1[:64])
    d_s1 = d_cat1[64:].copy()
    d_h2a, g["L2b"] = conv_grads_planes(a["h2a"], w["L2b"], d_h2b)
    d_p2, g["L2a"] = conv_grads_planes(a["p2"], w["L2a"], d_h2a)
    d_s1 += pool2_adjoint(d_p2)
    d_h1a, g["L1b"] = conv_grads_planes(a["h1a"], w["L1b"], d_s1)
    d_p1, g["L1a"] = conv_grads_planes(a["p1"], w["L1a"], d_h1a)
    d_s0 += pool2_adjoint(d_p1)
    d_h0a, g["L0b"] = conv_grads_planes(a["h0a"], w["L0b"], d_s0)
    _, g["L0a"] = conv_grads_planes(a["x0"], w["L0a"], d_h0a)
    return join_weights(g)


def apply(flat: np.ndarray, X: np.ndarray, B=None) -> np.ndarray:
    return forward(flat, X, B)[0]


def loss(flat: np.ndarray, X: np.ndarray, T: np.ndarray, B=None) -> float:
    b = _b(B, nfields(X), X.ndim)
    d = b * (apply(flat, X, B) - T)
    return 0.5 * float(np.sum(d * d)) / float(np.sum((b * X) ** 2))


def loss_grad(flat: np.ndarray, X: np.ndarray, T: np.ndarray, B=None):
    """(L, dL/dw) for L = 1/2 ||B (N(X) - T)||^2 / ||B X||^2."""
    b = _b(B, nfields(X), X.ndim)
    y, a = forward(flat, X, B)
    xn2 = float(np.sum((b * X) ** 2))
    r = b * (y - T)                      # raw output minus B T
    return 0.5 * float(np.sum(r * r)) / xn2, backward(flat, a, r / xn2)


# ------------------------------------------------------ preconditioner use
def newton_pair(model, U: np.ndarray, R: np.ndarray, xhat: np.ndarray, sweeps: int):
    """(X, T) of one Newton correction: X = -W R / beta, T = xhat / beta - M^{-1} X."""
    b = -model.scale(R)
    beta = float(np.sqrt(np.sum(b * b)))
    X = b / beta
    T = xhat / beta - model.precond(U, X, sweeps)
    return X, T


def arnoldi_pair(model, U: np.ndarray, z: np.ndarray, w: np.ndarray, sweeps: int):
    """(X, T) of one Arnoldi step with w = J_hat z: X = w / ||w||, T = (z - M^{-1} w) / ||w||."""
    nw = float(np.sqrt(np.sum(w * w)))
    return w / nw, (z - model.precond(U, w, sweeps)) / nw


def precond(model, flat: np.ndarray, U: np.ndarray, V: np.ndarray, sweeps: int, B=None) -> np.ndarray:
    """P v = M^{-1} v + N(v) (scaled units)."""
    return model.precond(U, V, sweeps) + apply(flat, V, B)
