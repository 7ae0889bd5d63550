"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This module only builds *inputs*: named parameter sets and initial fields
(numpy float64 arrays).  It holds none of the method's arithmetic (no
derivative, residual, Krylov or preconditioner code), so that the CUDA path
and the oracle stay independent while consuming identical inputs.

Layout of every state array: field-major planes, x fastest,
``[field][z][x]`` in 2D (fields u, w, theta, p) and ``[field][z][y][x]`` in
3D (fields u, v, w, theta, p).

Workloads are shaped on the paper's experiments:
* the dry thermal of Section 3.1 (domain [-10,10] x [0,10] km, warm bubble of
  radius 2 km centred at z = 2 km, theta_0 = 300 K, Table 1 exchange
  coefficients), neutral (beta = 0) or stably stratified (N = 0.01 1/s);
* the urban heat island of Section 3.2 (100 km x 2 km, surface heat flux
  H0 tanh profile over an urban patch, no-slip ground).
The bubble is cos^2 of the normalised radius, the noise Gaussian (seeded PCG64).
"""
from __future__ import annotations

import copy
import math

import numpy as np

# Physical constants of Section 2.1 (R, c_p, c_v, p_0) and gravity.
R_GAS = 287.0
CP = 1004.0
CV = 717.0
P0 = 1.0e5
GRAV = 9.81

SEED = 20200721

FREESLIP = 0
NOSLIP = 1

SGS_CONST = 0
SGS_SMAGORINSKY = 1
SGS_DEARDORFF = 2      # anisotropic closure of Section 2.4 (Eq. KmM)

PREC_FP64 = 0
PREC_MIXED = 1

PC_NONE = 0
PC_BLOCK = 1
PC_UNET = 2           # field block plus the learned correction
PC_SCHUR = 3
PC_NONLINEAR = 4      # nonlinear preconditioning (field block on the left)


def _base_case(dim, nx, nz, lx, lz, ny=1, ly=1.0):
    # Two Chebyshev sweeps per field block: at the eddy coefficients of these
    # workloads each block's Gershgorin interval [2/dt, 2/dt + 2.25 K_max sum 1/h^2]
    # has a condition number close to 1, where two sweeps already bound the
    # error of the block inverse by ~5e-4; three or four sweeps give the same
    # Krylov counts at a higher cost per apply.
    theta0 = 300.0
    return {
        "grid": {"dim": dim, "nx": nx, "ny": ny, "nz": nz,
                 "lx": lx, "ly": ly, "lz": lz,
                 "bc_bottom": FREESLIP, "bc_top": FREESLIP},
        "strat": {"theta0": theta0, "beta": 0.0, "pbar": CP, "g": GRAV,
                  "gamma_p": R_GAS / CV, "rho0": P0 / (R_GAS * theta0), "cp": CP},
        "sgs": {"mode": SGS_CONST, "K_M": 10.0, "K_H": 14.1, "Cs": 0.18, "Pr": 0.71},
        "opts": {"precision": PREC_FP64, "wavelet_p": 2, "krylov_m": 30,
                 "flexible": 1, "precond": PC_BLOCK, "pc_sweeps": 2,
                 "newton_rtol": 1e-8, "newton_atol_factor": 1e-13, "eta": 1e-4,
                 "max_newton": 20, "max_restarts": 20, "dt": 1.0,
                 "scale_u": 10.0, "scale_theta": 1.0, "scale_p": 0.01},
    }


def brunt_beta(n_bv, theta0=300.0, g=GRAV):
    """beta = d(theta_bar)/dz for a given Brunt-Vaisala frequency N (N^2 = g beta / theta0)."""
    return n_bv * n_bv * theta0 / g


def case(name: str) -> dict:
    """Named workloads (parameters only; fields come from ``initial_state``).

    thermal_neutral_128x64   2D neutral dry thermal, 128x64, constant K_M=10, K_H=14.1, FP64,
                             GMRES(30), Newton rtol 1e-8, dt = 1 s (Case A, Table 1 row 1).
    thermal_stable_1024x512  2D dry thermal, N = 0.01 1/s, 1024x512, Smagorinsky Cs = 0.18,
                             Pr = 0.71, bubble + 0.01 K white noise, FP32 stencils/basis with
                             FP64 Newton residual, FD difference, Givens and update.
    uhi_<nx>x<nz>            2D urban heat island, 100 km x 2 km, no-slip ground, beta = 3 K/km.
    thermal3d_<nx>x<ny>x<nz> 3D dry thermal, 20 x 20 x 10 km, N = 0.01 1/s, Smagorinsky, bubble +
                             noise, mixed precision, FGMRES(20).
    uhi3d_<nx>x<ny>x<nz>     3D heat island, 100 x 100 x 2 km, square 20 x 20 km urban patch.
    tiny_<nx>x<nz>           small variant of the thermal for unit tests (tiny3d_<nx>x<ny>x<nz> in 3D).
    """
    if name == "thermal_neutral_128x64":
        c = _base_case(2, 128, 64, 20000.0, 10000.0)
        c["init"] = {"kind": "bubble", "dtheta": 2.0, "radius": 2000.0, "zc": 2000.0,
                     "noise": 0.0}
        return c
    if name == "thermal_stable_1024x512":
        c = _base_case(2, 1024, 512, 20000.0, 10000.0)
        c["strat"]["beta"] = brunt_beta(0.01)
        c["sgs"].update(mode=SGS_SMAGORINSKY, Cs=0.18, Pr=0.71)
        c["opts"]["precision"] = PREC_MIXED
        c["init"] = {"kind": "bubble", "dtheta": 2.0, "radius": 2000.0, "zc": 2000.0,
                     "noise": 0.01}
        return c
    if name.startswith("thermal_stable_"):
        nx, nz = (int(v) for v in name[len("thermal_stable_"):].split("x"))
        c = case("thermal_stable_1024x512")
        c["grid"].update(nx=nx, nz=nz)
        return c
    if name.startswith("tiny_"):
        nx, nz = (int(v) for v in name[len("tiny_"):].split("x"))
        c = _base_case(2, nx, nz, 20000.0 * nx / 128.0, 10000.0 * nz / 64.0)
        c["init"] = {"kind": "bubble", "dtheta": 2.0, "radius": 2000.0, "zc": 2000.0,
                     "noise": 0.0}
        return c
    if name.startswith("thermal3d_"):
        nx, ny, nz = (int(v) for v in name[len("thermal3d_"):].split("x"))
        c = _base_case(3, nx, nz, 20000.0, 10000.0, ny=ny, ly=20000.0)
        c["strat"]["beta"] = brunt_beta(0.01)
        c["sgs"].update(mode=SGS_SMAGORINSKY, Cs=0.18, Pr=0.71)
        c["opts"]["precision"] = PREC_MIXED
        c["opts"]["krylov_m"] = 20
        c["init"] = {"kind": "bubble", "dtheta": 2.0, "radius": 2000.0, "zc": 2000.0,
                     "noise": 0.01}
        return c
    if name.startswith("tiny3d_"):
        nx, ny, nz = (int(v) for v in name[len("tiny3d_"):].split("x"))
        c = _base_case(3, nx, nz, 20000.0 * nx / 128.0, 10000.0 * nz / 64.0, ny=ny,
                       ly=20000.0 * ny / 128.0)
        c["init"] = {"kind": "bubble", "dtheta": 2.0, "radius": 2000.0, "zc": 2000.0,
                     "noise": 0.0}
        return c
    if name.startswith("uhi3d_"):
        nx, ny, nz = (int(v) for v in name[len("uhi3d_"):].split("x"))
        c = _base_case(3, nx, nz, 100000.0, 2000.0, ny=ny, ly=100000.0)
        c["grid"]["bc_bottom"] = NOSLIP
        c["strat"]["beta"] = 3.0e-3
        c["sgs"].update(mode=SGS_SMAGORINSKY, Cs=0.18, Pr=0.71)
        c["opts"]["precision"] = PREC_MIXED
        c["opts"]["krylov_m"] = 20
        c["init"] = {"kind": "rest", "H0": 100.0, "patch_halfwidth": 10000.0,
                     "xi": 0.1, "l": 1.5}
        return c
    if name.startswith("uhi_"):
        nx, nz = (int(v) for v in name[len("uhi_"):].split("x"))
        c = _base_case(2, nx, nz, 100000.0, 2000.0)
        c["grid"]["bc_bottom"] = NOSLIP
        c["strat"]["beta"] = 3.0e-3
        c["sgs"].update(mode=SGS_SMAGORINSKY, Cs=0.18, Pr=0.71)
        c["opts"]["precision"] = PREC_MIXED
        c["init"] = {"kind": "rest", "H0": 100.0, "patch_halfwidth": 10000.0,
                     "xi": 0.1, "l": 1.5}
        return c
    raise KeyError(name)


def uhi_batch(n: int = 16, nx0: int = 512, nz0: int = 128) -> list:
    """Batched urban heat island: instance i has nx = nx0 (1 + i mod 4), nz = nz0 (1 + i // 8)
    and H0 = 25 (930/25)^(i/(n-1)) W/m^2 (log-spaced), 100 km x 2 km, 20 km-wide urban patch."""
    out = []
    for i in range(n):
        nx = nx0 * (1 + i % 4)
        nz = nz0 * (1 + i // 8)
        c = case("uhi_%dx%d" % (nx, nz))
        c["init"]["H0"] = 25.0 * (930.0 / 25.0) ** (i / max(n - 1, 1))
        out.append(c)
    return out


def uhi3d_batch(n: int = 4, nx: int = 384, ny: int = 384, nz: int = 128, H0=(25.0, 100.0, 400.0, 930.0)) -> list:
    """Batched 3-D urban heat island: n instances of nx x ny x nz on 100 x 100 x 2 km with a
    20 x 20 km urban patch, surface heat flux H0[i] W/m^2, rest initial state."""
    out = []
    for i in range(n):
        c = case("uhi3d_%dx%dx%d" % (nx, ny, nz))
        c["init"]["H0"] = float(H0[i % len(H0)])
        out.append(c)
    return out


def with_options(c: dict, **kw) -> dict:
    """Deep copy of a case with some entries replaced (keys searched in every section)."""
    c = copy.deepcopy(c)
    for k, v in kw.items():
        for sec in ("grid", "strat", "sgs", "opts", "init"):
            if sec in c and k in c[sec]:
                c[sec][k] = v
                break
        else:
            raise KeyError(k)
    return c


def n_fields(c: dict) -> int:
    return 4 if c["grid"]["dim"] == 2 else 5


def shape(c: dict) -> tuple:
    g = c["grid"]
    if g["dim"] == 2:
        return (n_fields(c), g["nz"], g["nx"])
    return (n_fields(c), g["nz"], g["ny"], g["nx"])


def coords(c: dict):
    """Collocation nodes: x (and y) periodic, x_i = -L/2 + i dx; z cell-centred, z_k = (k+1/2) dz."""
    g = c["grid"]
    x = -0.5 * g["lx"] + np.arange(g["nx"]) * (g["lx"] / g["nx"])
    z = (np.arange(g["nz"]) + 0.5) * (g["lz"] / g["nz"])
    if g["dim"] == 2:
        return x, z
    y = -0.5 * g["ly"] + np.arange(g["ny"]) * (g["ly"] / g["ny"])
    return x, y, z


def _theta_index(c):
    return 2 if c["grid"]["dim"] == 2 else 3


def initial_state(c: dict, seed: int = SEED) -> np.ndarray:
    """Initial fields: rest wind, p' = 0, theta' = cos^2 bubble (+ seeded white noise)."""
    u = np.zeros(shape(c))
    ini = c.get("init", {"kind": "rest"})
    if ini["kind"] == "bubble":
        if c["grid"]["dim"] == 2:
            x, z = coords(c)
            X, Z = np.meshgrid(x, z, indexing="xy")
            L = np.sqrt((X / ini["radius"]) ** 2 + ((Z - ini["zc"]) / ini["radius"]) ** 2)
        else:
            x, y, z = coords(c)
            Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
            L = np.sqrt((X / ini["radius"]) ** 2 + (Y / ini["radius"]) ** 2
                        + ((Z - ini["zc"]) / ini["radius"]) ** 2)
        th = np.where(L <= 1.0, ini["dtheta"] * np.cos(0.5 * math.pi * L) ** 2, 0.0)
        if ini.get("noise", 0.0) > 0.0:
            rng = np.random.Generator(np.random.PCG64(seed))
            th = th + ini["noise"] * rng.standard_normal(th.shape)
        u[_theta_index(c)] = th
    return u


def random_state(c: dict, seed: int, amp=(1.0, 0.5, 0.005)) -> np.ndarray:
    """Bubble plus seeded random perturbations of every field (parity-test input).

    ``amp`` gives the standard deviations for (velocity, theta, p); velocity
    components share the first entry.
    """
    u = initial_state(with_options(c, noise=0.0) if c.get("init", {}).get("kind") == "bubble" else c)
    rng = np.random.Generator(np.random.PCG64(seed))
    nf = n_fields(c)
    for f in range(nf):
        a = amp[0] if f < nf - 2 else (amp[1] if f == nf - 2 else amp[2])
        u[f] = u[f] + a * rng.standard_normal(u[f].shape)
    return u


def random_vector(c: dict, seed: int) -> np.ndarray:
    """Seeded Gaussian direction vector (unit-free), same shape as the state."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape(c))


def heat_flux(c: dict) -> np.ndarray:
    """Surface heat-flux anomaly H(x) [W/m^2] of the heat-island experiment (Section 3.2).

    H = (H0/2) [tanh((xh+1)/xi) - tanh((xh-1)/xi)] for |xh| <= l, else 0, with
    xh = x / patch_halfwidth (reading of the printed profile: the half factor
    makes H0 the plateau value; xi and l are not given in the paper).
    Returns shape (nx,) in 2D and (ny, nx) in 3D.
    """
    ini = c["init"]
    g = c["grid"]
    if g["dim"] == 2:
        x, _ = coords(c)
        xh = x / ini["patch_halfwidth"]
        inside = np.abs(xh) <= ini["l"]
    else:
        x, y, _ = coords(c)
        Y, X = np.meshgrid(y, x, indexing="ij")
        xh = np.maximum(np.abs(X), np.abs(Y)) / ini["patch_halfwidth"]
        inside = np.abs(xh) <= ini["l"]
    H = 0.5 * ini["H0"] * (np.tanh((xh + 1.0) / ini["xi"]) - np.tanh((xh - 1.0) / ini["xi"]))
    return np.where(inside, H, 0.0)
