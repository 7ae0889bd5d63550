"""Discrete operators of the paper, plain float64 numpy (TEST INFRASTRUCTURE: oracle only).

Fields (2D): u, w, theta, p on arrays [z][x];  (3D): u, v, w, theta, p on [z][y][x].

Equations followed (Section 2.1, Eqs. ch2_28-ch2_30), with the readings used
throughout this project:

  dp/dt     = -C(u)p - gamma_p (pbar + p) div(u)                     (Eq. ch2_28)
  du_i/dt   = -C(u)u_i - theta0 D_i p + sum_j D_j(K_M D_j u_i)
              + (g theta/theta0) delta_i3                              (Eq. ch2_29)
  dtheta/dt = -C(u)theta - beta w + sum_j D_j(K_H D_j theta) + S_H     (Eq. ch2_30)

* C(u)phi = 1/2 sum_j D_j(u_j phi) + 1/2 sum_j u_j D_j phi is the skew-symmetric
  mean of flux and advective forms (Section 2.2), applied to every field.
* D_j is the Deslauriers-Dubuc collocation derivative (Section 2.3).
* Constant exchange coefficients (Table 1) or Smagorinsky
  nu = (Cs Delta)^2 sqrt(2 S_ij S_ij), K_M = nu, K_H = nu/Pr (Section 2.4), or
  the anisotropic Deardorff closure of Section 2.4 (Eq. KmM): horizontal
  and vertical coefficients K_m, K_M for momentum and K_h, K_H for heat,
  each acting along its own directions (``deardorff``).
* The stress divergence is taken in per-component Laplacian form
  sum_j D_j(K D_j phi) (symmetric negative semi-definite); p is not diffused.
* S_H = H(x)/(rho0 cp dz) in the bottom row of theta (surface heat flux of
  Section 3.2), zero when no flux is given.
* Boundaries: x (and y) periodic; z cell-centred with mirror walls, ghost
  values f_{-1-k} = s f_k and f_{nz+k} = s f_{nz-1-k}, parity s = -1 for w,
  +1 for theta and p, +1 (free slip) or -1 (no slip) for u and v.  The eddy
  coefficient K is mirrored even.

Time discretisation (Eq. ns):  R(u) = 2u/dt - F(u) - f,  f = 2u^n/dt + F(u^n).
Jacobian-vector product (Eq. fd) by a forward difference of R.
"""
from __future__ import annotations

import math

import numpy as np

from .wavelet import derivative_weights

FREESLIP = 0
NOSLIP = 1
SGS_CONST = 0
SGS_SMAGORINSKY = 1
SGS_DEARDORFF = 2
EPS_FP64 = 2.0 ** -52


class Model:
    """Spatial operator F, residual R and Jacobian-vector product for one grid."""

    def __init__(self, case: dict):
        g, st, sg, op = case["grid"], case["strat"], case["sgs"], case["opts"]
        self.dim = g["dim"]
        self.nx, self.ny, self.nz = g["nx"], g.get("ny", 1), g["nz"]
        self.dx = g["lx"] / g["nx"]
        self.dz = g["lz"] / g["nz"]
        self.dy = g["ly"] / g["ny"] if self.dim == 3 else None
        self.lz = g["lz"]
        self.d = derivative_weights(op["wavelet_p"])
        self.r = max(abs(l) for l in self.d)
        self.H = 2 * self.r
        if self.nz < self.H:
            raise ValueError("nz must be at least twice the stencil radius")
        self.theta0 = st["theta0"]
        self.beta = st["beta"]
        self.pbar = st["pbar"]
        self.g = st["g"]
        self.gamma_p = st["gamma_p"]
        self.rho0 = st["rho0"]
        self.cp = st["cp"]
        self.sgs_mode = sg["mode"]
        self.K_M, self.K_H = sg["K_M"], sg["K_H"]
        self.Cs, self.Pr = sg["Cs"], sg["Pr"]
        self.dt = op["dt"]
        self.heat = None                      # surface flux H(x[,y]) in W/m^2
        # field bookkeeping
        s_b = 1.0 if g["bc_bottom"] == FREESLIP else -1.0
        s_t = 1.0 if g["bc_top"] == FREESLIP else -1.0
        if self.dim == 2:
            self.iu, self.iw, self.ith, self.ip = 0, 1, 2, 3
            self.vel = [0, 1]                 # velocity component along each direction
            self.axes = [1, 0]                # array axis of x, z
            self.spacing = [self.dx, self.dz]
            self.parity = [(s_b, s_t), (-1.0, -1.0), (1.0, 1.0), (1.0, 1.0)]
        else:
            self.iu, self.iv, self.iw, self.ith, self.ip = 0, 1, 2, 3, 4
            self.vel = [0, 1, 2]
            self.axes = [2, 1, 0]             # x, y, z
            self.spacing = [self.dx, self.dy, self.dz]
            self.parity = [(s_b, s_t), (s_b, s_t), (-1.0, -1.0), (1.0, 1.0), (1.0, 1.0)]
        self.nf = len(self.parity)
        self.scales = np.array([op["scale_u"]] * self.dim + [op["scale_theta"], op["scale_p"]])
        self.delta_les = (self.dx * self.dz) ** 0.5 if self.dim == 2 else \
            (self.dx * self.dy * self.dz) ** (1.0 / 3.0)
        # horizontal cell size of the Deardorff closure: Delta_y reads as Delta_x in 2-D
        self.dy_h = self.dx if self.dim == 2 else self.dy
        self.N2 = self.g * self.beta / self.theta0          # background Brunt-Vaisala frequency squared

    # ------------------------------------------------------------------ ghosts
    def extend(self, a: np.ndarray, halo: int, parity) -> np.ndarray:
        """Ghost extension by ``halo`` points: periodic horizontally, mirror (signed) in z."""
        b = np.pad(a, [(0, 0)] + [(halo, halo)] * (a.ndim - 1), mode="wrap")
        b = np.pad(b, [(halo, halo)] + [(0, 0)] * (a.ndim - 1), mode="symmetric")
        b[:halo] *= parity[0]
        b[b.shape[0] - halo:] *= parity[1]
        return b

    @staticmethod
    def crop(a: np.ndarray, c: int, skip_axis=None) -> np.ndarray:
        """Remove ``c`` points from both ends of every axis except ``skip_axis``."""
        if c == 0:
            return a
        sl = [slice(None) if ax == skip_axis else slice(c, a.shape[ax] - c) for ax in range(a.ndim)]
        return a[tuple(sl)]

    # -------------------------------------------------------------- derivative
    def deriv(self, a: np.ndarray, axis: int, h: float) -> np.ndarray:
        """(D a)_j = (1/h) sum_l d_l a_{j-l} along ``axis``; the axis shrinks by 2r."""
        r = self.r
        n = a.shape[axis] - 2 * r
        out = np.zeros(a.shape[:axis] + (n,) + a.shape[axis + 1:])
        for l, dl in self.d.items():
            sl = [slice(None)] * a.ndim
            sl[axis] = slice(r - l, r - l + n)
            out += dl * a[tuple(sl)]
        return out / h

    def grad_halo(self, a_pad: np.ndarray) -> list:
        """First derivatives of a field with halo 2r, on the halo-r region (one per direction)."""
        r = self.r
        return [self.crop(self.deriv(a_pad, ax, h), r, skip_axis=ax)
                for ax, h in zip(self.axes, self.spacing)]

    def div_halo(self, vecs_r: list) -> np.ndarray:
        """sum_j D_j q_j for fields q_j given on the halo-r region; result on the interior."""
        r = self.r
        out = 0.0
        for q, ax, h in zip(vecs_r, self.axes, self.spacing):
            out = out + self.crop(self.deriv(q, ax, h), r, skip_axis=ax)
        return out

    # ------------------------------------------------------------- convection
    def convection(self, vel_pad: list, phi_pad: np.ndarray, grad_phi_r: list) -> np.ndarray:
        """Skew-symmetric convection 1/2 D_j(u_j phi) + 1/2 u_j D_j phi on the interior (Section 2.2).

        ``vel_pad`` / ``phi_pad`` carry halo 2r, ``grad_phi_r`` is D_j phi on the halo-r region.
        """
        r = self.r
        fluxes = [self.crop(uj * phi_pad, r) for uj in vel_pad]       # u_j phi on halo r
        flux_form = self.div_halo(fluxes)
        adv_form = 0.0
        for uj, g in zip(vel_pad, grad_phi_r):
            adv_form = adv_form + self.crop(uj, 2 * r) * self.crop(g, r)
        return 0.5 * flux_form + 0.5 * adv_form

    # -------------------------------------------------------------- eddy coef
    def smagorinsky_nu(self, grads_vel_int: list) -> np.ndarray:
        """nu = (Cs Delta)^2 sqrt(2 S_ij S_ij) from velocity gradients at interior points (Section 2.4).

        ``grads_vel_int[i][j]`` = D_j u_i.
        """
        n = self.dim
        ss = 0.0
        for i in range(n):
            for j in range(n):
                s_ij = 0.5 * (grads_vel_int[i][j] + grads_vel_int[j][i])
                ss = ss + s_ij * s_ij
        return (self.Cs * self.delta_les) ** 2 * np.sqrt(2.0 * ss)

    def strain_magnitude(self, grads_vel_int: list) -> np.ndarray:
        """s = sqrt(2 S_ij S_ij) from velocity gradients at interior points."""
        n = self.dim
        ss = 0.0
        for i in range(n):
            for j in range(n):
                s_ij = 0.5 * (grads_vel_int[i][j] + grads_vel_int[j][i])
                ss = ss + s_ij * s_ij
        return np.sqrt(2.0 * ss)

    def deardorff(self, s: np.ndarray):
        """Anisotropic exchange coefficients of Section 2.4 from the strain magnitude s.

        nu_tau = (Delta Cs)^2 s, epsilon = nu_tau S_ij S_ij = nu_tau s^2 / 2,
        K_m = Cs^(4/3) epsilon^(1/3) (Dx Dy)^(2/3),  K_M = Cs^(4/3) epsilon^(1/3) Dz^(4/3)   (Eq. KmM),
        K_h = (1 + 2 l / sqrt(Dx Dy)) K_m,  K_H = (1 + 2 l / Dz) K_M  (Deardorff's diffusivity ratios),
        l = 0.75 sqrt(e) / N, the subgrid mixing length, capped at Delta and equal to Delta
        where N^2 <= 0.  The subgrid kinetic energy e (tau_kk in Section 2.4) comes from
        Deardorff's eddy-viscosity relation nu_tau = 0.1 l e^(1/2) taken with l = Delta.
        Returns (K_m, K_M, K_h, K_H).
        """
        nu = (self.Cs * self.delta_les) ** 2 * s
        eps = nu * s * s / 2.0
        c = self.Cs ** (4.0 / 3.0) * np.cbrt(eps)
        Km = c * (self.dx * self.dy_h) ** (2.0 / 3.0)
        KM = c * self.dz ** (4.0 / 3.0)
        if self.N2 > 0.0:
            sqrt_e = nu / (0.1 * self.delta_les)
            l = np.minimum(self.delta_les, 0.75 * sqrt_e / math.sqrt(self.N2))
        else:
            l = self.delta_les * np.ones_like(s)
        Kh = (1.0 + 2.0 * l / math.sqrt(self.dx * self.dy_h)) * Km
        KH = (1.0 + 2.0 * l / self.dz) * KM
        return Km, KM, Kh, KH

    def eddy(self, U: np.ndarray):
        """(K_M, K_H) on the halo-r region: scalars (constant mode) or mirrored-even fields.

        In the Deardorff mode each is a list with one coefficient field per
        direction (x, [y,] z): momentum [K_m, (K_m,) K_M], heat [K_h, (K_h,) K_H].
        """
        if self.sgs_mode == SGS_CONST:
            return self.K_M, self.K_H
        r = self.r
        grads = []
        for i in self.vel:
            P = self.extend(U[i], self.H, self.parity[i])
            grads.append([self.crop(g, r) for g in self.grad_halo(P)])
        if self.sgs_mode == SGS_DEARDORFF:
            Km, KM, Kh, KH = (self.extend(k, r, (1.0, 1.0)) for k in self.deardorff(self.strain_magnitude(grads)))
            horiz = self.dim - 1
            return [Km] * horiz + [KM], [Kh] * horiz + [KH]
        nu = self.smagorinsky_nu(grads)
        nu_r = self.extend(nu, r, (1.0, 1.0))
        return nu_r, nu_r / self.Pr

    # -------------------------------------------------------------- diffusion
    def diffusion(self, K_r, grad_phi_r: list) -> np.ndarray:
        """sum_j D_j(K_j D_j phi) on the interior; K scalar, a field on the halo-r region, or
        a list of one such coefficient per direction (anisotropic closure)."""
        if isinstance(K_r, list):
            return self.div_halo([k * g for k, g in zip(K_r, grad_phi_r)])
        return self.div_halo([K_r * g for g in grad_phi_r])

    # ---------------------------------------------------------------------- F
    def set_heat_flux(self, H):
        self.heat = None if H is None else np.asarray(H, dtype=np.float64)

    def F(self, U: np.ndarray) -> np.ndarray:
        """Semi-discrete right-hand side F(u) of Eq. ds for all fields."""
        U = np.asarray(U, dtype=np.float64)
        H, r = self.H, self.r
        P = [self.extend(U[f], H, self.parity[f]) for f in range(self.nf)]
        G = [self.grad_halo(P[f]) for f in range(self.nf)]       # D_j f on halo r
        vel_pad = [P[i] for i in self.vel]
        K_M, K_H = self.eddy(U)
        out = np.zeros_like(U)
        interior = [self.crop(g, r) for g in G[self.ip]]        # D_j p on the interior
        div_u = 0.0
        for j, i in enumerate(self.vel):
            div_u = div_u + self.crop(G[i][j], r)
        for f in range(self.nf):
            out[f] = -self.convection(vel_pad, P[f], G[f])
        for j, i in enumerate(self.vel):                         # momentum
            out[i] += -self.theta0 * interior[j] + self.diffusion(K_M, G[i])
        out[self.iw] += self.g * U[self.ith] / self.theta0       # buoyancy
        out[self.ith] += -self.beta * U[self.iw] + self.diffusion(K_H, G[self.ith])
        if self.heat is not None:
            out[self.ith][0] += self.heat / (self.rho0 * self.cp * self.dz)
        out[self.ip] += -self.gamma_p * (self.pbar + U[self.ip]) * div_u
        return out

    # ---------------------------------------------------------------------- R
    def rhs_f(self, Un: np.ndarray) -> np.ndarray:
        """f(u^n) = 2u^n/dt + F(u^n), the right side of Eq. ns."""
        return 2.0 * Un / self.dt + self.F(Un)

    def residual(self, U: np.ndarray, f: np.ndarray) -> np.ndarray:
        """R(u) = L(u) - f = 2u/dt - F(u) - f (Eq. ns and the Newton residual of Section 2.5.1)."""
        return 2.0 * U / self.dt - self.F(U) - f

    # ------------------------------------------------------------ scaled norms
    def scale(self, V: np.ndarray) -> np.ndarray:
        """W v: every field divided by its scale (U, U, Theta, P)."""
        return V / self.scales.reshape((-1,) + (1,) * (V.ndim - 1))

    def unscale(self, V: np.ndarray) -> np.ndarray:
        return V * self.scales.reshape((-1,) + (1,) * (V.ndim - 1))

    def fd_epsilon(self, U: np.ndarray, Vhat: np.ndarray, eps_mach: float = EPS_FP64) -> float:
        """eps = sqrt(eps_mach (1 + ||W u||)) / ||v_hat||, both norms Euclidean in scaled units."""
        nv = float(np.sqrt(np.sum(Vhat * Vhat)))
        if nv == 0.0:
            return 0.0
        nu = float(np.sqrt(np.sum(self.scale(U) ** 2)))
        return math.sqrt(eps_mach * (1.0 + nu)) / nv

    def jv(self, U: np.ndarray, FU: np.ndarray, V: np.ndarray, eps: float) -> np.ndarray:
        """Forward-difference J v = 2v/dt - (F(u + eps v) - F(u))/eps (Eq. fd), unscaled units."""
        if eps == 0.0:
            return np.zeros_like(V)
        return 2.0 * V / self.dt - (self.F(U + eps * V) - FU) / eps

    def jv_scaled(self, U: np.ndarray, FU: np.ndarray, Vhat: np.ndarray) -> np.ndarray:
        """J_hat v_hat = W J W^{-1} v_hat with the epsilon rule applied to the scaled vectors."""
        V = self.unscale(Vhat)
        eps = self.fd_epsilon(U, Vhat)
        # the difference quotient is taken along V = W^{-1} v_hat with step eps
        return self.scale(self.jv(U, FU, V, eps))

    # -------------------------------------------------------- block precond.
    def frozen_eddy(self, U: np.ndarray):
        """Exchange coefficients frozen at the current Newton iterate (preconditioner input)."""
        return self.eddy(U)

    def block_operator(self, K_r, phi: np.ndarray, f: int) -> np.ndarray:
        """A_f phi = (2/dt) phi - sum_j D_j(K D_j phi): field block f of L without coupling."""
        out = 2.0 * phi / self.dt
        if f == self.ip:
            return out
        P = self.extend(phi, self.H, self.parity[f])
        return out - self.diffusion(K_r, self.grad_halo(P))

    def gershgorin_bounds(self, K_max):
        """Eigenvalue bounds of A_f: [2/dt, 2/dt + (sum_l |d_l|)^2 sum_j K_max,j / h_j^2], with
        K_max the largest exchange coefficient (one number, or one per direction)."""
        c = sum(abs(v) for v in self.d.values())
        lo = 2.0 / self.dt
        kj = K_max if isinstance(K_max, (list, tuple)) else [K_max] * len(self.spacing)
        return lo, lo + c * c * sum(k / (h * h) for k, h in zip(kj, self.spacing))

    @staticmethod
    def kmax_of(K):
        """Largest value of an exchange coefficient (scalar, field, or per-direction list)."""
        if isinstance(K, list):
            return [Model.kmax_of(k) for k in K]
        return float(K) if np.isscalar(K) else float(np.max(K))

    def precond(self, U_frozen: np.ndarray, Rhat: np.ndarray, sweeps: int) -> np.ndarray:
        """Field-block physics-based preconditioner z = M^{-1} r (Section 2.5.2).

        Off-diagonal field couplings and the (zero-diagonal) convection are
        dropped; every diagonal block A_f is inverted approximately by
        ``sweeps`` steps of the Chebyshev iteration on its Gershgorin interval
        (a fixed linear map).  Blocks are per-field, so the diagonal scaling W
        commutes with M and the map is applied to scaled vectors directly.
        """
        K_M, K_H = self.frozen_eddy(U_frozen)
        Z = np.zeros_like(Rhat)
        for f in range(self.nf):
            K = K_H if f == self.ith else K_M
            lo, hi = self.gershgorin_bounds(0.0 if f == self.ip else self.kmax_of(K))
            Z[f] = chebyshev(lambda x: self.block_operator(K, x, f), Rhat[f], lo, hi, sweeps)
        return Z

    def block_apply(self, U_frozen: np.ndarray, Xhat: np.ndarray) -> np.ndarray:
        """P x: the field-block operator whose blocks ``precond`` inverts (scaled units)."""
        K_M, K_H = self.frozen_eddy(U_frozen)
        return np.stack([self.block_operator(K_H if f == self.ith else K_M, Xhat[f], f) for f in range(self.nf)])

    # ------------------------------------------------- nonlinear preconditioning
    def nonlinear_pc_residual(self, U: np.ndarray, f: np.ndarray, sweeps: int) -> np.ndarray:
        """The preconditioned nonlinear residual of Section 2.5.2 in scaled units,
        R~(u) = u - P^{-1}(u) [f - L(u) + P(u) u], with P the field-block operator
        frozen at u and P^{-1} applied by ``precond`` (R = L(u) - f)."""
        Uh = self.scale(U)
        Rh = self.scale(self.residual(U, f))
        return Uh - self.precond(U, self.block_apply(U, Uh) - Rh, sweeps)

    def left_pc_residual(self, U: np.ndarray, f: np.ndarray, sweeps: int) -> np.ndarray:
        """M^{-1} W R(u): the same quantity for an exact P^{-1}; with the Chebyshev
        approximation M^{-1} it keeps the root of R (R~ above does not)."""
        return self.precond(U, self.scale(self.residual(U, f)), sweeps)

    # ------------------------------------------------- acoustic Schur complement
    def _d_interior(self, a: np.ndarray, parity, j: int) -> np.ndarray:
        """D_j a on the interior of a field with the given mirror parity."""
        return self.crop(self.grad_halo(self.extend(a, self.H, parity))[j], self.r)

    def helmholtz(self, p: np.ndarray) -> np.ndarray:
        """H p = (2/dt) p - a sum_j D_j D_j p, a = gamma_p pbar theta0 dt / 2 (p even in z)."""
        a = self.gamma_p * self.pbar * self.theta0 * self.dt / 2.0
        P = self.extend(p, self.H, self.parity[self.ip])
        return 2.0 * p / self.dt - a * self.div_halo(self.grad_halo(P))

    def helmholtz_bounds(self):
        """Gershgorin interval of H: [2/dt, 2/dt + (3/2)^2 a sum_j 1/h_j^2]."""
        a = self.gamma_p * self.pbar * self.theta0 * self.dt / 2.0
        return self.gershgorin_bounds(a)

    def schur_precond(self, U_frozen: np.ndarray, Vhat: np.ndarray, sweeps: int) -> np.ndarray:
        """Acoustic Schur-complement preconditioner z = P v (scaled units, 2-D and 3-D).

        Section 2.5 follows the semi-implicit elimination of the fast acoustic
        terms (Skamarock & Klemp): keeping only (2/dt) I and the pressure
        gradient / divergence couplings of Eqs. ch2_28-ch2_30 linearised about
        the reference pressure pbar,
            (2/dt) du_i + theta0 D_i dp = r_i  (every velocity component i),
            (2/dt) dp + gamma_p pbar sum_i D_i du_i = r_p,
        the velocities are eliminated, leaving the pressure Helmholtz problem
            H dp = r_p - gamma_p pbar (dt/2) sum_i D_i r_i,
        solved approximately by ``sweeps`` Chebyshev steps on its Gershgorin
        interval (a fixed linear map); then du_i = (dt/2)(r_i - theta0 D_i dp).
        Advection, diffusion and buoyancy are dropped; theta gets one
        Chebyshev step of its field block (r_theta / theta_c).  r = W^-1 v,
        z = W dz.
        """
        dt = self.dt
        r = self.unscale(Vhat)
        div_r = 0.0
        for j, i in enumerate(self.vel):
            div_r = div_r + self._d_interior(r[i], self.parity[i], j)
        rhs = r[self.ip] - self.gamma_p * self.pbar * (dt / 2.0) * div_r
        lo, hi = self.helmholtz_bounds()
        dp = chebyshev(self.helmholtz, rhs, lo, hi, sweeps)
        Z = np.zeros_like(r)
        for j, i in enumerate(self.vel):
            Z[i] = (dt / 2.0) * (r[i] - self.theta0 * self._d_interior(dp, self.parity[self.ip], j))
        K_M, K_H = self.frozen_eddy(U_frozen)
        lo_t, hi_t = self.gershgorin_bounds(self.kmax_of(K_H))
        Z[self.ith] = r[self.ith] / (0.5 * (lo_t + hi_t))
        Z[self.ip] = dp
        return self.scale(Z)

    # ------------------------------------------------------------ budgets
    def budgets(self, U: np.ndarray) -> dict:
        """Energy budgets and extremes (Section 3.1.3, literal E_k and E_p formulas)."""
        dV = self.dx * self.dz * (self.dy if self.dim == 3 else 1.0)
        z = (np.arange(self.nz) + 0.5) * self.dz
        zshape = (self.nz,) + (1,) * (U.ndim - 2)
        ek = 0.5 * sum(np.sum(U[i] ** 2) for i in self.vel) * dV
        ep = np.sum((self.lz - z).reshape(zshape) * U[self.ith]) * dV
        div = 0.0
        for j, i in enumerate(self.vel):
            P = self.extend(U[i], self.H, self.parity[i])
            div = div + self.crop(self.grad_halo(P)[j], self.r)
        return {
            "E_k": float(ek), "E_p": float(ep),
            "sum_theta": float(np.sum(U[self.ith]) * dV),
            "sum_div": float(np.sum(div) * dV),
            "max": [float(np.max(U[f])) for f in range(self.nf)],
            "min": [float(np.min(U[f])) for f in range(self.nf)],
        }


def chebyshev(apply_A, r: np.ndarray, lo: float, hi: float, steps: int) -> np.ndarray:
    """``steps`` Chebyshev iterations for A x = r from x = 0 on the spectrum [lo, hi].

    Three-term recurrence of the classical Chebyshev semi-iteration (Saad,
    Iterative Methods for Sparse Linear Systems, Alg. 12.1).
    """
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    if delta <= 1e-14 * theta:
        return r / theta
    sigma = theta / delta
    rho = 1.0 / sigma
    d = r / theta
    x = np.zeros_like(r)
    for k in range(steps):
        x = x + d
        if k == steps - 1:
            break
        res = r - apply_A(x)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * res
        rho = rho_new
    return x
