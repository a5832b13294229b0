"""FP64 oracle of the 1D normal shock solved end to end: full tensor and
adaptive low rank, first-order upwind in x, forward Euler in t.

TEST INFRASTRUCTURE ONLY (see the package docstring): imported by tests, the
smoke check and the benchmark's CPU leg, never by the CUDA library, with
which it shares no code.

Problem (paper Sec. 4, eqs. "eqn:normalshock", "eqn:normalshockboundary" and
the Rankine-Hugoniot solution "relation"; set-up of Sec. 5.2): x in
[-L_x, L_x] with N_x cells x_p = -L_x + (p - 1/2) dx, dx = 2 L_x / N_x;
velocity grid and collision operator of oracle.collision, or the Carleman
form of oracle.carleman on the same grid (R_gas = 1).
Upstream (rho, u, T)_L = (1, M sqrt(gamma), 1), gamma = (d+2)/d; downstream
from "relation".  Initial data: the Maxwellian of rho_0, u_0, T_0, each
blending L into R as (tanh(alpha x) + 1)/2 (reading of the garbled formula of
Sec. 5.2).  Inflow boundaries: f = f_L for v_1 > 0 at the left end and
f = f_R for v_1 < 0 at the right end (Sec. 2.3, "Treatment of the boundary
condition").

Full tensor (Sec. 2.3, eq. "scheme:fullupwind", forward Euler):
    f^{n+1} = f - dt (v1+ D+ f + v1- D- f) + dt Q(f, f),
    D+ f(x_p) = (f(x_p) - f(x_{p-1})) / dx,  D- f(x_p) = (f(x_{p+1}) - f(x_p)) / dx,
    ghost cells f(x_0) = f_L, f(x_{N+1}) = f_R; v1+- = (v1 +- |v1|) / 2.

Low rank (Sec. 2.4, the fully discrete scheme with the upwind forms of
Sec. 2.3; Sec. 3.1, adding basis; Sec. 3.2, dropping basis), state
f = sum_ij X_i(x) S_ij V_j(v), X_i and V_j orthonormal under the midpoint
rules <a, b>_x = dx sum a b and <a, b>_v = dv^d sum a b.  One step:
  0. add basis (Sec. 3.1, spatially homogeneous boundary data): SVD of
     F_b = [f_L; f_R], keep singular values >= 1e-10, append those right
     singular vectors to V and a random X_h (an input) to X, zero-pad S, QR
     both (Householder), S <- S_x S_hat S_v^T;
  1. K-step: K_j = sum_i X_i S_ij;
       K_j <- K_j - dt sum_l (A+_jl D+ K_l + A-_jl D- K_l) + dt sum_mn T_jmn K_m K_n,
       A+-_jl = <v1+- V_j V_l>_v, T_jmn = <V_j Q(V_m, V_n)>_v; K's boundary values
       (eq. "boundary general", outflow part extrapolated from the first
       interior cell)
         K_j(x_0)     = <f_L 1{v1 > 0}, V_j> + sum_l K_l(x_1) <1{v1 <= 0} V_l V_j>,
         K_j(x_{N+1}) = <f_R 1{v1 < 0}, V_j> + sum_l K_l(x_N) <1{v1 >= 0} V_l V_j>;
     QR: K_j = sum_i X'_i S1_ij;
  2. S-step: S2_ij = S1_ij + dt sum_l (A+_jl <X'_i D+ K_l> + A-_jl <X'_i D- K_l>)
                     - dt sum_mn T_jmn sum_l (sum_k E_ikl S1_km) S1_ln,
     with the updated K (and its boundary values), E_ikl = <X'_i X'_k X'_l>_x;
  3. L-step: L_i = sum_j S2_ij V_j, K~_j = sum_i X'_i S2_ij,
       L_i <- L_i - dt sum_l (v1+ <X'_i D+ K~_l> + v1- <X'_i D- K~_l>) V_l
                  + dt sum_pq C_ipq Q(V_p, V_q),  C_ipq = sum_n (sum_m E_imn S2_mp) S2_nq;
     QR: L_i = sum_j S'_ij V'_j;
  4. drop (Sec. 3.2): S' = U Sigma Q^T, keep sigma >= drop_tol, rotate X', V'.
The step also returns err = ||f^{n+1} - f^n||_{x,v} before the drop, from the
increments dK, dS, dL and the cross terms of Sec. 5.1 (f is not rebuilt).
Initial factors (Sec. 2.4): truncated SVD of f^0 under the two inner products.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import carleman as CM
from . import collision as C
from . import lowrank as LR


def shock_states(mach: float, d: int):
    """Upstream and downstream (rho, u, T) of Sec. 4 eq. "relation" (R_gas = 1)."""
    gamma = (d + 2.0) / d
    rho_l, t_l = 1.0, 1.0
    u_l = mach * math.sqrt(gamma * t_l)
    m2 = mach * mach
    rho_r = rho_l * (d + 1.0) * m2 / (m2 + d)
    u_r = u_l * (m2 + d) / ((d + 1.0) * m2)
    t_r = t_l * ((d + 2.0) * m2 - 1.0) * (m2 + d) / ((d + 1.0) ** 2 * m2)
    return (rho_l, u_l, t_l), (rho_r, u_r, t_r)


@dataclass
class ShockProblem:
    vel: C.Problem          # velocity grid and (by default) the separated collision operator
    n_x: int
    L_x: float
    mach: float
    alpha: float = 0.5
    carleman: CM.CarlemanProblem | None = None   # when set, Q is the Carleman form on the same grid

    def collide(self, fields: np.ndarray, pairs) -> np.ndarray:
        if self.carleman is not None:
            return CM.collide_fields(self.carleman, fields, pairs)
        return C.collide_fields(self.vel, fields, pairs)

    @property
    def dx(self) -> float:
        return 2.0 * self.L_x / self.n_x

    @property
    def x(self) -> np.ndarray:
        return -self.L_x + (np.arange(self.n_x) + 0.5) * self.dx

    @property
    def wv(self) -> float:
        return self.vel.dv ** self.vel.d

    def vgrid(self):
        """Velocity components [d][n_v] of the grid v_j = -L + j dv."""
        p = self.vel
        axis = -p.L + np.arange(p.N) * p.dv
        mesh = np.meshgrid(*([axis] * p.d), indexing="ij")
        return np.stack([m.reshape(-1) for m in mesh])

    def v1(self) -> np.ndarray:
        return self.vgrid()[0]

    def states(self):
        return shock_states(self.mach, self.vel.d)

    def maxwellian(self, rho, u, T) -> np.ndarray:
        """rho (2 pi T)^{-d/2} exp(-|v - u e_1|^2 / 2T) on the grid, [n_v] (or [n][n_v] for arrays)."""
        vg = self.vgrid()
        rho, u, T = (np.asarray(a, dtype=np.float64)[..., None] for a in (rho, u, T))
        d = self.vel.d
        e = (vg[0] - u) ** 2 + sum(vg[k] ** 2 for k in range(1, d))
        return rho / (2.0 * math.pi * T) ** (d / 2.0) * np.exp(-e / (2.0 * T))

    def boundary(self):
        (rl, ul, tl), (rr, ur, tr) = self.states()
        return self.maxwellian(rl, ul, tl), self.maxwellian(rr, ur, tr)

    def initial(self) -> np.ndarray:
        """f^0 [n_x][n_v]: Maxwellian of the tanh-blended states (Sec. 5.2)."""
        (rl, ul, tl), (rr, ur, tr) = self.states()
        s = (np.tanh(self.alpha * self.x) + 1.0) / 2.0
        return self.maxwellian(rl + (rr - rl) * s, ul + (ur - ul) * s, tl + (tr - tl) * s)

    def moments(self, f: np.ndarray):
        """Density, bulk velocity u_1 and temperature per cell of f [n_x][n_v]."""
        vg = self.vgrid()
        rho = self.wv * f.sum(axis=1)
        u1 = self.wv * (f * vg[0]).sum(axis=1) / rho
        e = (vg[0][None, :] - u1[:, None]) ** 2 + sum(vg[k][None, :] ** 2 for k in range(1, self.vel.d))
        T = self.wv * (f * e).sum(axis=1) / (self.vel.d * rho)
        return rho, u1, T


def collide_cells(sp: ShockProblem, f: np.ndarray) -> np.ndarray:
    """Q(f(x_p), f(x_p)) for every cell, [n_x][n_v]."""
    fields = f.reshape((f.shape[0],) + sp.vel.shape)
    Q = sp.collide(fields, [(p, p) for p in range(f.shape[0])])
    return Q.reshape(f.shape[0], -1)


def full_step(sp: ShockProblem, f: np.ndarray, dt: float, Q: np.ndarray | None = None) -> np.ndarray:
    """One forward-Euler step of the full-tensor upwind scheme (eq. "scheme:fullupwind")."""
    fL, fR = sp.boundary()
    v1 = sp.v1()
    vp, vm = np.maximum(v1, 0.0), np.minimum(v1, 0.0)
    left = np.vstack([fL[None, :], f[:-1]])
    right = np.vstack([f[1:], fR[None, :]])
    if Q is None:
        Q = collide_cells(sp, f)
    return f - dt * (vp * (f - left) / sp.dx + vm * (right - f) / sp.dx) + dt * Q


def mass_flux_balance(sp: ShockProblem, f: np.ndarray, dt: float):
    """Change of total mass over one full-tensor step minus the boundary fluxes
    (upwind scheme in conservation form; the collision term carries no mass)."""
    fL, fR = sp.boundary()
    v1 = sp.v1()
    vp, vm = np.maximum(v1, 0.0), np.minimum(v1, 0.0)
    g = full_step(sp, f, dt, Q=np.zeros_like(f))
    dm = sp.dx * sp.wv * (g.sum() - f.sum())
    flux_in = dt * sp.wv * ((vp * fL).sum() - (vp * f[-1]).sum() - (vm * fR).sum() + (vm * f[0]).sum())
    return dm, flux_in


# -------------------------------------------------------------------- low rank

def factor(sp: ShockProblem, f: np.ndarray, r: int):
    """Initial factors (Sec. 2.4): truncated SVD of f under <.,.>_x and <.,.>_v."""
    w = math.sqrt(sp.dx * sp.wv)
    U, s, Wt = np.linalg.svd(w * f, full_matrices=False)
    X = U[:, :r].T / math.sqrt(sp.dx)
    V = Wt[:r] / math.sqrt(sp.wv)
    return X, np.diag(s[:r]), V


def reconstruct(X: np.ndarray, S: np.ndarray, V: np.ndarray) -> np.ndarray:
    """f[x][v] = sum_ij X_i(x) S_ij V_j(v)."""
    return X.T @ S @ V


def add_basis(sp: ShockProblem, X, S, V, Xh):
    """Sec. 3.1 for spatially homogeneous boundary data: SVD of F_b = [f_L; f_R],
    singular values below 1e-10 dropped, concatenate, QR both, S_q = S_x S_hat S_v^T."""
    fL, fR = sp.boundary()
    _, sb, Qbt = np.linalg.svd(np.vstack([fL, fR]), full_matrices=False)
    Qb = Qbt[sb >= 1e-10]
    rb = Qb.shape[0]
    Xhat = np.vstack([X, Xh[:rb]])
    Vhat = np.vstack([V, Qb])
    r = S.shape[0]
    Shat = np.zeros((r + rb, r + rb))
    Shat[:r, :r] = S
    Xq, Sx = LR.qr_weighted(Xhat, sp.dx)
    Vq, Sv = LR.qr_weighted(Vhat, sp.wv)
    return Xq, Sx @ Shat @ Sv.T, Vq


def _ghosts(sp: ShockProblem, K: np.ndarray, V: np.ndarray):
    """Boundary values of K (eq. "boundary general"), outflow part from the first interior cell."""
    fL, fR = sp.boundary()
    v1 = sp.v1()
    w = sp.wv
    kL = w * (V * (fL * (v1 > 0))).sum(axis=1) + (w * (V * (v1 <= 0)) @ V.T).T @ K[:, 0]
    kR = w * (V * (fR * (v1 < 0))).sum(axis=1) + (w * (V * (v1 >= 0)) @ V.T).T @ K[:, -1]
    return kL, kR


def _upwind(sp: ShockProblem, K: np.ndarray, V: np.ndarray):
    """D+ K and D- K [r][n_x] with K's boundary values."""
    kL, kR = _ghosts(sp, K, V)
    left = np.hstack([kL[:, None], K[:, :-1]])
    right = np.hstack([K[:, 1:], kR[:, None]])
    return (K - left) / sp.dx, (right - K) / sp.dx


def lowrank_step(sp: ShockProblem, X, S, V, dt: float, drop_tol: float, Xh, return_parts: bool = False):
    """One adaptive low-rank step (Sec. 3.1, Sec. 2.4, Sec. 3.2)."""
    X, S, V = add_basis(sp, X, S, V, Xh)
    r = S.shape[0]
    v1 = sp.v1()
    vp, vm = np.maximum(v1, 0.0), np.minimum(v1, 0.0)
    Ap = sp.wv * (V * vp) @ V.T                 # A+_jl
    Am = sp.wv * (V * vm) @ V.T
    fields = V.reshape((r,) + sp.vel.shape)
    pairs = [(m, n) for m in range(r) for n in range(r)]
    Qv = sp.collide(fields, pairs).reshape(r * r, -1)
    T = C.project(sp.vel, fields, Qv.reshape((r * r,) + sp.vel.shape)).reshape(r, r, r)
    # K-step
    K = S.T @ X                                 # K_j = sum_i X_i S_ij
    Dp, Dm = _upwind(sp, K, V)
    K1 = K - dt * (Ap @ Dp + Am @ Dm) + dt * LR.kstep_collision(T, K)
    X1, S1 = LR.qr_weighted(K1, sp.dx)
    # S-step
    Dp, Dm = _upwind(sp, K1, V)
    Bp = sp.dx * X1 @ Dp.T                      # <X'_i D+ K_l>
    Bm = sp.dx * X1 @ Dm.T
    E = LR.triple_products(X1, sp.dx)
    S2 = S1 + dt * (Bp @ Ap.T + Bm @ Am.T) - dt * LR.sstep_collision(T, E, S1)
    # L-step
    L = S2 @ V
    Kt = S2.T @ X1
    Dp, Dm = _upwind(sp, Kt, V)
    Bp = sp.dx * X1 @ Dp.T
    Bm = sp.dx * X1 @ Dm.T
    L1 = L - dt * (vp * (Bp @ V) + vm * (Bm @ V)) + dt * LR.lstep_collision(Qv, LR.lstep_coupling(E, S2))
    Vn, R = LR.qr_weighted(L1, sp.wv)
    Sn = R.T                                    # L_i = sum_j Sn_ij V'_j
    # change of f over the step from the increments (Sec. 5.1, eqs. "err low rank1"
    # and "err low rank2"): dK, dS, dL and the three cross terms
    dK, dS, dL = K1 - K, S2 - S1, L1 - L
    P = sp.dx * X1 @ dK.T                       # P_ij = <dK_j, X'_i>_x
    Qc = sp.wv * dL @ V.T                       # Qc_ij = <dL_i, V_j>_v
    err2 = (sp.dx * (dK * dK).sum() + (dS * dS).sum() + sp.wv * (dL * dL).sum()
            + 2.0 * (P * dS).sum() + 2.0 * (dS * Qc).sum() + 2.0 * (P * Qc).sum())
    # drop
    U, sig, Qm, rk = LR.svd_truncate(Sn, drop_tol)
    Xd = LR.rotate(X1, U, rk)
    Vd = LR.rotate(Vn, Qm, rk)
    out = (Xd, np.diag(sig[:rk]), Vd)
    if return_parts:
        return out, {"rank_before_drop": r, "sigma": sig, "err": math.sqrt(max(err2, 0.0))}
    return out


def random_xh(n_x: int, rb: int = 2, seed: int = 0) -> np.ndarray:
    """The random X_h of Sec. 3.1 (an input: both sides receive the same values)."""
    return np.random.default_rng(seed).standard_normal((rb, n_x))
