"""Seeded synthetic inputs for the collision-operator workloads.

This module only produces input samples (physical values of distribution
functions on the velocity grid).  It holds none of the collision method's
arithmetic: no spectra, no quadrature, no collision integrals.  Both the FP64
oracle and the CUDA path consume what it returns, so neither side can bias the
other through its inputs.

Grid convention (Sec. 2.1 of the paper: a uniform grid on [-L, L]^d): the
velocity of index j along an axis is v_j = -L + j * (2L/N), j = 0..N-1, and a
field is stored C-ordered as [i0][i1]...[i_{d-1}] with axis 0 slowest.

Workload recipes (all seeded, all analytic, the paper ships no data):
  * BKW closed-form solutions for Maxwell molecules (2D and 3D);
  * Maxwellians M(rho, u, T);
  * Hermite-Maxwellian velocity bases V_j: random polynomials on a tensor
    probabilists' Hermite basis times the unit Maxwellian, orthonormalised in
    the midpoint-rule inner product <.,.>_v (Sec. 2.4, midpoint rule);
  * normal-shock cells f_x = (1-w(x)) M_L + w(x) M_R with Rankine-Hugoniot
    states (Sec. 4, eq. "relation").
"""
from __future__ import annotations

import math
from itertools import product

import numpy as np


def velocity_axis(N: int, L: float) -> np.ndarray:
    """Grid points v_j = -L + j*2L/N along one axis (FP64)."""
    return -L + np.arange(N, dtype=np.float64) * (2.0 * L / N)


def velocity_mesh(N: int, d: int, L: float) -> list[np.ndarray]:
    """d arrays of shape [N]*d holding v_0..v_{d-1} at every grid point."""
    ax = velocity_axis(N, L)
    return list(np.meshgrid(*([ax] * d), indexing="ij"))


def maxwellian(N: int, d: int, L: float, rho: float = 1.0, u=None, T: float = 1.0) -> np.ndarray:
    """rho (2 pi T)^(-d/2) exp(-|v-u|^2 / (2T)) sampled on the grid."""
    u = np.zeros(d) if u is None else np.asarray(u, dtype=np.float64)
    V = velocity_mesh(N, d, L)
    r2 = sum((V[a] - u[a]) ** 2 for a in range(d))
    return rho * (2.0 * math.pi * T) ** (-d / 2.0) * np.exp(-r2 / (2.0 * T))


# --------------------------------------------------------------------------
# BKW solutions (Bobylev-Krook-Wu), Maxwell molecules, kernel constant
# b = 1/|S^{d-1}|.  Mass 1, zero mean velocity, temperature 1.
# --------------------------------------------------------------------------

def bkw_K(d: int, t: float) -> float:
    """The BKW scale K(t): 1 - e^{-t/8}/2 in 2D, 1 - e^{-t/6} in 3D."""
    if d == 2:
        return 1.0 - 0.5 * math.exp(-t / 8.0)
    if d == 3:
        return 1.0 - math.exp(-t / 6.0)
    raise ValueError("d must be 2 or 3")


def bkw_profile(r2: np.ndarray, d: int, K: float) -> np.ndarray:
    """BKW f as a function of |v|^2 for a given K."""
    if d == 2:
        return np.exp(-r2 / (2 * K)) / (2 * math.pi * K * K) * (2 * K - 1 + (1 - K) * r2 / (2 * K))
    return (2 * math.pi * K) ** -1.5 * np.exp(-r2 / (2 * K)) * (
        (5 * K - 3) / (2 * K) + (1 - K) * r2 / (2 * K * K))


def bkw(N: int, d: int, L: float, t: float) -> np.ndarray:
    V = velocity_mesh(N, d, L)
    r2 = sum(x * x for x in V)
    return bkw_profile(r2, d, bkw_K(d, t))


# --------------------------------------------------------------------------
# Hermite-Maxwellian bases
# --------------------------------------------------------------------------

def _hermite_prob(n: int, x: np.ndarray) -> np.ndarray:
    """Probabilists' Hermite polynomial He_n(x) by its three-term recurrence."""
    h0 = np.ones_like(x)
    if n == 0:
        return h0
    h1 = x.copy()
    for k in range(1, n):
        h0, h1 = h1, x * h1 - k * h0
    return h1


def basis_degree(d: int, r: int) -> int:
    """Smallest total degree >= 3 whose polynomial space in d variables has dim >= r."""
    deg = 3
    while math.comb(deg + d, d) < r:
        deg += 1
    return deg


def hermite_maxwellian_basis(N: int, d: int, L: float, r: int, seed: int) -> np.ndarray:
    """r functions V_j(v) = p_j(v) * (2pi)^{-d/2} e^{-|v|^2/2}, orthonormal under
    <a,b>_v = dv^d sum_v a b (midpoint rule).  p_j has N(0,1) coefficients on
    the tensor Hermite basis of total degree <= basis_degree(d, r).
    Returns FP64 [r][N]*d."""
    deg = basis_degree(d, r)
    rng = np.random.default_rng(seed)
    V = velocity_mesh(N, d, L)
    m = (2 * math.pi) ** (-d / 2.0) * np.exp(-0.5 * sum(x * x for x in V))
    H = [[_hermite_prob(k, V[a]) for k in range(deg + 1)] for a in range(d)]
    monos = [e for e in product(range(deg + 1), repeat=d) if sum(e) <= deg]
    coeff = rng.standard_normal((r, len(monos)))
    funcs = np.zeros((r,) + (N,) * d)
    for i, e in enumerate(monos):
        term = np.ones((N,) * d)
        for a in range(d):
            term = term * H[a][e[a]]
        funcs += coeff[:, i].reshape((r,) + (1,) * d) * term
    funcs *= m
    dv = (2.0 * L / N) ** d
    flat = funcs.reshape(r, -1)
    # modified Gram-Schmidt, two sweeps, midpoint-rule inner product
    for _ in range(2):
        for j in range(r):
            for i in range(j):
                flat[j] -= dv * np.dot(flat[i], flat[j]) * flat[i]
            flat[j] /= math.sqrt(dv * np.dot(flat[j], flat[j]))
    return flat.reshape((r,) + (N,) * d)


# --------------------------------------------------------------------------
# Normal-shock cells (Sec. 4, eq. "relation"; Sec. 5.2 geometry)
# --------------------------------------------------------------------------

def rankine_hugoniot(d: int, mach: float, rho_L: float = 1.0, T_L: float = 1.0, R_gas: float = 1.0):
    """Upstream/downstream (rho, u, T) for upstream Mach number `mach`, gas
    constant gamma = (d+2)/d (the paper's relation for the normal shock)."""
    gam = (d + 2.0) / d
    u_L = mach * math.sqrt(gam * R_gas * T_L)
    M2 = mach * mach
    rho_R = rho_L * (d + 1) * M2 / (M2 + d)
    u_R = u_L * (M2 + d) / ((d + 1) * M2)
    T_R = T_L * ((d + 2) * M2 - 1) * (M2 + d) / ((d + 1) ** 2 * M2)
    return (rho_L, u_L, T_L), (rho_R, u_R, T_R)


def shock_cell_weights(n_cells: int = 512, x_min: float = -30.0, x_max: float = 30.0,
                       delta: float = 2.0) -> np.ndarray:
    """w(x_p) = (1 + tanh(x_p/delta))/2 at cell centres x_p of [x_min, x_max]."""
    h = (x_max - x_min) / n_cells
    x = x_min + (np.arange(n_cells) + 0.5) * h
    return 0.5 * (1.0 + np.tanh(x / delta))


def shock_states_fields(N: int, d: int, L: float, mach: float = 3.0):
    """The two Maxwellians M_L (upstream) and M_R (downstream), drift along axis 0."""
    (rL, uL, TL), (rR, uR, TR) = rankine_hugoniot(d, mach)
    eL = np.zeros(d); eL[0] = uL
    eR = np.zeros(d); eR[0] = uR
    return maxwellian(N, d, L, rL, eL, TL), maxwellian(N, d, L, rR, eR, TR)


def shock_cells(N: int, d: int, L: float, n_cells: int = 512, mach: float = 3.0,
                delta: float = 2.0):
    """Cell distributions f_x = (1-w) M_L + w M_R, FP64 [n_cells][N]*d, plus w."""
    fL, fR = shock_states_fields(N, d, L, mach)
    w = shock_cell_weights(n_cells, delta=delta)
    wb = w.reshape((-1,) + (1,) * d)
    return (1.0 - wb) * fL[None] + wb * fR[None], w


def random_fields(N: int, d: int, L: float, n: int, seed: int) -> np.ndarray:
    """n smooth random fields: Maxwellians with random (rho, u, T) plus a small
    seeded Hermite perturbation; used for edge-case parity inputs."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n,) + (N,) * d)
    for i in range(n):
        rho = rng.uniform(0.5, 2.0)
        u = rng.uniform(-1.0, 1.0, size=d)
        T = rng.uniform(0.6, 1.6)
        out[i] = maxwellian(N, d, L, rho, u, T)
    pert = hermite_maxwellian_basis(N, d, L, min(n, math.comb(3 + d, d)), seed + 7919)
    for i in range(n):
        out[i] += 0.05 * pert[i % pert.shape[0]]
    return out
