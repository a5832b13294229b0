"""FP64 oracle of the Carleman-form fast spectral collision operator for
gamma = d - 2 (2D Maxwell molecules, 3D hard spheres), the Mouhot-Pareschi
algorithm the paper cites and uses for its experiments (Sec. 2.1, Sec. 5).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Derivation (from the definition of Q in Sec. 1).  With x = v' - v and
y = v'_* - v one has x + y = -q, x . y = 0, and the Carleman change of
variables turns the collision integral into
    Q+(g,f)(v) = int int Bt(x,y) delta(x.y) g(v + y) f(v + x) dx dy,
    Q-(g,f)(v) = f(v) int int Bt(x,y) delta(x.y) g(v + x + y) dx dy,
    Bt = 2^{d-1} b |x + y|^{gamma - d + 2}  = 2^{d-1} b  for gamma = d - 2.
This form truncates |x| <= R and |y| <= R (the separated form of
oracle/collision.py truncates |q| <= R instead: a different truncated
operator).  On trigonometric interpolants, Q+hat_k = sum_{l+m=k} beta(l,m)
ghat_l fhat_m with
    beta(l,m) = Bt int_{|x|,|y|<=R} delta(x.y) exp(i pi (l.y + m.x)/L) dx dy
              = Bt int_{half sphere} phi(pi m.e / L) psi(pi |l - (l.e) e| / L) de,
    phi(s) = int_{-R}^{R} |rho|^{d-2} exp(i rho s) drho,
    psi(t) = int_{|y|<=R, y perp e} exp(i y.l pi/L) d^{d-1}y,
closed forms
    d = 2:  phi(s) = 2 sin(R s)/s,                       psi(t) = 2 sin(R t)/t
    d = 3:  phi(s) = 2 (R sin(R s)/s + (cos(R s) - 1)/s^2), psi(t) = 2 pi R J1(R t)/t.
The half sphere is discretised by one direction of each antipodal pair of the
centrally symmetric rule (sigma_p, w_p) of oracle/quadrature (weights summing
to |S^{d-1}|/2).  Hence
    Q+(v) = Bt sum_p w_p A_p(v) B_p(v),  A_p = IDFT(psi_p ghat), B_p = IDFT(phi_p fhat),
    Q-(v) = f_N(v) IDFT(G- ghat)(v),      G-(l) = Bt sum_p w_p phi(pi l.e_p/L) psi_p(l),
where the loss uses the same discrete beta at m = l (so that
beta(l, -l) = beta(l, l) and mass is conserved to rounding).  The grid values
of the gain are the wrapped (mod N) convolution, as in the separated form.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import j1 as _bessel_j1

from . import collision as C
from . import quadrature as quad


@dataclass
class CarlemanProblem:
    N: int
    d: int
    L: float
    R: float
    M: int                      # size of the (full-sphere) direction rule
    b: float | None = None
    _cache: dict = field(default_factory=dict, repr=False)

    def __post_init__(self):
        if self.b is None:
            self.b = 1.0 / C.sphere_area(self.d)
        sigma, w = quad.direction_rule(self.d, self.M)
        keep = []
        for p in range(len(w)):
            ap = int(np.argmin(np.sum((sigma + sigma[p]) ** 2, axis=1)))
            if ap > p:
                keep.append(p)
        self.e = sigma[keep]
        self.w = w[keep]
        self.Bt = 2.0 ** (self.d - 1) * self.b
        # the oracle's spectral helpers take a separated-form Problem for the grid only
        self.grid = C.Problem(N=self.N, d=self.d, L=self.L, R=self.R, gamma=self.d - 2.0, n_rho=1, M=self.M)

    @property
    def shape(self):
        return (self.N,) * self.d


def phi(d: int, R: float, s):
    """int_{-R}^{R} |rho|^{d-2} exp(i rho s) drho (real, even in s)."""
    s = np.asarray(s, dtype=np.float64)
    small = np.abs(s) < 1e-6
    ss = np.where(small, 1.0, s)
    if d == 2:
        out = 2.0 * np.sin(R * ss) / ss
        return np.where(small, 2.0 * R - R ** 3 * s * s / 3.0, out)
    out = 2.0 * (R * np.sin(R * ss) / ss + (np.cos(R * ss) - 1.0) / (ss * ss))
    return np.where(small, R * R - R ** 4 * s * s / 4.0, out)


def psi(d: int, R: float, t):
    """Integral of exp(i y.t) over the (d-1)-ball of radius R perpendicular to e, |t| = t."""
    t = np.abs(np.asarray(t, dtype=np.float64))
    small = t < 1e-6
    tt = np.where(small, 1.0, t)
    if d == 2:
        out = 2.0 * np.sin(R * tt) / tt
        return np.where(small, 2.0 * R - R ** 3 * t * t / 3.0, out)
    out = 2.0 * math.pi * R * _bessel_j1(R * tt) / tt
    return np.where(small, math.pi * R * R * (1.0 - (R * t) ** 2 / 8.0), out)


def wave_vectors(prob: CarlemanProblem) -> np.ndarray:
    """Wrapped integer frequencies k of every spectral index, [d][N]*d."""
    k = C.freq_of_index(prob.N).astype(np.float64)
    return np.stack(np.meshgrid(*([k] * prob.d), indexing="ij"))


def multipliers(prob: CarlemanProblem):
    """phi_p(k) = phi(pi k.e_p / L) and psi_p(k) = psi(pi |k - (k.e_p) e_p| / L)."""
    if "mult" in prob._cache:
        return prob._cache["mult"]
    K = wave_vectors(prob)
    ph, ps = [], []
    for e in prob.e:
        ke = np.tensordot(e, K, axes=(0, 0))
        perp = K - e.reshape((-1,) + (1,) * prob.d) * ke[None]
        kp = np.sqrt(np.sum(perp * perp, axis=0))
        ph.append(phi(prob.d, prob.R, math.pi * ke / prob.L))
        ps.append(psi(prob.d, prob.R, math.pi * kp / prob.L))
    prob._cache["mult"] = (np.stack(ph), np.stack(ps))
    return prob._cache["mult"]


def loss_weight(prob: CarlemanProblem) -> np.ndarray:
    ph, ps = multipliers(prob)
    return prob.Bt * np.tensordot(prob.w, ph * ps, axes=(0, 0))


def collide(prob: CarlemanProblem, spec: np.ndarray, pairs, return_parts: bool = False):
    """Q(g, f) for every (j, l) of `pairs` (g = input j, f = input l); spec are
    the full input spectra (oracle.collision.spectrum)."""
    grid = prob.grid
    pairs = [(int(j), int(l)) for j, l in pairs]
    jj = np.array([j for j, _ in pairs])
    ll = np.array([l for _, l in pairs])
    ph, ps = multipliers(prob)
    P = np.zeros((len(pairs),) + prob.shape)
    for p in range(len(prob.w)):
        A = C.synthesize(grid, ps[p][None] * spec)      # g side: psi_p
        Bf = C.synthesize(grid, ph[p][None] * spec)     # f side: phi_p
        P += prob.w[p] * A[jj] * Bf[ll]
    Q_plus = prob.Bt * P
    lam = C.synthesize(grid, loss_weight(prob)[None] * spec)
    fN = C.synthesize(grid, spec)
    Q_minus = fN[ll] * lam[jj]
    Q = Q_plus - Q_minus
    return (Q, Q_plus, Q_minus) if return_parts else Q


def collide_fields(prob: CarlemanProblem, fields: np.ndarray, pairs, return_parts: bool = False):
    return collide(prob, C.spectrum(prob.grid, fields), pairs, return_parts)


def direct_sum(prob: CarlemanProblem, ghat: np.ndarray, fhat: np.ndarray) -> np.ndarray:
    """Qhat_k = sum_{l+m = k mod N} [beta(l,m) - beta(l,l)] ghat_l fhat_m with the
    discrete beta(l,m) = Bt sum_p w_p phi(pi m.e_p/L) psi(pi |l - (l.e_p)e_p|/L).
    O(n^2 M): tiny grids only."""
    N, d = prob.N, prob.d
    fr = C.freq_of_index(N)
    grids = np.meshgrid(*([fr] * d), indexing="ij")
    kv = np.stack([g.ravel() for g in grids], axis=1).astype(np.float64)     # [n, d]
    n = kv.shape[0]
    gh = ghat.ravel()
    fh = fhat.ravel()
    out = np.zeros(n, dtype=np.complex128)
    idx = {tuple(int(x) for x in k): i for i, k in enumerate(kv)}
    Gm = loss_weight(prob).ravel()
    for a in range(n):
        l = kv[a]
        lperp = [np.linalg.norm(l - np.dot(l, e) * e) for e in prob.e]
        for c in range(n):
            m = kv[c]
            beta = prob.Bt * sum(prob.w[p] * phi(d, prob.R, math.pi * np.dot(m, e) / prob.L)
                                 * psi(d, prob.R, math.pi * lperp[p] / prob.L) for p, e in enumerate(prob.e))
            k = tuple(int(x) for x in ((l + m + N // 2) % N - N // 2))
            out[idx[k]] += (beta - Gm[a]) * gh[a] * fh[c]
    return out.reshape(ghat.shape)
