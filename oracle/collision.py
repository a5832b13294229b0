"""Plain FP64 CPU oracle of the separated fast-spectral collision operator.

TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference the
CUDA library is checked against.  Only tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does, and
the two share no code.

What is computed (paper Sec. 1, eqs. "eqn:collision_operator" and
"eqn:collision velocity"; Sec. 2.1 states the discrete-velocity interface and
cites the general-kernel fast spectral algorithm without printing it):

    Q(g,f)(v) = int_{|q|<=R} int_{S^{d-1}} b |q|^gamma
                [ g(v'_*) f(v') - g(v-q) f(v) ] dsigma dq,
    v'  = v - q/2 + |q| sigma / 2,   v'_* = v - q/2 - |q| sigma / 2,

with g, f replaced by their trigonometric interpolants on the periodised grid
[-L, L]^d (v_j = -L + j dv, dv = 2L/N) and the integrals by the separated
quadrature: Gauss-Legendre radial nodes (rho_q, w_q) on [0, R] times the
direction rule (sigma_p, w_p).  Writing q = rho * omega, the omega-integral of
exp(-i pi rho k.omega / (2L)) is done exactly, F_3(s) = 4 pi sin(s)/s,
F_2(s) = 2 pi J0(s).  Steps, in the order the method takes them:

  1. spectra   fhat_k = n^-1 sum_j f(v_j) exp(-i pi k.v_j / L), Nyquist zeroed
  2. quadrature (oracle.quadrature)
  3. shifted fields A_{q,p} = g_N(v - rho_q sigma_p/2), B_{q,p} = f_N(v + rho_q sigma_p/2)
  4. sigma-accumulate P_q = sum_p w_p A_{q,p} B_{q,p}
  5. Qhat+_k = sum_q b w_q rho_q^{gamma+d-1} F_d(pi rho_q |k| / (2L)) DFT[P_q]_k
  6. loss: Lambda_g = sum_l G-(l) ghat_l e^{i pi l.v/L},
     G-(l) = b |S^{d-1}| sum_q w_q rho_q^{gamma+d-1} F_d(pi rho_q |l| / L);
     Q- = f_N * Lambda_g.  Option loss="mass_consistent": the sigma-average
     taken with the gain's own direction rule instead of exactly,
     G-(l) = b F_d(0) sum_q w_q rho_q^{gamma+d-1} sum_p w_p e^{-i pi rho_q l.sigma_p / L}
           = G_sep(l, -l), so that Qhat_0 (the mass of Q) vanishes to rounding
  7. Q = Re IDFT(Qhat+) - Q-
  8. projection T_kjl = dv^d sum_v V_k(v) Q_jl(v) (midpoint rule, Sec. 2.4)
  9. direct sum (tiny grids): Qhat_k = sum_{l+m = k mod N} [G_sep(l,m) - G-(l)] ghat_l fhat_m

Conventions where the paper is silent (each is a stated reading): kernel
constant b = 1/|S^{d-1}| unless given; grid includes -L; wrapped (mod N)
convolution; Nyquist modes of the inputs zeroed, output modes all kept.
All arithmetic is FP64; every transform is a plain separable direct sum
(one dense matrix per axis) with exactly reduced angles, no FFT.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import j0 as _bessel_j0

from . import quadrature as quad


def sphere_area(d: int) -> float:
    return 2.0 * math.pi if d == 2 else 4.0 * math.pi


def F_d(d: int, s):
    """Exact omega-average kernel: int_{S^{d-1}} exp(-i s.omega) domega for |s| = s."""
    s = np.asarray(s, dtype=np.float64)
    if d == 3:
        return 4.0 * math.pi * np.sinc(s / math.pi)       # sin(s)/s, = 1 at 0
    if d == 2:
        return 2.0 * math.pi * _bessel_j0(s)
    raise ValueError("d must be 2 or 3")


@dataclass
class Problem:
    """One velocity grid plus the separated quadrature (Sec. 2.1 interface)."""
    N: int
    d: int
    L: float
    R: float
    gamma: float
    n_rho: int = 0
    M: int = 0
    b: float | None = None
    loss: str = "exact"
    rho: np.ndarray | None = None
    w_rho: np.ndarray | None = None
    sigma: np.ndarray | None = None
    w_sigma: np.ndarray | None = None
    _cache: dict = field(default_factory=dict, repr=False)

    def __post_init__(self):
        if self.N % 2:
            raise ValueError("N must be even")
        if self.loss not in ("exact", "mass_consistent"):
            raise ValueError("loss must be 'exact' or 'mass_consistent'")
        if self.b is None:
            self.b = 1.0 / sphere_area(self.d)
        if self.rho is None:
            self.rho, self.w_rho = quad.radial_rule(self.n_rho, self.R)
        if self.sigma is None:
            self.sigma, self.w_sigma = quad.direction_rule(self.d, self.M)
        self.n_rho = len(self.rho)
        self.M = len(self.w_sigma)

    @property
    def n(self) -> int:
        return self.N ** self.d

    @property
    def dv(self) -> float:
        return 2.0 * self.L / self.N

    @property
    def shape(self):
        return (self.N,) * self.d


# --------------------------------------------------------------------------
# frequencies and per-axis transform matrices
# --------------------------------------------------------------------------

def freq_of_index(N: int) -> np.ndarray:
    """Integer frequency of each DFT index: 0..N/2-1, then -N/2..-1."""
    i = np.arange(N)
    return np.where(i < N // 2, i, i - N)


def _analysis_matrix(N: int) -> np.ndarray:
    """E[k, j] = n_axis^-1 exp(-i pi k v_j / L).  With v_j = -L + 2Lj/N the angle
    is 2 pi (k j - k N/2)/N, reduced exactly in integers before cos/sin."""
    k = freq_of_index(N)[:, None]
    j = np.arange(N)[None, :]
    m = np.mod(k * j - k * (N // 2), N)
    return np.exp(-2j * math.pi * m / N) / N


def _synthesis_matrix(N: int, L: float, shift: float) -> np.ndarray:
    """S[j, k] = exp(i pi k (v_j - shift) / L): evaluates the trigonometric
    interpolant at the grid points moved by -shift."""
    k = freq_of_index(N)[None, :]
    j = np.arange(N)[:, None]
    m = np.mod(k * j - k * (N // 2), N)
    return np.exp(2j * math.pi * m / N) * np.exp(-1j * math.pi * k * shift / L)


def _apply_axis(F: np.ndarray, mat: np.ndarray, axis: int) -> np.ndarray:
    return np.moveaxis(np.tensordot(mat, F, axes=([1], [axis])), 0, axis)


def dft(prob: Problem, f: np.ndarray) -> np.ndarray:
    """Full spectrum (all modes) of real/complex fields f[..., N,...,N] (step 1 / 5)."""
    E = _analysis_matrix(prob.N)
    F = np.asarray(f, dtype=np.complex128)
    nb = F.ndim - prob.d
    for a in range(prob.d):
        F = _apply_axis(F, E, nb + a)
    return F


def zero_nyquist(prob: Problem, F: np.ndarray) -> np.ndarray:
    F = F.copy()
    nb = F.ndim - prob.d
    for a in range(prob.d):
        idx = [slice(None)] * F.ndim
        idx[nb + a] = prob.N // 2
        F[tuple(idx)] = 0.0
    return F


def spectrum(prob: Problem, f: np.ndarray) -> np.ndarray:
    """Input spectra: fhat_k = n^-1 sum_j f(v_j) e^{-i pi k.v_j/L}, Nyquist zeroed."""
    return zero_nyquist(prob, dft(prob, f))


def synthesize(prob: Problem, F: np.ndarray, shift=None, return_imag=False):
    """sum_k F_k exp(i pi k.(v_j - shift)/L) at every grid point (step 3 / 7)."""
    shift = np.zeros(prob.d) if shift is None else np.asarray(shift, dtype=np.float64)
    G = np.asarray(F, dtype=np.complex128)
    nb = G.ndim - prob.d
    for a in range(prob.d):
        G = _apply_axis(G, _synthesis_matrix(prob.N, prob.L, float(shift[a])), nb + a)
    if return_imag:
        return G.real, float(np.max(np.abs(G.imag))) if G.size else 0.0
    return G.real


def kabs(prob: Problem) -> np.ndarray:
    """|k| of the wrapped frequency at every spectral index."""
    k = freq_of_index(prob.N).astype(np.float64)
    K = np.meshgrid(*([k] * prob.d), indexing="ij")
    return np.sqrt(sum(x * x for x in K))


def kernel_power(prob: Problem) -> float:
    """Exponent of rho in the radial integrand: |q|^gamma times the Jacobian rho^{d-1}."""
    return prob.gamma + prob.d - 1


def gain_shifts(prob: Problem, q: int, p: int):
    """Shifts of the g-side and f-side fields at node (q, p): v'_* = v - rho sigma/2
    and v' = v + rho sigma/2 once the q/2 part has gone into the omega-average."""
    s = 0.5 * prob.rho[q] * prob.sigma[p]
    return +s, -s


def radial_multiplier(prob: Problem, kmag: np.ndarray) -> np.ndarray:
    """c_q(|k|) = b w_q rho_q^{gamma+d-1} F_d(pi rho_q |k| / (2L)), shape [n_rho, ...]."""
    out = np.empty((prob.n_rho,) + kmag.shape)
    for q in range(prob.n_rho):
        out[q] = (prob.b * prob.w_rho[q] * prob.rho[q] ** kernel_power(prob)
                  * F_d(prob.d, math.pi * prob.rho[q] * kmag / (2.0 * prob.L)))
    return out


def loss_weight(prob: Problem, kmag: np.ndarray) -> np.ndarray:
    """G-(l) = b |S^{d-1}| sum_q w_q rho_q^{gamma+d-1} F_d(pi rho_q |l| / L)."""
    acc = np.zeros(kmag.shape)
    for q in range(prob.n_rho):
        acc += prob.w_rho[q] * prob.rho[q] ** kernel_power(prob) \
            * F_d(prob.d, math.pi * prob.rho[q] * kmag / prob.L)
    return prob.b * sphere_area(prob.d) * acc


def loss_weight_mass_consistent(prob: Problem, lvec: np.ndarray) -> np.ndarray:
    """G-(l) = G_sep(l, -l) = b F_d(0) sum_q w_q rho_q^{gamma+d-1} sum_p w_p
    exp(-i pi rho_q l.sigma_p / L) for integer frequency vectors l [..., d]:
    the gain's separated kernel at m = -l, where |l + m| = 0.  The direction
    rules are centrally symmetric, so the sum is real (its cosine part)."""
    lv = np.asarray(lvec, dtype=np.float64)
    acc = np.zeros(lv.shape[:-1])
    for q in range(prob.n_rho):
        sig = np.zeros(lv.shape[:-1])
        for p in range(prob.M):
            sig += prob.w_sigma[p] * np.cos(math.pi * prob.rho[q] * (lv @ prob.sigma[p]) / prob.L)
        acc += prob.w_rho[q] * prob.rho[q] ** kernel_power(prob) * sig
    return prob.b * float(F_d(prob.d, 0.0)) * acc


def freq_vectors(prob: Problem) -> np.ndarray:
    """Integer frequency vector of every spectral index, shape [N]*d + [d]."""
    fr = freq_of_index(prob.N)
    return np.stack(np.meshgrid(*([fr] * prob.d), indexing="ij"), axis=-1)


def loss_table(prob: Problem) -> np.ndarray:
    """G-(l) at every spectral index, for the loss reading the problem names."""
    if prob.loss == "mass_consistent":
        return loss_weight_mass_consistent(prob, freq_vectors(prob))
    return loss_weight(prob, kabs(prob))


# --------------------------------------------------------------------------
# the collision operator
# --------------------------------------------------------------------------

def loss_field(fN: np.ndarray, lam: np.ndarray, jj, ll) -> np.ndarray:
    """Q-(g,f) = f_N(v) * Lambda_g(v): f of the pair's second slot times the
    g-side loss field of its first slot."""
    return fN[ll] * lam[jj]


def collide(prob: Problem, spec: np.ndarray, pairs, return_parts: bool = False):
    """Q(g,f) for every (j, l) in `pairs`: g = input j, f = input l.

    spec: full input spectra [n_inputs][N]*d (from `spectrum`).
    Returns Q [n_pairs][N]*d (and, if asked, the gain Q+ and loss Q- fields).
    """
    pairs = [(int(j), int(l)) for j, l in pairs]
    used = sorted({i for pr in pairs for i in pr})
    slot = {i: s for s, i in enumerate(used)}
    S = spec[used]
    jj = np.array([slot[j] for j, _ in pairs], dtype=np.int64)
    ll = np.array([slot[l] for _, l in pairs], dtype=np.int64)
    n_pairs = len(pairs)
    kmag = kabs(prob)
    cq = radial_multiplier(prob, kmag)
    Qhat_plus = np.zeros((n_pairs,) + prob.shape, dtype=np.complex128)
    for q in range(prob.n_rho):
        P = np.zeros((n_pairs,) + prob.shape)
        for p in range(prob.M):
            sA, sB = gain_shifts(prob, q, p)
            A = synthesize(prob, S, sA)          # g_N(v - rho sigma / 2)
            B = synthesize(prob, S, sB)          # f_N(v + rho sigma / 2)
            P += prob.w_sigma[p] * A[jj] * B[ll]
        Qhat_plus += cq[q][None] * dft(prob, P)
    Q_plus = synthesize(prob, Qhat_plus)
    Gm = loss_table(prob)
    lam = synthesize(prob, Gm[None] * S)          # Lambda_g for every used input
    fN = synthesize(prob, S)                      # f_N on the grid
    Q_minus = loss_field(fN, lam, jj, ll)
    Q = Q_plus - Q_minus
    if return_parts:
        return Q, Q_plus, Q_minus
    return Q


def collide_fields(prob: Problem, fields: np.ndarray, pairs, return_parts: bool = False):
    """Convenience: physical inputs -> spectra -> Q."""
    return collide(prob, spectrum(prob, fields), pairs, return_parts)


def scale(Q, Q_plus, Q_minus) -> np.ndarray:
    """Per-result error scale s = max(max|Q|, max|Q+|, max|Q-|)."""
    ax = tuple(range(1, np.ndim(Q)))
    return np.maximum(np.maximum(np.max(np.abs(Q), axis=ax), np.max(np.abs(Q_plus), axis=ax)),
                      np.max(np.abs(Q_minus), axis=ax))


def project(prob: Problem, V: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """T[k, p] = dv^d sum_v V_k(v) Q_p(v): the r^3 tensor <V_k, Q(V_j,V_l)>_v
    (Sec. 2.4, midpoint rule) with p = j*r + l."""
    r = V.shape[0]
    return prob.dv ** prob.d * V.reshape(r, -1) @ Q.reshape(Q.shape[0], -1).T


def velocity_axis(prob: Problem) -> np.ndarray:
    """Grid points of one velocity axis, v_j = -L + j dv (Sec. 2.1 uniform grid)."""
    return -prob.L + np.arange(prob.N) * prob.dv


def cell_volume(prob: Problem) -> float:
    """Weight of one grid point in the midpoint rule for int dv (Sec. 2.4): dv^d."""
    return prob.dv ** prob.d


def moments(prob: Problem, Q: np.ndarray) -> np.ndarray:
    """dv^d sum_v Q(v) {1, v_0..v_{d-1}, |v|^2} for each result (Sec. 1)."""
    ax = velocity_axis(prob)
    V = np.meshgrid(*([ax] * prob.d), indexing="ij")
    phis = [np.ones(prob.shape)] + list(V) + [sum(x * x for x in V)]
    Qf = Q.reshape(-1, *prob.shape)
    return np.stack([[cell_volume(prob) * np.sum(qq * ph) for ph in phis] for qq in Qf])


# --------------------------------------------------------------------------
# step 9: brute-force direct sum on tiny grids
# --------------------------------------------------------------------------

def direct_sum(prob: Problem, ghat: np.ndarray, fhat: np.ndarray) -> np.ndarray:
    """Qhat_k = sum_{l+m = k (mod N)} [G_sep(l,m) - G-(l)] ghat_l fhat_m, with
    G_sep(l,m) = sum_q b w_q rho_q^{gamma+d-1} F_d(pi rho_q |k_w| / (2L))
                 * sum_p w_p exp(-i pi rho_q (l-m).sigma_p / (2L)),
    k_w the wrapped representative of l+m.  O(n^2 N_rho M)."""
    N, d = prob.N, prob.d
    fr = freq_of_index(N)
    grids = np.meshgrid(*([fr] * d), indexing="ij")
    lv = np.stack([g.ravel() for g in grids], axis=1)                 # [n, d]
    n = lv.shape[0]
    diff = lv[:, None, :] - lv[None, :, :]                             # l - m
    ssum = lv[:, None, :] + lv[None, :, :]                             # l + m
    kw = np.mod(ssum + N // 2, N) - N // 2                             # wrapped
    kw_abs = np.sqrt(np.sum(kw.astype(np.float64) ** 2, axis=-1))
    G = np.zeros((n, n), dtype=np.complex128)
    for q in range(prob.n_rho):
        H = np.zeros((n, n), dtype=np.complex128)
        for p in range(prob.M):
            H += prob.w_sigma[p] * np.exp(
                -1j * math.pi * prob.rho[q] * (diff @ prob.sigma[p]) / (2.0 * prob.L))
        G += (prob.b * prob.w_rho[q] * prob.rho[q] ** kernel_power(prob)
              * F_d(d, math.pi * prob.rho[q] * kw_abs / (2.0 * prob.L))) * H
    if prob.loss == "mass_consistent":
        G -= loss_weight_mass_consistent(prob, lv)[:, None]
    else:
        labs = np.sqrt(np.sum(lv.astype(np.float64) ** 2, axis=1))
        G -= loss_weight(prob, labs)[:, None]
    gl = ghat.reshape(-1)
    fm = fhat.reshape(-1)
    contrib = G * gl[:, None] * fm[None, :]
    # scatter-add into the wrapped target index
    kidx = np.zeros((n, n), dtype=np.int64)
    for a in range(d):
        kidx = kidx * N + np.mod(ssum[..., a], N)
    out = np.zeros(n, dtype=np.complex128)
    np.add.at(out, kidx.ravel(), contrib.ravel())
    return out.reshape(prob.shape)
