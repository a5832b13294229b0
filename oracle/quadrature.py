"""FP64 quadrature rules for the separated collision quadrature (oracle side).

TEST INFRASTRUCTURE ONLY: this package is the slow, plain reference the CUDA
path is checked against.  Only tests, the smoke check and the CPU-baseline leg
of the benchmark may import it; the product library never does.

Rules (the paper cites the general-kernel fast spectral method of its Sec. 2.1
without printing it; the separated form needs a radial rule on [0, R] and a
direction rule on S^{d-1}):
  * radial: N_rho-point Gauss-Legendre on [0, R], roots by Newton's method on
    the Legendre three-term recurrence (a textbook method);
  * 2D directions: uniform circle rule theta_p = 2 pi p / M, w_p = 2 pi / M;
  * 3D directions: octahedrally symmetric (Lebedev-type) rules with 6, 14, 26,
    38, 50 or 86 points, DERIVED here by solving the moment equations
    sum_i w_i x^a y^b z^c = int_{S^2} x^a y^b z^c for every monomial up to the
    design degree (variable projection: weights by linear least squares, orbit
    parameters by Gauss-Newton).  No table is copied; exactness is verified.
"""
from __future__ import annotations

import math
from functools import lru_cache
from itertools import permutations, product

import numpy as np


# --------------------------------------------------------------------------
# Gauss-Legendre
# --------------------------------------------------------------------------

def gauss_legendre(n: int):
    """Nodes/weights of the n-point Gauss-Legendre rule on [-1, 1] (ascending)."""
    if n < 1:
        raise ValueError("n >= 1")
    i = np.arange(n, dtype=np.float64)
    x = np.cos(math.pi * (i + 0.75) / (n + 0.5))      # initial guesses
    for _ in range(200):
        p_prev = np.ones_like(x)
        p = x.copy()
        for k in range(2, n + 1):
            p_prev, p = p, ((2 * k - 1) * x * p - (k - 1) * p_prev) / k
        if n == 1:
            p_prev, p = np.ones_like(x), x.copy()
        dp = n * (x * p - p_prev) / (x * x - 1.0)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-15:
            break
    # final derivative at converged roots
    p_prev = np.ones_like(x)
    p = x.copy()
    for k in range(2, n + 1):
        p_prev, p = p, ((2 * k - 1) * x * p - (k - 1) * p_prev) / k
    if n == 1:
        p_prev = np.ones_like(x)
    dp = n * (x * p - p_prev) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def radial_rule(n_rho: int, R: float):
    """Gauss-Legendre on [0, R]: rho_q = R (x_q + 1)/2, w_q = R w/2."""
    x, w = gauss_legendre(n_rho)
    return 0.5 * R * (x + 1.0), 0.5 * R * w


# --------------------------------------------------------------------------
# Circle
# --------------------------------------------------------------------------

def circle_rule(M: int):
    """theta_p = 2 pi p / M; exact for trigonometric polynomials of degree < M."""
    th = 2.0 * math.pi * np.arange(M) / M
    return np.stack([np.cos(th), np.sin(th)], axis=1), np.full(M, 2.0 * math.pi / M)


# --------------------------------------------------------------------------
# Sphere
# --------------------------------------------------------------------------

def sphere_monomial_integral(a: int, b: int, c: int) -> float:
    """int_{S^2} x^a y^b z^c dsigma (zero unless all exponents are even)."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    g = math.gamma
    return 2.0 * g((a + 1) / 2) * g((b + 1) / 2) * g((c + 1) / 2) / g((a + b + c + 3) / 2)


def _signed_perms(base):
    pts = set()
    for perm in permutations(base):
        for signs in product((1, -1), repeat=3):
            pts.add(tuple(s * x for s, x in zip(signs, perm)))
    return np.array(sorted(pts), dtype=np.float64)


def _orbit(kind: str, param: float | None = None) -> np.ndarray:
    s2, s3 = 1.0 / math.sqrt(2.0), 1.0 / math.sqrt(3.0)
    if kind == "a1":
        return _signed_perms((1.0, 0.0, 0.0))
    if kind == "a2":
        return _signed_perms((0.0, s2, s2))
    if kind == "a3":
        return _signed_perms((s3, s3, s3))
    if kind == "b":          # (l, l, m), 2 l^2 + m^2 = 1
        m = math.sqrt(max(0.0, 1.0 - 2.0 * param * param))
        return _signed_perms((param, param, m))
    if kind == "c":          # (p, q, 0), p^2 + q^2 = 1
        q = math.sqrt(max(0.0, 1.0 - param * param))
        return _signed_perms((param, q, 0.0))
    raise ValueError(kind)


# orbit structure and design degree of each supported rule
SPHERE_RULES = {
    6: (("a1",), 3),
    14: (("a1", "a3"), 5),
    26: (("a1", "a2", "a3"), 7),
    38: (("a1", "a3", "c"), 9),
    50: (("a1", "a2", "a3", "b"), 11),
    86: (("a1", "a3", "b", "b", "c"), 15),
}


def _even_exponents(degree):
    return np.array([(a, b, c) for a in range(0, degree + 1, 2) for b in range(0, degree + 1, 2)
                     for c in range(0, degree + 1, 2) if a + b + c <= degree], dtype=np.float64)


def _moment_system(orbits, params, degree):
    """Rows: monomials of even exponents with total degree <= degree; columns:
    orbits (sum of the monomial over the orbit's points)."""
    exps = _even_exponents(degree)
    pts = []
    it = iter(params)
    for kind in orbits:
        pts.append(_orbit(kind, next(it) if kind in ("b", "c") else None))
    cols = []
    for P in pts:
        mono = (P[:, None, 0] ** exps[None, :, 0]) * (P[:, None, 1] ** exps[None, :, 1]) \
            * (P[:, None, 2] ** exps[None, :, 2])
        cols.append(mono.sum(axis=0))
    A = np.stack(cols, axis=1)
    rhs = np.array([sphere_monomial_integral(*map(int, e)) for e in exps])
    return A, rhs, pts


def _residual(orbits, params, degree):
    A, rhs, _ = _moment_system(orbits, params, degree)
    w, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    return A @ w - rhs, w


@lru_cache(maxsize=None)
def sphere_rule(M: int):
    """Octahedrally symmetric rule with M points on S^2: (sigma [M,3], w [M]).
    Weights sum to 4 pi; the rule is centrally symmetric."""
    if M not in SPHERE_RULES:
        raise ValueError(f"unsupported sphere rule size {M}")
    orbits, degree = SPHERE_RULES[M]
    n_par = sum(k in ("b", "c") for k in orbits)
    limits = [(1e-3, 1.0 / math.sqrt(2.0) - 1e-3) for _ in range(n_par)]
    best = None
    if n_par == 0:
        params = ()
    else:
        # coarse scan of the orbit parameters, then Gauss-Newton refinement
        grids = [np.linspace(lo, hi, 17 if n_par > 1 else 200) for lo, hi in limits]
        cands = []
        for pt in product(*grids):
            if n_par > 1 and not all(pt[i] < pt[i + 1] for i in range(n_par - 2)):
                continue    # the two b-orbits are ordered l1 < l2
            r, _ = _residual(orbits, pt, degree)
            cands.append((float(np.dot(r, r)), pt))
        cands.sort(key=lambda t: t[0])
        for _, start in cands[:40]:
            p = np.array(start, dtype=np.float64)
            for _ in range(100):
                r, _ = _residual(orbits, p, degree)
                J = np.empty((r.size, n_par))
                for k in range(n_par):
                    h = 1e-7
                    dp = p.copy(); dp[k] += h
                    dm = p.copy(); dm[k] -= h
                    J[:, k] = (_residual(orbits, dp, degree)[0] - _residual(orbits, dm, degree)[0]) / (2 * h)
                step, *_ = np.linalg.lstsq(J, -r, rcond=None)
                p = p + step
                if np.max(np.abs(step)) < 1e-15:
                    break
            r, w = _residual(orbits, p, degree)
            if (np.max(np.abs(r)) < 1e-12 and np.all(w > 0)
                    and all(lo < x < hi for x, (lo, hi) in zip(p, limits))):
                best = tuple(float(x) for x in p)
                break
        if best is None:
            raise RuntimeError(f"sphere rule {M}: moment equations not solved")
        params = best
    A, rhs, pts = _moment_system(orbits, params, degree)
    w, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    sig = np.concatenate(pts, axis=0)
    wts = np.concatenate([np.full(P.shape[0], w[i]) for i, P in enumerate(pts)])
    if sig.shape[0] != M:
        raise RuntimeError("orbit sizes do not add up")
    return sig, wts


def sphere_rule_degree(M: int) -> int:
    return SPHERE_RULES[M][1]


def product_sphere_rule(n_theta: int, n_phi: int):
    """Gauss-Legendre in cos(theta) x uniform in phi: exact for polynomials of
    degree <= min(2 n_theta - 1, n_phi - 1).  Used for fine reference
    quadratures, not by the method."""
    x, wx = gauss_legendre(n_theta)
    phi = 2.0 * math.pi * np.arange(n_phi) / n_phi
    st = np.sqrt(1.0 - x * x)
    X = (st[:, None] * np.cos(phi)[None, :]).ravel()
    Y = (st[:, None] * np.sin(phi)[None, :]).ravel()
    Z = np.repeat(x, n_phi)
    W = np.repeat(wx, n_phi) * (2.0 * math.pi / n_phi)
    return np.stack([X, Y, Z], axis=1), W


def direction_rule(d: int, M: int):
    """The method's direction rule: circle (d=2) or octahedral sphere rule (d=3)."""
    if d == 2:
        if M % 2:
            raise ValueError("2D direction count must be even (central symmetry)")
        return circle_rule(M)
    if d == 3:
        return sphere_rule(M)
    raise ValueError("d must be 2 or 3")


def antipode_index(sigma: np.ndarray) -> np.ndarray:
    """Index of -sigma_p in the rule (rules here are centrally symmetric)."""
    M = sigma.shape[0]
    out = np.empty(M, dtype=np.int64)
    for p in range(M):
        dist = np.max(np.abs(sigma + sigma[p]), axis=1)
        out[p] = int(np.argmin(dist))
        if dist[out[p]] > 1e-12:
            raise ValueError("rule is not centrally symmetric")
    return out
