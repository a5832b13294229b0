"""Independent physical-space quadrature of the collision integral.

Evaluates the paper's definition (Sec. 1, eqs. "eqn:collision_operator" and
"eqn:collision velocity") directly, with v_* = v - q, q = rho*omega:

  Q(g,f)(v) = int_0^R rho^{d-1} b rho^gamma int_S int_S
              [g(v - q/2 - rho sigma/2) f(v - q/2 + rho sigma/2) - g(v - q) f(v)]
              dsigma domega drho

for analytic callables g, f (no grid, no periodisation, no Fourier series),
using fine product rules: Gauss-Legendre in rho, trapezoid on the circle or
Gauss x trapezoid on the sphere for omega and sigma.  It shares the oracle's
quadrature helpers only for node generation (Gauss-Legendre and the product
sphere rule), which are pinned on their own.  Used only to pin the oracle.
"""
import math

import numpy as np

from oracle.quadrature import gauss_legendre, product_sphere_rule


def _dirs(d, n):
    if d == 2:
        th = 2 * math.pi * np.arange(n) / n
        return np.stack([np.cos(th), np.sin(th)], 1), np.full(n, 2 * math.pi / n)
    return product_sphere_rule(n, 2 * n)


def q_physical(g, f, v, d, R, gamma, b, n_rho=48, n_dir=64):
    """Gain, loss and Q at one velocity v (FP64)."""
    x, wx = gauss_legendre(n_rho)
    rho = 0.5 * R * (x + 1)
    wr = 0.5 * R * wx
    om, wo = _dirs(d, n_dir)
    sg, ws = _dirs(d, n_dir)
    v = np.asarray(v, dtype=np.float64)
    gain = 0.0
    loss = 0.0
    area = 2 * math.pi if d == 2 else 4 * math.pi
    for q in range(n_rho):
        kern = b * rho[q] ** (gamma + d - 1) * wr[q]
        qv = rho[q] * om                               # [n_om, d]
        base = v[None, :] - 0.5 * qv                   # v - q/2
        vs = base[:, None, :] - 0.5 * rho[q] * sg[None, :, :]   # v'_*
        vp = base[:, None, :] + 0.5 * rho[q] * sg[None, :, :]   # v'
        val = g(vs.reshape(-1, d)) * f(vp.reshape(-1, d))
        gain += kern * np.sum(val.reshape(len(wo), len(ws)) * wo[:, None] * ws[None, :])
        loss += kern * area * np.sum(wo * g(v[None, :] - qv))
    loss *= f(v[None, :])[0]
    return gain, loss, gain - loss


def maxwellian_fn(rho, u, T):
    u = np.asarray(u, dtype=np.float64)
    d = u.size

    def fn(x):
        r2 = np.sum((x - u[None, :]) ** 2, axis=1)
        return rho * (2 * math.pi * T) ** (-d / 2) * np.exp(-r2 / (2 * T))
    return fn
