"""FP64 oracle of the Mott-Smith strong-shock closure (paper Sec. 4.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The bimodal ansatz f(x_1, v) = a(x_1) f_L(v) + (1 - a(x_1)) f_R(v) with the
v_1^2 moment of the shock equation gives
    alpha = int v_1^2 ( Q(f_L, f_R) + Q(f_R, f_L) ) dv          (eq. "eqn:alpha")
    beta  = alpha / ( (d - 1) rho_L u_L R (T_L - T_R) ),
    a(x_1) = 1 / (exp(beta x_1) + 1),
    rho(x_1) / rho_L = (1 + (d+1) M^2 / (M^2 + d) exp(beta x_1)) / (1 + exp(beta x_1)).
The shock drifts along velocity axis 0 (v_1); the integral is the midpoint
rule on the collision grid.
"""
from __future__ import annotations

import math

import numpy as np

from . import collision as C


def axis0_second_moment(prob: C.Problem, Q: np.ndarray) -> np.ndarray:
    """dv^d sum_v v_1^2 Q_f(v) for every field f of Q [n][N]^d."""
    dv = 2.0 * prob.L / prob.N
    v1 = -prob.L + np.arange(prob.N) * dv
    shape = (prob.N,) + (1,) * (prob.d - 1)
    w = (v1 ** 2).reshape(shape)
    Q = np.asarray(Q, dtype=np.float64)
    return dv ** prob.d * np.sum(Q * w[None], axis=tuple(range(1, Q.ndim)))


def alpha(prob: C.Problem, fL: np.ndarray, fR: np.ndarray) -> float:
    Q = C.collide_fields(prob, np.stack([fL, fR]), [(0, 1), (1, 0)])
    m = axis0_second_moment(prob, Q)
    return float(m[0] + m[1])


def beta(alpha_value: float, d: int, rho_L: float, u_L: float, T_L: float, T_R: float, R_gas: float = 1.0) -> float:
    return alpha_value / ((d - 1) * rho_L * u_L * R_gas * (T_L - T_R))


def profile_a(x, beta_value: float):
    return 1.0 / (np.exp(beta_value * np.asarray(x, dtype=np.float64)) + 1.0)


def density_ratio(x, beta_value: float, d: int, mach: float):
    e = np.exp(beta_value * np.asarray(x, dtype=np.float64))
    return (1.0 + (d + 1) * mach ** 2 / (mach ** 2 + d) * e) / (1.0 + e)
