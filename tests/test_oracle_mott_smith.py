"""Pins of the Mott-Smith oracle (paper Sec. 4.2): the bilinear expansion of
the v_1^2 moment of Q(f, f) for the bimodal f, the sign of alpha for a
compressive shock, and the density profile against the Rankine-Hugoniot
mixture."""
import math

import numpy as np

from oracle import collision as C
from oracle import mott_smith as MS
from paper_2112_02695_gb300 import workloads as W


def problem():
    return C.Problem(N=16, d=3, L=8.0, R=8.0, gamma=1.0, n_rho=4, M=14)


def test_moment_of_bimodal_collision_is_a_one_minus_a_alpha():
    prob = problem()
    fL, fR = W.shock_states_fields(16, 3, 8.0)
    al = MS.alpha(prob, fL, fR)
    for a in (0.2, 0.5, 0.9):
        f = a * fL + (1 - a) * fR
        Qf = C.collide_fields(prob, f[None], [(0, 0)])
        QLL, QRR = C.collide_fields(prob, np.stack([fL, fR]), [(0, 0), (1, 1)])
        lhs = MS.axis0_second_moment(prob, Qf)[0]
        self_terms = MS.axis0_second_moment(prob, np.stack([QLL, QRR]))
        rhs = a * a * self_terms[0] + a * (1 - a) * al + (1 - a) ** 2 * self_terms[1]
        assert abs(lhs - rhs) <= 1e-12 * abs(al)
        # Q(M, M) ~ 0: the resolved upstream Maxwellian's own term is small next to the
        # cross term (the hot downstream state needs a finer grid than 16^3 for this)
        assert abs(self_terms[0]) < 0.01 * abs(al)


def test_alpha_negative_beta_positive_for_a_compressive_shock():
    prob = problem()
    (rL, uL, TL), (rR, uR, TR) = W.rankine_hugoniot(3, 3.0)
    fL, fR = W.shock_states_fields(16, 3, 8.0)
    al = MS.alpha(prob, fL, fR)
    be = MS.beta(al, 3, rL, uL, TL, TR)
    assert al < 0 and be > 0
    assert MS.profile_a(-50.0, be) > 0.999 and MS.profile_a(50.0, be) < 1e-3   # upstream at -inf


def test_density_profile_is_the_rankine_hugoniot_mixture():
    (rL, uL, TL), (rR, uR, TR) = W.rankine_hugoniot(3, 3.0)
    x = np.linspace(-5, 5, 11)
    be = 0.7
    a = MS.profile_a(x, be)
    assert np.allclose(MS.density_ratio(x, be, 3, 3.0), (a * rL + (1 - a) * rR) / rL, rtol=1e-14)
    assert math.isclose(rR / rL, 4 * 9 / 12)
