"""Pins of the oracle's quadrature rules (CPU).  Each rule is checked against
closed-form integrals, a library routine, or its design degree."""
import math
import os

import numpy as np
import pytest

from oracle import collision as C
from oracle import quadrature as Q

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [1, 2, 5, 16, 32, 48])
def test_gauss_legendre_matches_numpy(n):
    x, w = Q.gauss_legendre(n)
    x2, w2 = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - x2)) < 1e-14
    assert np.max(np.abs(w - w2)) < 1e-14


@pytest.mark.parametrize("n", [4, 16, 32])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = Q.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13
    # at degree 2n the error is the textbook constant 2^{2n+1}(n!)^4/((2n+1)((2n)!)^2)
    c_n = 2.0 ** (2 * n + 1) * math.factorial(n) ** 4 / ((2 * n + 1) * math.factorial(2 * n) ** 2)
    err = 2.0 / (2 * n + 1) - np.dot(w, x ** (2 * n))
    if c_n > 1e-10:
        assert abs(err - c_n) < 1e-6 * c_n


def test_radial_rule_on_0_R():
    rho, w = Q.radial_rule(16, 8.0)
    assert np.all((rho > 0) & (rho < 8.0))
    for k in range(31):
        assert abs(np.dot(w, rho ** k) - 8.0 ** (k + 1) / (k + 1)) < 1e-12 * 8.0 ** (k + 1)


@pytest.mark.parametrize("M", [8, 16, 32])
def test_circle_rule_trig_exactness(M):
    sig, w = Q.circle_rule(M)
    th = np.arctan2(sig[:, 1], sig[:, 0])
    assert abs(w.sum() - 2 * math.pi) < 1e-14
    for m in range(1, M):
        assert abs(np.dot(w, np.cos(m * th))) < 1e-13
    assert abs(np.dot(w, np.cos(M * th)) - 2 * math.pi) < 1e-12   # aliasing at degree M


@pytest.mark.parametrize("M", sorted(Q.SPHERE_RULES))
def test_sphere_rule_design_degree(M):
    sig, w = Q.sphere_rule(M)
    deg = Q.sphere_rule_degree(M)
    assert sig.shape == (M, 3)
    assert np.all(w > 0)
    assert abs(w.sum() - 4 * math.pi) < 1e-13
    assert np.max(np.abs(np.sum(sig ** 2, axis=1) - 1)) < 1e-14
    Q.antipode_index(sig)                          # centrally symmetric
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                val = np.dot(w, sig[:, 0] ** a * sig[:, 1] ** b * sig[:, 2] ** c)
                assert abs(val - Q.sphere_monomial_integral(a, b, c)) < 1e-13, (a, b, c)
    # not exact one even degree above the design degree
    d2 = deg + 1 if deg % 2 else deg + 2
    errs = [abs(np.dot(w, sig[:, 0] ** a * sig[:, 1] ** b * sig[:, 2] ** (d2 - a - b))
                - Q.sphere_monomial_integral(a, b, d2 - a - b))
            for a in range(0, d2 + 1, 2) for b in range(0, d2 + 1 - a, 2)]
    assert max(errs) > 1e-6


@pytest.mark.parametrize("M", [38, 86])
def test_sphere_rule_rotated_polynomial(M):
    """Exactness is frame independent: a randomly rotated rule integrates a
    random polynomial of the design degree like a fine product rule does."""
    rng = np.random.default_rng(5)
    sig, w = Q.sphere_rule(M)
    deg = Q.sphere_rule_degree(M)
    Rm, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    ref_s, ref_w = Q.product_sphere_rule(24, 48)
    terms = [(a, b, c, rng.standard_normal()) for a in range(deg + 1)
             for b in range(deg + 1 - a) for c in range(deg + 1 - a - b)]

    def poly(P):
        return sum(cf * P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** c for a, b, c, cf in terms)
    got = np.dot(w, poly(sig @ Rm.T))
    ref = np.dot(ref_w, poly(ref_s))
    assert abs(got - ref) < 1e-11 * max(1.0, abs(ref))


def test_F_d_special_values():
    assert abs(C.F_d(3, 0.0) - 4 * math.pi) < 1e-15
    assert abs(C.F_d(2, 0.0) - 2 * math.pi) < 1e-15
    zeros = [float(x) for x in open(os.path.join(GOLDEN, "bessel_j0_zeros.txt"))
             if x.strip() and not x.startswith("#")]
    for z in zeros:
        assert abs(C.F_d(2, z)) < 1e-13
    assert abs(C.F_d(3, math.pi)) < 1e-14          # sin(pi) = 0


@pytest.mark.parametrize("s", [0.3, 2.0, 7.5, 19.0])
def test_F_d_is_the_direction_average(s):
    """F_d(|s|) = int_S exp(-i s.omega) domega, checked by fine quadrature."""
    th = 2 * math.pi * np.arange(512) / 512
    val2 = np.sum(np.exp(-1j * s * np.cos(th))) * 2 * math.pi / 512
    assert abs(val2 - C.F_d(2, s)) < 1e-12
    sig, w = Q.product_sphere_rule(48, 96)
    val3 = np.dot(w, np.exp(-1j * s * sig[:, 2]))
    assert abs(val3 - C.F_d(3, s)) < 1e-12
