"""Pins of the Carleman-form oracle (oracle/carleman.py, gamma = d - 2):
the 2D BKW closed form for Maxwell molecules, the brute-force direct sum,
the closed forms of phi and psi against numerical quadrature of their
defining integrals, exact mass conservation, Q(M, M) ~ 0, and agreement with
the separated form of oracle/collision.py on well-resolved data."""
import math

import numpy as np
from scipy import integrate
from scipy.special import j0

from oracle import carleman as CM
from oracle import collision as C
from paper_2112_02695_gb300 import workloads as W
from test_oracle_collision import _bkw_dt


def test_bkw_2d_maxwell_closed_form():
    """2D Maxwell molecules, b = 1/(2 pi): Q(f, f) = d/dt f_BKW."""
    prob = CM.CarlemanProblem(N=64, d=2, L=8.0, R=6.0, M=64)
    f = W.bkw(64, 2, 8.0, 0.5)
    Q = CM.collide_fields(prob, f[None], [(0, 0)])[0]
    ex = _bkw_dt(64, 2, 8.0, 0.5)
    assert np.max(np.abs(Q - ex)) / np.abs(ex).max() < 1e-7


def test_closed_forms_against_quadrature():
    R = 3.0
    for s in (0.0, 0.7, 2.3):
        for d in (2, 3):
            num = integrate.quad(lambda r: abs(r) ** (d - 2) * math.cos(r * s), -R, R, limit=200)[0]
            assert abs(CM.phi(d, R, s) - num) < 1e-10
        # d = 2: a segment of half-length R; d = 3: a disk of radius R
        num2 = integrate.quad(lambda y: math.cos(y * s), -R, R)[0]
        assert abs(CM.psi(2, R, s) - num2) < 1e-10
        num3 = 2 * math.pi * integrate.quad(lambda r: r * j0(r * s), 0, R)[0]
        assert abs(CM.psi(3, R, s) - num3) < 1e-10


def test_direct_sum_matches_the_fft_form():
    for N, d, M in [(8, 2, 8), (4, 3, 14)]:
        prob = CM.CarlemanProblem(N=N, d=d, L=4.0, R=3.0, M=M)
        rng = np.random.default_rng(N + d)
        g, f = rng.standard_normal((2,) + prob.shape)
        S = C.spectrum(prob.grid, np.stack([g, f]))
        Q = CM.collide(prob, S, [(0, 1)])[0]
        Qd = CM.direct_sum(prob, S[0], S[1])
        assert np.max(np.abs(C.dft(prob.grid, Q) - Qd)) <= 1e-12 * np.max(np.abs(Qd))


def test_mass_exact_and_maxwellian_equilibrium_3d():
    prob = CM.CarlemanProblem(N=16, d=3, L=8.0, R=5.0, M=38)
    rng = np.random.default_rng(3)
    F = np.abs(rng.standard_normal((2,) + prob.shape))
    Q = CM.collide_fields(prob, F, [(0, 1), (1, 0)])
    assert np.max(np.abs(Q.reshape(2, -1).sum(axis=1))) < 1e-12 * np.max(np.abs(Q)) * Q[0].size
    M = W.maxwellian(16, 3, 8.0, 1.0, np.array([0.5, 0.0, -0.3]), 1.0)
    Qm, Qp, _ = CM.collide_fields(prob, M[None], [(0, 0)], return_parts=True)
    assert np.max(np.abs(Qm)) < 1e-2 * np.max(np.abs(Qp))     # spectral accuracy at 16^3


def test_agrees_with_separated_form_on_resolved_data():
    """Both forms approximate the same Q where truncation does not matter."""
    N, L = 32, 8.0
    u = np.array([1.0, 0.0, 0.0])
    f = 0.5 * (W.maxwellian(N, 3, L, 1.0, u, 0.5) + W.maxwellian(N, 3, L, 1.0, -u, 0.5))
    pm = CM.CarlemanProblem(N=N, d=3, L=L, R=5.0, M=38)
    ps = C.Problem(N=N, d=3, L=L, R=5.0, gamma=1.0, n_rho=12, M=38)
    Qm = CM.collide_fields(pm, f[None], [(0, 0)])[0]
    Qs, Qsp, Qsm = C.collide_fields(ps, f[None], [(0, 0)], return_parts=True)
    assert np.max(np.abs(Qm - Qs[0])) < 1e-2 * C.scale(Qs, Qsp, Qsm)[0]
