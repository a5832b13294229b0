"""Pins of the 1D normal-shock oracle (oracle/shock.py) against what the paper
and the mathematics fix: the Rankine-Hugoniot states (Sec. 4, eq. "relation"
and the closed forms of Sec. 5.2 for d = 2), the conservation form of the
upwind scheme (mass change = boundary fluxes), equilibrium preservation,
basis augmentation leaving f unchanged (Sec. 3.1), and the low-rank
splitting's first-order consistency with the full-tensor step at full
spatial rank (Sec. 2.4)."""
import math

import numpy as np
import pytest

from oracle import collision as C
from oracle import shock as SH


def problem(n_x=8, N=16, L_v=10.0, mach=1.4, L_x=6.0):
    vel = C.Problem(N=N, d=2, L=L_v, R=L_v, gamma=0.0, n_rho=6, M=12)
    return SH.ShockProblem(vel=vel, n_x=n_x, L_x=L_x, mach=mach)


def test_rankine_hugoniot_states_and_fluxes():
    M = 1.4
    (rl, ul, tl), (rr, ur, tr) = SH.shock_states(M, 2)
    # the closed forms the paper prints for d = 2, R = 1 (Sec. 5.2)
    assert rl == 1.0 and tl == 1.0 and ul == pytest.approx(math.sqrt(2.0) * M)
    assert rr == pytest.approx(3 * M ** 2 / (M ** 2 + 2))
    assert ur == pytest.approx(rl * ul / rr)
    assert tr == pytest.approx((4 * M ** 2 - 1) / (3 * rr))
    # equal fluxes of mass, momentum and energy through the shock (Sec. 4),
    # by quadrature of the two Maxwellians on a wide, fine velocity grid
    sp = problem(N=64, L_v=12.0)
    fL, fR = sp.boundary()
    vg = sp.vgrid()
    e = (vg ** 2).sum(axis=0)
    for g in (np.ones_like(e), vg[0], e):
        a = sp.wv * (vg[0] * fL * g).sum()
        b = sp.wv * (vg[0] * fR * g).sum()
        assert abs(a - b) <= 1e-9 * abs(a)


def test_full_tensor_transport_conserves_mass_up_to_boundary_fluxes():
    sp = problem()
    f = sp.initial() * (1.0 + 0.1 * np.random.default_rng(1).standard_normal((sp.n_x, 1)))
    dm, flux = SH.mass_flux_balance(sp, f, 0.01)
    assert abs(dm - flux) <= 1e-13 * max(abs(dm), abs(flux), 1.0)
    # and the sign of an outward flux: all mass leaving at the right end
    fz = np.zeros_like(f)
    fz[-1] = sp.boundary()[1] * 0 + 1.0
    dm, flux = SH.mass_flux_balance(sp, fz, 0.01)
    assert abs(dm - flux) <= 1e-13


def test_uniform_equilibrium_is_preserved_by_both_schemes():
    sp = problem(mach=1.0)            # Mach 1: f_L = f_R, a uniform Maxwellian
    f0 = sp.initial()
    fL, fR = sp.boundary()
    assert np.allclose(fL, fR) and np.allclose(f0, fL[None, :])
    qscale = np.abs(SH.collide_cells(sp, f0[:1])).max()
    f1 = SH.full_step(sp, f0, 0.01)
    assert np.max(np.abs(f1 - f0)) <= 0.01 * qscale + 1e-14
    X, S, V = SH.factor(sp, f0, 1)
    X1, S1, V1 = SH.lowrank_step(sp, X, S, V, 0.01, 1e-6, SH.random_xh(sp.n_x))
    assert np.max(np.abs(SH.reconstruct(X1, S1, V1) - f0)) <= 0.01 * qscale + 1e-12
    # the added boundary direction carries weight only through the spectral
    # error of Q(M, M) (sigma_2 ~ dt |Q(M,M)| ~ 4e-8 here) and is dropped
    assert S1.shape[0] == 1


def test_adding_basis_leaves_f_unchanged():
    sp = problem(mach=1.4)
    f0 = sp.initial()
    X, S, V = SH.factor(sp, f0, 3)
    Xq, Sq, Vq = SH.add_basis(sp, X, S, V, SH.random_xh(sp.n_x, seed=3))
    assert Sq.shape == (5, 5)
    assert np.allclose(sp.dx * Xq @ Xq.T, np.eye(5), atol=1e-12)
    assert np.allclose(sp.wv * Vq @ Vq.T, np.eye(5), atol=1e-12)
    assert np.max(np.abs(SH.reconstruct(Xq, Sq, Vq) - SH.reconstruct(X, S, V))) <= 1e-13 * np.abs(f0).max()


def test_lowrank_step_is_consistent_with_the_full_tensor_step():
    """At full spatial rank (X spans every cell: rank 6 plus the two added
    directions on 8 cells) the K-S-L splitting differs from the full-tensor
    Euler step by O(dt^2) in the interior cells.  In the two boundary cells it
    differs at O(dt): the low-rank step sees the inflow data only through its
    projection onto span(V) (eq. "boundary general"), the full-tensor step
    sees f_L and f_R exactly."""
    sp = problem(n_x=8, mach=1.4)
    f0 = sp.initial()
    X, S, V = SH.factor(sp, f0, 6)
    Xh = SH.random_xh(sp.n_x, seed=4)
    f_start = SH.reconstruct(X, S, V)              # the rank-6 state both steps start from
    inner, edge = [], []
    for dt in (0.002, 0.001, 0.0005):
        d = SH.reconstruct(*SH.lowrank_step(sp, X, S, V, dt, 0.0, Xh)) - SH.full_step(sp, f_start, dt)
        inner.append(np.max(np.abs(d[1:-1])))
        edge.append(np.max(np.abs(d[[0, -1]])))
    for a, b in zip(inner, inner[1:]):
        assert 3.6 < a / b < 4.4, inner
    for a, b in zip(edge[1:], edge[2:]):
        assert 1.6 < a / b < 2.4, edge
    assert inner[0] <= 1e-5 * np.abs(f0).max()


def test_convergence_measure_equals_the_norm_of_the_change():
    """Sec. 5.1: err from the increments and the three cross terms equals
    ||f^{n+1} - f^n|| of the rebuilt solutions (before the drop)."""
    sp = problem(n_x=12, mach=1.4)
    f0 = sp.initial()
    X, S, V = SH.factor(sp, f0, 4)
    (X1, S1, V1), parts = SH.lowrank_step(sp, X, S, V, 0.005, 0.0, SH.random_xh(sp.n_x, seed=5),
                                          return_parts=True)
    d = SH.reconstruct(X1, S1, V1) - SH.reconstruct(X, S, V)
    direct = np.sqrt(sp.dx * sp.wv * (d * d).sum())
    assert parts["err"] == pytest.approx(direct, rel=1e-10)
    assert direct > 0
