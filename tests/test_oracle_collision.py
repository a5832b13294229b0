"""Pins of the oracle's collision operator (CPU, FP64).

Each test ties the oracle to something other than itself: the brute-force
direct sum, the BKW closed form, an independent physical-space quadrature of
the paper's integral (Sec. 1, eq. "eqn:collision_operator"), collision
invariants (Sec. 1 moments; Sec. 4.1 kernel of L_M), exact symmetries, and the
paper's Rankine-Hugoniot relation.  The last group plants plausible mistakes in
the oracle and checks that a pin catches each of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import collision as C
from oracle import quadrature as Qd
from paper_2112_02695_gb300 import workloads as W
from physical_quadrature import maxwellian_fn, q_physical

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b, s):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / s)


# ---------------------------------------------------------------- direct sum

@pytest.mark.parametrize("N,d,n_rho,M,gamma", [
    (16, 2, 6, 8, 1.0), (16, 2, 5, 16, 0.0), (8, 2, 4, 4, 1.0), (8, 3, 4, 14, 1.0), (8, 3, 3, 6, 0.0)])
def test_separated_path_equals_direct_sum(N, d, n_rho, M, gamma):
    """Steps 3-7 (shifted fields, products, per-node DFT, radial multiplier,
    loss) against the O(n^2) sum over l+m = k (mod N): exact to rounding."""
    prob = C.Problem(N=N, d=d, L=8.0, R=8.0, gamma=gamma, n_rho=n_rho, M=M)
    f = W.random_fields(N, d, 8.0, 2, seed=11 + N + d)
    spec = C.spectrum(prob, f)
    Q, Qp, Qm = C.collide(prob, spec, [(0, 1)], return_parts=True)
    Qd_hat = C.direct_sum(prob, spec[0], spec[1])
    s = C.scale(Q, Qp, Qm)[0]
    assert rel(C.synthesize(prob, Qd_hat), Q[0], s) < 1e-13
    # also in spectral space: the direct sum is the DFT of the grid values
    assert np.max(np.abs(C.dft(prob, Q[0]) - Qd_hat)) / np.max(np.abs(Qd_hat)) < 1e-12


# ---------------------------------------------------------------- BKW

def _bkw_dt(N, d, L, t):
    V = W.velocity_mesh(N, d, L)
    r2 = sum(x * x for x in V)
    K = W.bkw_K(d, t)
    if d == 2:
        dK = math.exp(-t / 8.0) / 16.0
        e = np.exp(-r2 / (2 * K))
        pre = e / (2 * math.pi * K * K)
        dpre = pre * (r2 / (2 * K * K) - 2.0 / K)
        br = 2 * K - 1 + (1 - K) * r2 / (2 * K)
        dbr = 2.0 - r2 / (2 * K * K)
        return (dpre * br + pre * dbr) * dK
    dK = math.exp(-t / 6.0) / 6.0
    pre = (2 * math.pi * K) ** -1.5 * np.exp(-r2 / (2 * K))
    dpre = pre * (-1.5 / K + r2 / (2 * K * K))
    br = (5 * K - 3) / (2 * K) + (1 - K) * r2 / (2 * K * K)
    dbr = 3.0 / (2 * K * K) + r2 * (-1.0 / (2 * K * K) - (1 - K) / (K ** 3))
    return (dpre * br + pre * dbr) * dK


def test_bkw_mass_and_temperature():
    for d, L, N, t in [(2, 8.0, 64, 0.5), (3, 8.0, 48, 6.0)]:
        f = W.bkw(N, d, L, t)
        dv = (2 * L / N) ** d
        V = W.velocity_mesh(N, d, L)
        assert abs(dv * f.sum() - 1.0) < 1e-10
        assert abs(dv * np.sum(f * sum(x * x for x in V)) / d - 1.0) < 1e-9


def test_bkw_2d_maxwell_closed_form():
    """2D Maxwell molecules, b = 1/(2 pi): Q(f,f) = d/dt f_BKW (closed form)."""
    prob = C.Problem(N=64, d=2, L=8.0, R=8.0, gamma=0.0, n_rho=32, M=64)
    f = W.bkw(64, 2, 8.0, 0.5)
    Q = C.collide_fields(prob, f[None], [(0, 0)])[0]
    ex = _bkw_dt(64, 2, 8.0, 0.5)
    assert rel(Q, ex, np.abs(ex).max()) < 1e-10


def test_bkw_2d_convergence_in_N():
    errs = []
    for N in (16, 24, 32, 48):
        prob = C.Problem(N=N, d=2, L=8.0, R=8.0, gamma=0.0, n_rho=16, M=32)
        f = W.bkw(N, 2, 8.0, 0.5)
        Q = C.collide_fields(prob, f[None], [(0, 0)])[0]
        ex = _bkw_dt(N, 2, 8.0, 0.5)
        errs.append(rel(Q, ex, np.abs(ex).max()))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5


@pytest.mark.slow
def test_bkw_3d_maxwell_closed_form():
    """3D Maxwell molecules (gamma = 0), b = 1/(4 pi), 86-point rule."""
    prob = C.Problem(N=32, d=3, L=6.0, R=6.0, gamma=0.0, n_rho=16, M=86)
    f = W.bkw(32, 3, 6.0, 6.0)
    Q = C.collide_fields(prob, f[None], [(0, 0)])[0]
    ex = _bkw_dt(32, 3, 6.0, 6.0)
    assert rel(Q, ex, np.abs(ex).max()) < 1e-5


# ---------------------------------------------------------------- physical quadrature

def test_matches_physical_space_quadrature_2d_hard_spheres():
    """gamma = 1, g != f: the oracle at fine quadrature equals an independent
    quadrature of the defining integral at sample velocities."""
    L = 8.0
    gp = (1.0, [0.5, -0.3], 0.8)
    fp = (1.2, [-0.4, 0.2], 1.1)
    N = 48
    prob = C.Problem(N=N, d=2, L=L, R=L, gamma=1.0, n_rho=32, M=64)
    g = W.maxwellian(N, 2, L, *gp)
    f = W.maxwellian(N, 2, L, *fp)
    Q, Qp, Qm = C.collide_fields(prob, np.stack([g, f]), [(0, 1)], return_parts=True)
    s = C.scale(Q, Qp, Qm)[0]
    ax = W.velocity_axis(N, L)
    for i, j in [(24, 24), (27, 19), (18, 26), (32, 25)]:
        _, _, q = q_physical(maxwellian_fn(*gp), maxwellian_fn(*fp), [ax[i], ax[j]], 2, L, 1.0,
                             prob.b, n_rho=48, n_dir=96)
        assert abs(q - Q[0, i, j]) / s < 1e-7


@pytest.mark.slow
def test_matches_physical_space_quadrature_3d_hard_spheres():
    L = 6.0
    gp = (1.0, [0.5, -0.3, 0.1], 0.8)
    fp = (1.2, [-0.4, 0.2, 0.0], 1.1)
    N = 32
    prob = C.Problem(N=N, d=3, L=L, R=L, gamma=1.0, n_rho=16, M=86)
    g = W.maxwellian(N, 3, L, *gp)
    f = W.maxwellian(N, 3, L, *fp)
    Q, Qp, Qm = C.collide_fields(prob, np.stack([g, f]), [(0, 1)], return_parts=True)
    s = C.scale(Q, Qp, Qm)[0]
    ax = W.velocity_axis(N, L)
    for i, j, k in [(16, 16, 16), (18, 13, 17)]:
        _, _, q = q_physical(maxwellian_fn(*gp), maxwellian_fn(*fp), [ax[i], ax[j], ax[k]], 3, L,
                             1.0, prob.b, n_rho=32, n_dir=16)
        assert abs(q - Q[0, i, j, k]) / s < 1e-5


# ---------------------------------------------------------------- invariants

def test_maxwellian_is_an_equilibrium():
    """Q(M, M) = 0 for a Maxwellian (Sec. 4.1 uses this), to spectral accuracy."""
    prob = C.Problem(N=48, d=2, L=8.0, R=8.0, gamma=1.0, n_rho=24, M=32)
    m = W.maxwellian(48, 2, 8.0, 1.3, [0.4, -0.2], 1.0)
    Q, Qp, Qm = C.collide_fields(prob, m[None], [(0, 0)], return_parts=True)
    assert np.abs(Q).max() / np.abs(Qp).max() < 1e-6


@pytest.mark.parametrize("d,N,rho,u,T", [(2, 64, 1.3, [0.7, -0.4], 0.8), (3, 48, 0.6, [-0.5, 0.3, 0.9], 1.2)])
def test_moments_of_a_maxwellian_match_the_closed_form(d, N, rho, u, T):
    """The moment sums of Sec. 1 against the closed-form moments of a
    Maxwellian rho (2 pi T)^(-d/2) exp(-|v-u|^2/(2T)) resolved on the grid
    (the periodic midpoint rule is spectrally accurate; what is left is the
    tail beyond the box, ~1e-9 here): mass rho, momentum rho u, energy
    rho (|u|^2 + d T).  A wrong cell volume or a grid origin off by half a
    cell fails it (see the planted mistakes below)."""
    prob = C.Problem(N=N, d=d, L=8.0, R=8.0, gamma=1.0, n_rho=2, M=8 if d == 2 else 6)
    m = W.maxwellian(N, d, 8.0, rho, u, T)
    mom = C.moments(prob, m[None])[0]
    u = np.asarray(u)
    exact = np.concatenate([[rho], rho * u, [rho * (u @ u + d * T)]])
    assert np.max(np.abs(mom - exact)) < 1e-7 * max(1.0, np.max(np.abs(exact)))


MOMENT_MUTATIONS = {
    "cell volume dv^(d-1)": ("cell_volume", lambda orig: (lambda prob: prob.dv ** (prob.d - 1))),
    "grid origin at the cell centre": ("velocity_axis",
        lambda orig: (lambda prob: orig(prob) + 0.5 * prob.dv)),
}


@pytest.mark.parametrize("name", sorted(MOMENT_MUTATIONS))
def test_planted_moment_mistake_is_caught(name, monkeypatch):
    attr, make = MOMENT_MUTATIONS[name]
    monkeypatch.setattr(C, attr, make(getattr(C, attr)))
    with pytest.raises(AssertionError):
        test_moments_of_a_maxwellian_match_the_closed_form(3, 48, 0.6, [-0.5, 0.3, 0.9], 1.2)


def test_conservation_of_mass_momentum_energy():
    """int Q {1, v, |v|^2} dv = 0 (Sec. 1 moments, collision invariants) for
    Q(f,f) and the symmetrised Q(g,f) + Q(f,g); a single Q(g,f), g != f, keeps
    only mass (momentum and energy need the v <-> v_* swap, which swaps g, f).
    R = 5 < 4L/(3+sqrt 2) keeps post-collision velocities from wrapping around
    the periodic box, so the invariants hold to rounding."""
    prob = C.Problem(N=64, d=2, L=8.0, R=5.0, gamma=1.0, n_rho=24, M=32)
    f = W.random_fields(64, 2, 8.0, 2, seed=4)
    Q, Qp, Qm = C.collide_fields(prob, f, [(0, 1), (1, 0), (0, 0)], return_parts=True)
    scl = np.max(C.moments(prob, np.abs(Qp))[:, 0])
    mom = C.moments(prob, np.stack([Q[0] + Q[1], Q[2]]))
    assert np.max(np.abs(mom)) / scl < 1e-10
    assert np.max(np.abs(C.moments(prob, Q[:2])[:, 0])) / scl < 1e-10
    assert np.max(np.abs(C.moments(prob, Q[:1])[:, 1:])) / scl > 1e-3


def test_bilinearity_and_bimodal_identity():
    """Q(a f1 + (1-a) f2, same) = a^2 Q11 + a(1-a)(Q12 + Q21) + (1-a)^2 Q22."""
    prob = C.Problem(N=16, d=3, L=8.0, R=8.0, gamma=1.0, n_rho=4, M=14)
    fL, fR = W.shock_states_fields(16, 3, 8.0)
    a = 0.3
    mix = a * fL + (1 - a) * fR
    Qs = C.collide_fields(prob, np.stack([fL, fR, mix]), [(0, 0), (0, 1), (1, 0), (1, 1), (2, 2)])
    pred = a * a * Qs[0] + a * (1 - a) * (Qs[1] + Qs[2]) + (1 - a) ** 2 * Qs[3]
    assert rel(pred, Qs[4], np.abs(Qs[4]).max()) < 1e-12


def test_gain_is_symmetric():
    """Q+(g,f) = Q+(f,g) for a centrally symmetric direction rule."""
    for d, N, M in [(2, 16, 8), (3, 8, 38)]:
        prob = C.Problem(N=N, d=d, L=8.0, R=8.0, gamma=1.0, n_rho=4, M=M)
        f = W.random_fields(N, d, 8.0, 2, seed=9)
        _, Qp, _ = C.collide_fields(prob, f, [(0, 1), (1, 0)], return_parts=True)
        assert rel(Qp[0], Qp[1], np.abs(Qp).max()) < 1e-13


def test_grid_shift_equivariance():
    """Rolling both inputs by whole grid steps rolls Q the same way."""
    prob = C.Problem(N=16, d=2, L=8.0, R=8.0, gamma=1.0, n_rho=5, M=8)
    f = W.random_fields(16, 2, 8.0, 2, seed=21)
    Q = C.collide_fields(prob, f, [(0, 1)])[0]
    fs = np.roll(f, (3, -2), axis=(1, 2))
    Qs = C.collide_fields(prob, fs, [(0, 1)])[0]
    assert rel(np.roll(Q, (3, -2), axis=(0, 1)), Qs, np.abs(Q).max()) < 1e-13


@pytest.mark.parametrize("d,N,M", [(2, 16, 8), (3, 8, 38)])
def test_quarter_turn_equivariance(d, N, M):
    """A quarter turn v -> (-v_1, v_0, ...) maps the periodic grid to itself and
    the direction rule to itself, so it commutes with Q."""
    prob = C.Problem(N=N, d=d, L=8.0, R=8.0, gamma=1.0, n_rho=4, M=M)
    f = W.random_fields(N, d, 8.0, 2, seed=33)

    def turn(x):
        # new(v0, v1) = old(v1, -v0): index i0' <- i1, i1' <- (N - i0) mod N
        y = np.swapaxes(x, -d, -d + 1)
        return np.roll(np.flip(y, axis=-d + 1), 1, axis=-d + 1)
    Q = C.collide_fields(prob, f, [(0, 1)])[0]
    Qt = C.collide_fields(prob, turn(f), [(0, 1)])[0]
    assert rel(turn(Q), Qt, np.abs(Q).max()) < 1e-13


def test_projection_is_midpoint_rule():
    prob = C.Problem(N=8, d=3, L=8.0, R=8.0, gamma=1.0, n_rho=3, M=6)
    V = W.hermite_maxwellian_basis(8, 3, 8.0, 4, seed=1)
    Qs = np.random.default_rng(2).standard_normal((16,) + prob.shape)
    T = C.project(prob, V, Qs)
    k, p = 2, 7
    assert abs(T[k, p] - prob.dv ** 3 * np.sum(V[k] * Qs[p])) < 1e-12


def test_hermite_basis_is_orthonormal():
    V = W.hermite_maxwellian_basis(16, 3, 8.0, 16, seed=2112)
    dv = 1.0 ** 3
    G = dv * V.reshape(16, -1) @ V.reshape(16, -1).T
    assert np.max(np.abs(G - np.eye(16))) < 1e-12


def test_rankine_hugoniot_matches_golden():
    vals = {}
    for line in open(os.path.join(GOLDEN, "rankine_hugoniot_d3_mach3.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    (rL, uL, TL), (rR, uR, TR) = W.rankine_hugoniot(3, 3.0)
    assert abs(rR - vals["rho_R"]) < 1e-14
    assert abs(uR / uL - vals["u_ratio"]) < 1e-14
    assert abs(TR - vals["T_R"]) < 1e-14
    assert abs(uL - vals["u_L"]) < 1e-14


# ---------------------------------------------------------------- planted mistakes

def _pins_pass():
    """The cheap pins: 2D BKW closed form and the 2D hard-sphere physical
    quadrature with g != f.  Returns True iff both pass."""
    try:
        test_bkw_2d_maxwell_closed_form()
        test_matches_physical_space_quadrature_2d_hard_spheres()
    except AssertionError:
        return False
    return True


MUTATIONS = {
    "dropped half in the node shift": ("gain_shifts",
        lambda orig: (lambda prob, q, p: tuple(2 * s for s in orig(prob, q, p)))),
    "both fields shifted the same way": ("gain_shifts",
        lambda orig: (lambda prob, q, p: (orig(prob, q, p)[0], orig(prob, q, p)[0]))),
    "missing Jacobian rho^{d-1}": ("kernel_power",
        lambda orig: (lambda prob: prob.gamma)),
    "g and f swapped in the loss": ("loss_field",
        lambda orig: (lambda fN, lam, jj, ll: fN[jj] * lam[ll])),
    "omega-average at |k|/L instead of |k|/(2L)": ("radial_multiplier",
        lambda orig: (lambda prob, kmag: orig(prob, 2.0 * kmag))),
}


def test_pins_pass_on_the_unmodified_oracle():
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, make = MUTATIONS[name]
    monkeypatch.setattr(C, attr, make(getattr(C, attr)))
    assert not _pins_pass(), f"mistake not caught: {name}"
