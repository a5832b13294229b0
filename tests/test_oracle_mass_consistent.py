"""Pins of the oracle's mass-consistent loss option (CPU, FP64).

Reading of the loss weight (Sec. 2.1 cites the separated spectral method
without printing its loss term): by default G-(l) is the exact sigma- and
omega-average; the option loss="mass_consistent" takes the sigma-average with
the gain's own direction rule, G-(l) = G_sep(l, -l).  Then the k = 0 mode of
Q, its mass (Sec. 1 collision invariants), cancels exactly: the direct sum
gives Qhat_0 = sum_l [G_sep(l, -l) - G-(l)] ghat_l fhat_-l.

Pins: (1) mass of Q(g, f), g != f, vanishes to rounding with the option on
coarse rules where the exact average leaves a visible defect; (2) the
separated path equals the O(n^2) direct sum, whose G_sep is evaluated by its
own code; (3) on a circle rule fine enough to integrate every Fourier mode of
the grid, the two loss weights coincide (the rule's average converges to
2 pi J0); (4) planted mistakes in the weight are caught.
"""
import math

import numpy as np
import pytest

from oracle import collision as C
from paper_2112_02695_gb300 import workloads as W


@pytest.mark.parametrize("d,N,n_rho,M,gamma", [
    (2, 16, 4, 8, 1.0), (2, 16, 6, 12, 0.0), (3, 8, 4, 14, 1.0), (3, 8, 3, 6, 0.0)])
def test_mass_consistent_loss_conserves_mass(d, N, n_rho, M, gamma):
    f = W.random_fields(N, d, 8.0, 2, seed=31 + N + d)
    out = {}
    for loss in ("exact", "mass_consistent"):
        prob = C.Problem(N=N, d=d, L=8.0, R=8.0, gamma=gamma, n_rho=n_rho, M=M, loss=loss)
        Q, Qp, _ = C.collide_fields(prob, f, [(0, 1), (1, 0), (1, 1)], return_parts=True)
        scl = np.max(np.abs(C.moments(prob, Qp)[:, 0]))
        out[loss] = np.max(np.abs(C.moments(prob, Q)[:, 0])) / scl
    assert out["mass_consistent"] < 1e-13
    assert out["exact"] > 1e-6          # the coarse rules leave a visible mass defect


@pytest.mark.parametrize("d,N,n_rho,M,gamma", [
    (2, 16, 5, 8, 1.0), (2, 8, 4, 4, 0.0), (3, 8, 4, 14, 1.0), (3, 8, 3, 6, 0.0)])
def test_mass_consistent_separated_path_equals_direct_sum(d, N, n_rho, M, gamma):
    prob = C.Problem(N=N, d=d, L=8.0, R=8.0, gamma=gamma, n_rho=n_rho, M=M, loss="mass_consistent")
    f = W.random_fields(N, d, 8.0, 2, seed=17 + N + d)
    spec = C.spectrum(prob, f)
    Q, Qp, Qm = C.collide(prob, spec, [(0, 1)], return_parts=True)
    Qd_hat = C.direct_sum(prob, spec[0], spec[1])
    s = C.scale(Q, Qp, Qm)[0]
    assert float(np.max(np.abs(C.synthesize(prob, Qd_hat) - Q[0]))) / s < 1e-13
    assert abs(Qd_hat.reshape(-1)[0]) / np.max(np.abs(Qd_hat)) < 1e-14


def test_mass_consistent_weight_converges_to_the_exact_average():
    """2D, circle rule with M = 128 directions: sum_p w_p e^{-i x.sigma_p}
    equals 2 pi J0(|x|) up to terms of order J_M(|x|), below 1e-15 for the
    grid's largest |x| = pi R |l|max / L < 36."""
    prob_e = C.Problem(N=16, d=2, L=8.0, R=8.0, gamma=1.0, n_rho=6, M=128)
    prob_m = C.Problem(N=16, d=2, L=8.0, R=8.0, gamma=1.0, n_rho=6, M=128, loss="mass_consistent")
    Ge = C.loss_table(prob_e)
    Gm = C.loss_table(prob_m)
    assert np.max(np.abs(Ge - Gm)) / np.max(np.abs(Ge)) < 1e-12


def test_mass_consistent_weight_at_zero_frequency():
    """G-(0) = b |S^{d-1}| sum_q w_q rho_q^{gamma+d-1} |S^{d-1}| for both
    readings: at l = 0 every direction contributes exp(0) = 1 and the rule's
    weights sum to |S^{d-1}|."""
    for d, M in ((2, 8), (3, 14)):
        prob = C.Problem(N=8, d=d, L=8.0, R=8.0, gamma=1.0, n_rho=4, M=M, loss="mass_consistent")
        g0 = C.loss_table(prob).reshape(-1)[0]
        area = C.sphere_area(d)
        want = prob.b * area * area * sum(prob.w_rho[q] * prob.rho[q] ** (1.0 + d - 1) for q in range(prob.n_rho))
        assert abs(g0 - want) / want < 1e-14


def _half_phase(orig):
    def wrong(prob, lvec):
        return orig(prob, 0.5 * np.asarray(lvec, dtype=np.float64))
    return wrong


def _no_fd0(orig):
    def wrong(prob, lvec):
        return orig(prob, lvec) / float(C.F_d(prob.d, 0.0))
    return wrong


MC_MUTATIONS = {
    "phase rho l.sigma / (2L) instead of / L": ("loss_weight_mass_consistent", _half_phase),
    "omega-average F_d(0) dropped": ("loss_weight_mass_consistent", _no_fd0),
}


@pytest.mark.parametrize("name", sorted(MC_MUTATIONS))
def test_planted_mass_consistent_mistake_is_caught(name, monkeypatch):
    attr, make = MC_MUTATIONS[name]
    monkeypatch.setattr(C, attr, make(getattr(C, attr)))
    with pytest.raises(AssertionError):
        test_mass_consistent_loss_conserves_mass(3, 8, 4, 14, 1.0)
    with pytest.raises(AssertionError):
        test_mass_consistent_weight_converges_to_the_exact_average()
