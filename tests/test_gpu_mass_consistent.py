"""GPU parity of the mass-consistent loss option (BOLTZ_LOSS_MASS_CONSISTENT).

The loss weight G-(l) = G_sep(l, -l) (the gain's own direction rule as the
sigma-average; the reading of the separated kernel of Sec. 2.1 under which
the k = 0 mode of Q cancels) is applied per spectral mode by every separated
path.  Against the FP64 oracle with the same option on each kernel family
(single-CTA 2D and 3D grids, the 2D 128^2 path, the 3D 32^3 node-block and
pipelined schedules, the FP64 check build), and the mass of Q, from the
library's FP64 moment sums, against the exact loss's mass defect.
Tolerance as the other parity tests: 1e-5 of the oracle's per-result scale
(FP64 build: 1e-11).
"""
import numpy as np
import pytest

from gpu_helpers import as_fp32, gpu_collide, oracle_collide, rel_err, require_gpu
from paper_2112_02695_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5
MC = 1


@pytest.fixture(scope="module")
def B():
    return require_gpu()


@pytest.mark.parametrize("cfg,schedule", [
    ((16, 2, 8.0, 8.0, 1.0, 4, 8), 0),
    ((16, 3, 8.0, 8.0, 1.0, 3, 14), 0),
    ((128, 2, 8.0, 8.0, 0.0, 2, 8), 0),
    ((32, 3, 8.0, 8.0, 1.0, 2, 14), 0),        # pipelined
    ((32, 3, 8.0, 8.0, 1.0, 2, 14), 1),        # node blocks
])
def test_mass_consistent_against_oracle(B, cfg, schedule):
    N, d = cfg[0], cfg[1]
    f = as_fp32(W.random_fields(N, d, 8.0, 3, seed=500 + N + d))
    pairs = [(0, 1), (1, 0), (2, 2), (0, 2)]
    launches = {}
    Qg = gpu_collide(B, cfg, f, pairs, schedule=schedule, launches=launches, loss=MC)
    if N == 32 and d == 3:
        assert (launches["pipeline"] == 1) == (schedule == 0)
    _, Qo, s = oracle_collide(cfg, f, pairs, loss="mass_consistent")
    assert rel_err(Qg, Qo, s).max() < TOL


def test_mass_consistent_loss_conserves_mass_on_the_gpu(B):
    """3D 32^3 pipelined, rank-4 basis: the FP64 mass sums of Q(V_j, V_l) with
    the option sit at FP32 rounding, orders of magnitude below the exact
    loss's quadrature defect on the same coarse rule."""
    import torch
    cfg = (32, 3, 8.0, 8.0, 1.0, 2, 14)
    V = as_fp32(W.hermite_maxwellian_basis(32, 3, 8.0, 4, seed=77))
    pairs = [(j, l) for j in range(4) for l in range(4)]
    _, _, s = oracle_collide(cfg, V, pairs)
    mass = {}
    for loss in (0, MC):
        g = B.boltz_grid_init(*cfg, loss=loss)
        try:
            spec = B.boltz_spectrum(g, torch.tensor(np.asarray(V, dtype=np.float32), device="cuda"))
            Q = B.boltz_collide_batched(g, spec, [p[0] for p in pairs], [p[1] for p in pairs])
            mom = B.boltz_moments(g, Q).cpu().numpy()
            B.boltz_sync_status(g)
        finally:
            g.close()
        dv3 = (16.0 / 32) ** 3
        mass[loss] = np.max(np.abs(mom[:, 0]) / (s * 32 ** 3 * dv3))
    assert mass[MC] < 1e-7
    assert mass[0] > 100 * mass[MC]


def test_mass_consistent_fp64_build(B):
    import torch
    cfg = (16, 3, 8.0, 8.0, 1.0, 3, 14)
    f = W.random_fields(16, 3, 8.0, 2, seed=510)
    pairs = [(0, 1), (1, 1)]
    g = B.boltz_grid_init(*cfg, loss=MC)
    try:
        spec = B.boltz_spectrum_f64(g, torch.tensor(f, dtype=torch.float64, device="cuda"))
        Q = B.boltz_collide_batched_f64(g, spec, [p[0] for p in pairs], [p[1] for p in pairs])
        B.boltz_sync_status(g)
        Qg = Q.cpu().numpy()
    finally:
        g.close()
    _, Qo, s = oracle_collide(cfg, f, pairs, loss="mass_consistent")
    assert rel_err(Qg, Qo, s).max() < 1e-11
    assert np.max(np.abs(Qg.reshape(2, -1).sum(axis=1))) / (s.max() * 16 ** 3) < 1e-13


def test_bad_loss_option_is_rejected(B):
    with pytest.raises(B.BoltzError):
        B.boltz_grid_init(16, 3, 8.0, 8.0, 1.0, 2, 6, loss=7)
