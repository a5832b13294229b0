"""GPU parity of the Carleman form (gamma = d - 2) against oracle/carleman.py.

Gate: relative L-infinity error <= 1e-5 of the per-result scale
s = max(max|Q|, max|Q+|, max|Q-|) of the oracle (FP32 arithmetic)."""
import numpy as np
import pytest

from gpu_helpers import as_fp32, rel_err, require_gpu
from paper_2112_02695_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5
CARLEMAN = 3


@pytest.fixture(scope="module")
def B():
    return require_gpu()


def gpu_carleman(B, cfg, fields, pairs, return_T=False):
    import torch
    g = B.boltz_grid_init(*cfg)
    try:
        f = torch.tensor(np.asarray(fields, dtype=np.float32), device="cuda")
        spec = B.boltz_spectrum(g, f)
        Q = B.boltz_collide_batched(g, spec, [p[0] for p in pairs], [p[1] for p in pairs], form=CARLEMAN)
        T = B.boltz_project(g, f, Q) if return_T else None
        B.boltz_sync_status(g)
        out = Q.cpu().numpy().astype(np.float64)
        return (out, T.cpu().numpy().astype(np.float64)) if return_T else out
    finally:
        g.close()


def oracle(cfg, fields, pairs):
    from oracle import carleman as CM
    from oracle import collision as C
    N, d, L, R, gamma, n_rho, M = cfg
    prob = CM.CarlemanProblem(N=N, d=d, L=L, R=R, M=M)
    Q, Qp, Qm = CM.collide_fields(prob, fields, pairs, return_parts=True)
    return prob, Q, C.scale(Q, Qp, Qm)


def test_2d_bkw_maxwell(B):
    """C1's distribution (2D BKW at t = 0.5, Maxwell molecules) in the Carleman
    form; the oracle matches the closed form d/dt f_BKW to 5e-9 at 64^2."""
    cfg = (32, 2, 8.0, 6.0, 0.0, 1, 32)
    f = as_fp32(W.bkw(32, 2, 8.0, 0.5))[None]
    Qg = gpu_carleman(B, cfg, f, [(0, 0)])
    _, Qo, s = oracle(cfg, f, [(0, 0)])
    assert rel_err(Qg, Qo, s).max() < TOL


def test_3d_hard_spheres_all_ordered_pairs_and_projection(B):
    from oracle import collision as C
    cfg = (32, 3, 8.0, 6.0, 1.0, 1, 38)
    V = as_fp32(W.hermite_maxwellian_basis(32, 3, 8.0, 4, seed=17))
    pairs = [(j, l) for j in range(4) for l in range(4)]
    Qg, Tg = gpu_carleman(B, cfg, V, pairs, return_T=True)
    prob, Qo, s = oracle(cfg, V, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL
    To = C.project(prob.grid, V, Qo).reshape(4, 4, 4)
    assert np.max(np.abs(Tg - To)) / np.max(np.abs(To)) < TOL


def test_full_strips_and_list_tail(B):
    """r = 20 inputs on 8^3: a complete 16 x 16 block of ordered pairs (FULL
    strips) and a ragged list tail; all 400 ordered pairs."""
    cfg = (8, 3, 8.0, 5.0, 1.0, 1, 26)
    F = as_fp32(W.random_fields(8, 3, 8.0, 20, seed=23))
    pairs = [(j, l) for j in range(20) for l in range(20)]
    Qg = gpu_carleman(B, cfg, F, pairs)
    _, Qo, s = oracle(cfg, F, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL


@pytest.mark.parametrize("N,d,M", [(16, 2, 16), (24, 2, 12), (64, 2, 8), (16, 3, 14), (24, 3, 6), (64, 3, 6), (48, 3, 6)])
def test_sizes(B, N, d, M):
    cfg = (N, d, 8.0, 5.0, float(d - 2), 1, M)
    F = as_fp32(W.random_fields(N, d, 8.0, 3, seed=N + 7 * d))
    pairs = [(0, 1), (1, 0), (2, 2), (0, 2)]
    Qg = gpu_carleman(B, cfg, F, pairs)
    _, Qo, s = oracle(cfg, F, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL


def test_mass_conserved_and_duplicates(B):
    import torch
    cfg = (32, 3, 8.0, 6.0, 1.0, 1, 38)
    F = as_fp32(np.abs(W.random_fields(32, 3, 8.0, 3, seed=5)))
    pairs = [(0, 1), (0, 1), (1, 0), (2, 2)]
    g = B.boltz_grid_init(*cfg)
    try:
        f = torch.tensor(F, dtype=torch.float32, device="cuda")
        spec = B.boltz_spectrum(g, f)
        Q = B.boltz_collide_batched(g, spec, [p[0] for p in pairs], [p[1] for p in pairs], form=CARLEMAN)
        mom = B.boltz_moments(g, Q).cpu().numpy()
        B.boltz_sync_status(g)
        Qn = Q.cpu().numpy()
    finally:
        g.close()
    assert np.array_equal(Qn[0], Qn[1])
    scale = (0.5 ** 3) * np.abs(Qn).reshape(4, -1).sum(axis=1)
    assert np.max(np.abs(mom[:, 0]) / scale) < 1e-6


def test_rejections(B):
    import torch
    g = B.boltz_grid_init(16, 3, 8.0, 8.0, 0.0, 2, 6)          # gamma = 0 != d - 2
    try:
        spec = B.boltz_spectrum(g, torch.zeros((1, 16, 16, 16), device="cuda"))
        with pytest.raises(B.BoltzError) as ei:
            B.boltz_collide_batched(g, spec, [0], [0], form=CARLEMAN)
        assert ei.value.status == B.BOLTZ_EINVAL
    finally:
        g.close()
    g = B.boltz_grid_init(128, 2, 8.0, 8.0, 0.0, 2, 8)
    try:
        spec = B.boltz_spectrum(g, torch.zeros((1, 128, 128), device="cuda"))
        with pytest.raises(B.BoltzError) as ei:
            B.boltz_collide_batched(g, spec, [0], [0], form=CARLEMAN)
        assert ei.value.status == B.BOLTZ_EUNSUPPORTED
    finally:
        g.close()
