"""GPU parity of the FP64 check build against the FP64 oracle.

The FP64 calls run the same kernels and schedule as the FP32 path on double,
so their error against the oracle is rounding only (~1e-14); the gate is a
relative L-infinity error of 1e-11 of the per-result scale
s = max(max|Q|, max|Q+|, max|Q-|) of the oracle (T normalised by max|T|).
Inputs are seeded FP64 values (no FP32 rounding on this path).
"""
import numpy as np
import pytest

from gpu_helpers import oracle_collide, rel_err, require_gpu
from paper_2112_02695_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-11


@pytest.fixture(scope="module")
def B():
    return require_gpu()


def gpu_collide64(B, cfg, fields, pairs, form=0, return_T=False):
    import torch
    N, d, L, R, gamma, n_rho, M = cfg
    g = B.boltz_grid_init(N, d, L, R, gamma, n_rho, M)
    try:
        f = torch.tensor(np.asarray(fields, dtype=np.float64), device="cuda")
        spec = B.boltz_spectrum_f64(g, f)
        Q = B.boltz_collide_batched_f64(g, spec, [p[0] for p in pairs], [p[1] for p in pairs], form=form)
        T = B.boltz_project_f64(g, f, Q) if return_T else None
        B.boltz_sync_status(g)
        torch.cuda.synchronize()
        return (Q.cpu().numpy(), T.cpu().numpy()) if return_T else Q.cpu().numpy()
    finally:
        g.close()


@pytest.mark.parametrize("N,d", [(8, 3), (16, 3), (16, 2), (32, 2)])
def test_fp64_spectrum_matches_oracle(B, N, d):
    import torch
    from oracle import collision as C
    f = W.random_fields(N, d, 8.0, 3, seed=300 + N)
    g = B.boltz_grid_init(N, d, 8.0, 8.0, 1.0, 4, 6 if d == 3 else 8)
    try:
        spec = B.boltz_spectrum_f64(g, torch.tensor(f, dtype=torch.float64, device="cuda")).cpu().numpy()
    finally:
        g.close()
    prob = C.Problem(N=N, d=d, L=8.0, R=8.0, gamma=1.0, n_rho=4, M=6 if d == 3 else 8)
    ref = C.spectrum(prob, f)[..., : N // 2 + 1]
    assert np.max(np.abs(spec - ref)) / np.max(np.abs(ref)) < 1e-13


def test_fp64_c1_bkw_2d_and_fp32_rounding_error(B):
    """2D N=32 on [-8,8]^2, Maxwell molecules, R=8, N_rho=16 x M=16, BKW at
    t=0.5: the FP64 build meets 1e-11; the FP32 path's distance to it is
    its rounding error alone, inside the FP32 gate."""
    from gpu_helpers import gpu_collide
    cfg = (32, 2, 8.0, 8.0, 0.0, 16, 16)
    f = W.bkw(32, 2, 8.0, 0.5)[None]
    Q64 = gpu_collide64(B, cfg, f, [(0, 0)])
    _, Qo, s = oracle_collide(cfg, f, [(0, 0)])
    assert rel_err(Q64, Qo, s).max() < TOL64
    f32 = np.asarray(f, dtype=np.float32).astype(np.float64)
    Q32 = gpu_collide(B, cfg, f32, [(0, 0)])
    Q64r = gpu_collide64(B, cfg, f32, [(0, 0)])
    assert rel_err(Q32, Q64r, s).max() < 1e-5


@pytest.mark.parametrize("form", [0, 1])
def test_fp64_3d_all_pairs_and_projection(B, form):
    """3D N=16, rank-4 Hermite-Maxwellian basis, all 16 ordered pairs + T."""
    from oracle import collision as C
    cfg = (16, 3, 8.0, 8.0, 1.0, 8, 14)
    V = W.hermite_maxwellian_basis(16, 3, 8.0, 4, seed=7)
    pairs = [(j, l) for j in range(4) for l in range(4)]
    Qg, Tg = gpu_collide64(B, cfg, V, pairs, form=form, return_T=True)
    prob, Qo, s = oracle_collide(cfg, V, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL64
    To = C.project(prob, V, Qo).reshape(4, 4, 4)
    assert np.max(np.abs(Tg - To)) / np.max(np.abs(To)) < TOL64


def test_fp64_tiles_and_ragged_tail(B):
    """r = 20 inputs on 8^3: 8-wide triangular and full tiles plus a ragged
    list tail; all 400 ordered pairs."""
    cfg = (8, 3, 8.0, 8.0, 1.0, 3, 38)
    V = W.random_fields(8, 3, 8.0, 20, seed=21)
    pairs = [(j, l) for j in range(20) for l in range(20)]
    Qg = gpu_collide64(B, cfg, V, pairs)
    _, Qo, s = oracle_collide(cfg, V, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL64


def test_fp64_2d_16_hard_spheres_mixed_pairs(B):
    cfg = (16, 2, 6.0, 6.0, 1.0, 12, 24)
    V = W.random_fields(16, 2, 6.0, 5, seed=22)
    pairs = [(0, 1), (1, 0), (4, 4), (2, 3), (3, 2), (0, 4)]
    Qg = gpu_collide64(B, cfg, V, pairs)
    _, Qo, s = oracle_collide(cfg, V, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL64


def test_fp64_unsupported_grid_is_reported_and_grid_stays_usable(B):
    import torch
    g = B.boltz_grid_init(32, 3, 8.0, 8.0, 1.0, 2, 6)
    try:
        f64 = torch.zeros((1, 32, 32, 32), dtype=torch.float64, device="cuda")
        with pytest.raises(B.BoltzError) as ei:
            B.boltz_spectrum_f64(g, f64)
        assert ei.value.status == B.BOLTZ_EUNSUPPORTED
        f32 = torch.tensor(W.random_fields(32, 3, 8.0, 1, seed=5), dtype=torch.float32, device="cuda")
        spec = B.boltz_spectrum(g, f32)
        Q = B.boltz_collide_batched(g, spec, [0], [0])
        B.boltz_sync_status(g)
        assert torch.isfinite(Q).all()
    finally:
        g.close()


def test_fp64_and_fp32_calls_alternate_on_one_grid(B):
    """The two precisions share the grid's workspace and cached plan."""
    import torch
    cfg = (16, 3, 8.0, 8.0, 1.0, 4, 14)
    V = W.hermite_maxwellian_basis(16, 3, 8.0, 3, seed=9)
    pairs = [(j, l) for j in range(3) for l in range(3)]
    _, Qo, s = oracle_collide(cfg, V, pairs)
    g = B.boltz_grid_init(*cfg)
    try:
        f64 = torch.tensor(V, dtype=torch.float64, device="cuda")
        f32 = torch.tensor(V, dtype=torch.float32, device="cuda")
        pj, pl = [p[0] for p in pairs], [p[1] for p in pairs]
        for _ in range(2):
            Q64 = B.boltz_collide_batched_f64(g, B.boltz_spectrum_f64(g, f64), pj, pl)
            Q32 = B.boltz_collide_batched(g, B.boltz_spectrum(g, f32), pj, pl)
            B.boltz_sync_status(g)
            assert rel_err(Q64.cpu().numpy(), Qo, s).max() < TOL64
            assert rel_err(Q32.cpu().numpy().astype(np.float64), Qo, s).max() < 1e-5
    finally:
        g.close()
