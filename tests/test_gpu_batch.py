"""Mixed batch under one captured CUDA graph: grids of different N, d,
quadrature and rank in one boltz_batch; every replay must reproduce the
individual calls exactly, and one item is checked against the oracle."""
import numpy as np
import pytest

from gpu_helpers import as_fp32, oracle_collide, rel_err, require_gpu
from paper_2112_02695_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CFGS = [  # (N, d, L, R, gamma, N_rho, M, r)
    (16, 3, 8.0, 8.0, 1.0, 4, 14, 4),
    (32, 2, 8.0, 8.0, 0.0, 8, 16, 5),
    (24, 3, 8.0, 8.0, 0.0, 3, 6, 3),
]


def test_batch_graph_replays_match_individual_calls():
    import torch
    B = require_gpu()
    grids, items, ref = [], [], []
    for i, (N, d, L, R, gamma, n_rho, M, r) in enumerate(CFGS):
        g = B.boltz_grid_init(N, d, L, R, gamma, n_rho, M)
        grids.append(g)
        V = as_fp32(W.hermite_maxwellian_basis(N, d, L, r, seed=2114 + i))
        f = torch.tensor(V, dtype=torch.float32, device="cuda")
        pj = [j for j in range(r) for _ in range(r)]
        pl = [l for _ in range(r) for l in range(r)]
        spec = torch.zeros((r,) + g.half_shape, dtype=torch.complex64, device="cuda")
        Q = torch.full((r * r,) + g.shape, float("nan"), device="cuda")
        T = torch.full((r, r, r), float("nan"), device="cuda")
        items.append(dict(grid=g, fields=f, spectra=spec, pair_j=pj, pair_l=pl, Q_out=Q, V=f, T_out=T))
        # the same work through the individual calls
        s1 = B.boltz_spectrum(g, f)
        Q1 = B.boltz_collide_batched(g, s1, pj, pl)
        T1 = B.boltz_project(g, f, Q1)
        ref.append((Q1.clone(), T1.clone(), V, pj, pl))
    torch.cuda.synchronize()
    batch = B.boltz_batch_plan(items)
    try:
        assert B.boltz_batch_kernel_count(batch) > 0
        for rep in range(2):
            for it in items:
                it["Q_out"].fill_(float("nan"))
            B.boltz_batch_run(batch)
            torch.cuda.synchronize()
            for it, (Q1, T1, _, _, _) in zip(items, ref):
                assert torch.equal(it["Q_out"], Q1), rep
                assert torch.equal(it["T_out"], T1), rep
        for g in grids:
            B.boltz_sync_status(g)
    finally:
        batch.close()
    # one item against the oracle
    N, d, L, R, gamma, n_rho, M, r = CFGS[1]
    Q1, _, V, pj, pl = ref[1]
    _, Qo, s = oracle_collide((N, d, L, R, gamma, n_rho, M), V, list(zip(pj, pl)))
    assert rel_err(Q1.cpu().numpy().astype(np.float64), Qo, s).max() < 1e-5
    for g in grids:
        g.close()


def test_batch_rejects_two_items_on_one_grid():
    import torch
    B = require_gpu()
    g = B.boltz_grid_init(8, 3, 8.0, 8.0, 1.0, 2, 6)
    try:
        spec = torch.zeros((2,) + g.half_shape, dtype=torch.complex64, device="cuda")
        Q = torch.zeros((1,) + g.shape, device="cuda")
        it = dict(grid=g, spectra=spec, pair_j=[0], pair_l=[1], Q_out=Q)
        with pytest.raises(B.BoltzError) as ei:
            B.boltz_batch_plan([it, dict(it)])
        assert ei.value.status == B.BOLTZ_EINVAL
    finally:
        g.close()


def test_autotune_picks_a_candidate_and_caches_it(tmp_path):
    import json
    import torch
    B = require_gpu()
    cfg = (16, 3, 8.0, 8.0, 1.0, 6, 14)
    V = as_fp32(W.hermite_maxwellian_basis(16, 3, 8.0, 6, seed=9))
    pairs = [(j, l) for j in range(6) for l in range(6)]
    g = B.boltz_grid_init(*cfg)
    try:
        f = torch.tensor(V, dtype=torch.float32, device="cuda")
        spec = B.boltz_spectrum(g, f)
        before = B.boltz_collide_batched(g, spec, [p[0] for p in pairs], [p[1] for p in pairs]).clone()
        cache = str(tmp_path / "tune.json")
        mb = B.boltz_autotune(g, spec, [p[0] for p in pairs], [p[1] for p in pairs], cache_path=cache)
        assert mb in (48, 96, 192, 384, 768)
        entries = json.load(open(cache))
        assert list(entries.values()) == [mb]
        assert B.boltz_autotune(g, spec, [p[0] for p in pairs], [p[1] for p in pairs], cache_path=cache) == mb
        after = B.boltz_collide_batched(g, spec, [p[0] for p in pairs], [p[1] for p in pairs])
        torch.cuda.synchronize()
        scale = before.abs().max().item()
        assert (after - before).abs().max().item() <= 1e-6 * scale
    finally:
        g.close()


# the six-grid uneven mixed batch: (N, d, gamma, M, r), R = L = 8, N_rho = N, bases seeded 2114 + i
C5_GRIDS = [(24, 3, 0.0, 38, 32), (32, 3, 1.0, 38, 16), (48, 3, 0.0, 86, 8), (64, 3, 1.0, 86, 4),
            (64, 2, 0.0, 16, 16), (128, 2, 1.0, 16, 8)]
# sampled pair per grid checked against the oracle (None: the 64^3 grid at N_rho = 64 takes the
# oracle several minutes; its kernels are the ones the 64^3 full-quadrature test checks)
C5_SAMPLES = [(3, 17), (5, 2), (1, 1), None, (0, 15), (6, 3)]


@pytest.mark.slow
def test_c5_six_grid_batch_against_oracle():
    """The whole C5 workload (six grids, 1680 pairs and six projections) as one
    graph replay; each grid's replayed Q equals its individual call bit for
    bit, and one sampled pair per grid matches the oracle (FP32 gate 1e-5)."""
    import torch
    B = require_gpu()
    grids, items, fields = [], [], []
    for i, (N, d, gamma, M, r) in enumerate(C5_GRIDS):
        g = B.boltz_grid_init(N, d, 8.0, 8.0, gamma, N, M)
        grids.append(g)
        V = as_fp32(W.hermite_maxwellian_basis(N, d, 8.0, r, seed=2114 + i))
        fields.append(V)
        f = torch.tensor(V, dtype=torch.float32, device="cuda")
        pj = [j for j in range(r) for _ in range(r)]
        pl = [l for _ in range(r) for l in range(r)]
        items.append(dict(grid=g, fields=f, spectra=torch.zeros((r,) + g.half_shape, dtype=torch.complex64,
                                                                device="cuda"),
                          pair_j=pj, pair_l=pl, Q_out=torch.full((r * r,) + g.shape, float("nan"), device="cuda"),
                          V=f, T_out=torch.full((r, r, r), float("nan"), device="cuda")))
    batch = B.boltz_batch_plan(items)
    try:
        B.boltz_batch_run(batch)
        torch.cuda.synchronize()
        for g in grids:
            B.boltz_sync_status(g)
        replayed = [it["Q_out"].clone() for it in items]
    finally:
        batch.close()
    for i, ((N, d, gamma, M, r), g, it) in enumerate(zip(C5_GRIDS, grids, items)):
        spec = B.boltz_spectrum(g, it["fields"])
        Q1 = B.boltz_collide_batched(g, spec, it["pair_j"], it["pair_l"])
        B.boltz_sync_status(g)
        assert torch.equal(replayed[i], Q1), i
        if C5_SAMPLES[i] is None:
            continue
        a, b = C5_SAMPLES[i]
        sub = sorted({a, b})
        loc = {k: n for n, k in enumerate(sub)}
        _, Qo, s = oracle_collide((N, d, 8.0, 8.0, gamma, N, M), fields[i][sub], [(loc[a], loc[b])])
        Qg = replayed[i][a * r + b].cpu().numpy().astype(np.float64)[None]
        assert rel_err(Qg, Qo, s).max() < 1e-5, i
    for g in grids:
        g.close()
