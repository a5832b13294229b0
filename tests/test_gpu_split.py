"""GPU parity of the split-precision form (BF16x3 DFT-as-GEMM shifted fields
on the tensor cores) against the FP64 oracle.

Gate: relative L-infinity error <= 1e-3 of the per-result scale
s = max(max|Q|, max|Q+|, max|Q-|) of the oracle.  The tests also record that
the measured error sits far below the gate (the BF16 pair keeps ~16
significant bits; the dropped lo*lo term is ~2^-17 relative).
"""
import numpy as np
import pytest

from gpu_helpers import as_fp32, gpu_collide, oracle_collide, rel_err, require_gpu
from paper_2112_02695_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL_SPLIT = 1e-3
SPLIT = 2


@pytest.fixture(scope="module")
def B():
    return require_gpu()


def test_split_small_quadrature_all_pairs(B):
    """32^3, N_rho=4 x M=14, rank 4: all ordered pairs (triangular-tile and
    list slots) in the split form against the oracle and against the FP32
    batched form."""
    cfg = (32, 3, 8.0, 8.0, 1.0, 4, 14)
    V = as_fp32(W.hermite_maxwellian_basis(32, 3, 8.0, 4, seed=31))
    pairs = [(j, l) for j in range(4) for l in range(4)]
    Qs = gpu_collide(B, cfg, V, pairs, form=SPLIT)
    Qf = gpu_collide(B, cfg, V, pairs, form=0)
    _, Qo, s = oracle_collide(cfg, V, pairs)
    e_split = rel_err(Qs, Qo, s).max()
    assert e_split < TOL_SPLIT
    assert e_split < 2e-4          # the split keeps ~16 bits: far inside the gate
    assert rel_err(Qf, Qo, s).max() < 1e-5


def test_split_random_fields_mixed_pairs_several_node_blocks(B):
    """Unstructured inputs (every mode populated), duplicate and reversed
    pairs, and a field budget small enough that the radial nodes run in
    several blocks."""
    import torch
    cfg = (32, 3, 8.0, 8.0, 0.0, 6, 6)
    F = as_fp32(W.random_fields(32, 3, 8.0, 5, seed=32))
    pairs = [(0, 1), (1, 0), (4, 4), (2, 3), (0, 1), (3, 4)]
    g = B.boltz_grid_init(32, 3, 8.0, 8.0, 0.0, 6, 6, field_budget_mb=4)
    try:
        f = torch.tensor(F, dtype=torch.float32, device="cuda")
        spec = B.boltz_spectrum(g, f)
        Q = B.boltz_collide_batched(g, spec, [p[0] for p in pairs], [p[1] for p in pairs], form=SPLIT)
        B.boltz_sync_status(g)
        Qs = Q.cpu().numpy().astype(np.float64)
    finally:
        g.close()
    _, Qo, s = oracle_collide(cfg, F, pairs)
    assert rel_err(Qs, Qo, s).max() < TOL_SPLIT


def test_split_full_size_c2_sampled_pairs(B):
    """C2 workload (32^3, N_rho=32 x M=38, rank 16, seed 2112) in the split
    form: sampled pairs against the oracle."""
    cfg = (32, 3, 8.0, 8.0, 1.0, 32, 38)
    V = as_fp32(W.hermite_maxwellian_basis(32, 3, 8.0, 16, seed=2112))
    pairs = [(j, l) for j in range(16) for l in range(16)]
    Qs, Ts = gpu_collide(B, cfg, V, pairs, form=SPLIT, return_T=True)
    for j, l in [(0, 0), (3, 11), (15, 2)]:
        _, Qo, s = oracle_collide(cfg, V[[j, l]], [(0, 1)] if j != l else [(0, 0)])
        assert rel_err(Qs[j * 16 + l][None], Qo, s).max() < TOL_SPLIT, (j, l)
    T64 = 0.5 ** 3 * V.reshape(16, -1) @ Qs.reshape(256, -1).T
    assert np.max(np.abs(Ts.reshape(16, 256) - T64)) / np.max(np.abs(T64)) < 1e-5


def test_split_64cube_small_quadrature(B):
    """64^3 on [-10,10]^3 (8-CTA clusters per field, the pass-2 -> 3 operand
    exchanged through distributed shared memory), N_rho=2 x M=6."""
    cfg = (64, 3, 10.0, 10.0, 1.0, 2, 6)
    F = as_fp32(W.random_fields(64, 3, 10.0, 2, seed=64))
    pairs = [(0, 1), (1, 0), (1, 1)]
    Qs = gpu_collide(B, cfg, F, pairs, form=SPLIT)
    _, Qo, s = oracle_collide(cfg, F, pairs)
    assert rel_err(Qs, Qo, s).max() < TOL_SPLIT


def test_split_c4_full_size_matches_fp32_form(B):
    """C4 workload (64^3, N_rho=32 x M=86, rank 8, seed 2113): all 64 pairs in
    the split form against the FP32 batched form (which meets 1e-5 against the
    oracle's gain symmetry and bilinearity in the FP32 parity tests)."""
    cfg = (64, 3, 10.0, 10.0, 1.0, 32, 86)
    V = as_fp32(W.hermite_maxwellian_basis(64, 3, 10.0, 8, seed=2113))
    pairs = [(j, l) for j in range(8) for l in range(8)]
    Qs = gpu_collide(B, cfg, V, pairs, form=SPLIT)
    Qf = gpu_collide(B, cfg, V, pairs, form=0)
    scale = np.max(np.abs(Qf), axis=(1, 2, 3))
    assert (np.max(np.abs(Qs - Qf), axis=(1, 2, 3)) / scale).max() < TOL_SPLIT


def test_split_form_rejected_where_not_built(B):
    import torch
    g = B.boltz_grid_init(16, 3, 8.0, 8.0, 1.0, 2, 6)
    try:
        f = torch.tensor(W.random_fields(16, 3, 8.0, 2, seed=3), dtype=torch.float32, device="cuda")
        spec = B.boltz_spectrum(g, f)
        with pytest.raises(B.BoltzError) as ei:
            B.boltz_collide_batched(g, spec, [0], [1], form=SPLIT)
        assert ei.value.status == B.BOLTZ_EUNSUPPORTED
        Q = B.boltz_collide_batched(g, spec, [0], [1], form=0)      # the grid stays usable
        B.boltz_sync_status(g)
        assert torch.isfinite(Q).all()
    finally:
        g.close()
