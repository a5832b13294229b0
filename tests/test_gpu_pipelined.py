"""GPU parity of the pipelined schedule of the batched form (3D 32^3 grids,
at most 16 distinct inputs): axis-0 and axis-1 inverse passes shared by the
directions with equal sigma_0 and (sigma_0, sigma_1), the last inverse pass
fused with the sigma-contraction and the first forward pass, all radial nodes
in one persistent kernel.

Against the FP64 oracle at quadratures small enough for the oracle (every
built direction rule, so every shape of the direction tree), with ragged and
repeated pair lists; against the node-block schedule on the full 256-pair
rank-16 batch; bit-for-bit reproducible across calls (every sum has a fixed
order).  Tolerance: relative L-infinity 1e-5 of the oracle's per-result scale
s = max(max|Q|, max|Q+|, max|Q-|).
"""
import numpy as np
import pytest

from gpu_helpers import as_fp32, gpu_collide, oracle_collide, rel_err, require_gpu
from paper_2112_02695_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def B():
    return require_gpu()


@pytest.mark.parametrize("M,n_rho,r", [(38, 3, 4), (6, 2, 3), (14, 1, 5), (26, 2, 2), (50, 1, 3), (86, 1, 2)])
def test_pipelined_against_oracle(B, M, n_rho, r):
    """All r^2 ordered pairs of a Hermite-Maxwellian basis, every direction rule."""
    cfg = (32, 3, 8.0, 8.0, 1.0, n_rho, M)
    V = as_fp32(W.hermite_maxwellian_basis(32, 3, 8.0, r, seed=40 + M))
    pairs = [(j, l) for j in range(r) for l in range(r)]
    launches = {}
    Qg = gpu_collide(B, cfg, V, pairs, launches=launches)
    assert launches["pipeline"] == 1 and launches["shift"] == 0
    _, Qo, s = oracle_collide(cfg, V, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL


def test_pipelined_ragged_pair_list(B):
    """Inputs used out of order and not all of them, a pair list with
    repeats, reversed pairs and diagonal pairs, gamma = 0, L != R."""
    cfg = (32, 3, 7.0, 6.0, 0.0, 2, 38)
    F = as_fp32(W.random_fields(32, 3, 7.0, 9, seed=31))
    pairs = [(8, 2), (2, 8), (5, 5), (0, 7), (7, 0), (8, 2), (3, 3), (2, 5), (0, 0)]
    launches = {}
    Qg = gpu_collide(B, cfg, F, pairs, launches=launches)
    assert launches["pipeline"] == 1
    _, Qo, s = oracle_collide(cfg, F, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL


def test_pipelined_sixteen_inputs_against_oracle(B):
    """A full chunk: 16 inputs, the 136 unordered gain slots, sampled ordered pairs."""
    cfg = (32, 3, 8.0, 8.0, 1.0, 1, 14)
    V = as_fp32(W.hermite_maxwellian_basis(32, 3, 8.0, 16, seed=16))
    rng = np.random.default_rng(16)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, 16, size=(24, 2))] + [(15, 15), (0, 15), (15, 0)]
    Qg = gpu_collide(B, cfg, V, pairs)
    _, Qo, s = oracle_collide(cfg, V, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL


def test_pipelined_equals_node_blocks_on_the_rank16_batch(B):
    """The 256-pair rank-16 batch at the full quadrature (N_rho = 32, M = 38):
    both schedules compute the same quadrature, so they agree to FP32
    rounding (gate 1e-5 of each result's largest value)."""
    cfg = (32, 3, 8.0, 8.0, 1.0, 32, 38)
    V = as_fp32(W.hermite_maxwellian_basis(32, 3, 8.0, 16, seed=2112))
    pairs = [(j, l) for j in range(16) for l in range(16)]
    lp, ln = {}, {}
    Qp = gpu_collide(B, cfg, V, pairs, launches=lp)
    Qn = gpu_collide(B, cfg, V, pairs, schedule=1, launches=ln)
    assert lp["pipeline"] == 1 and ln["pipeline"] == 0 and ln["shift"] > 0
    scale = np.max(np.abs(Qn), axis=(1, 2, 3))
    assert (np.max(np.abs(Qp - Qn), axis=(1, 2, 3)) / scale).max() < TOL


def test_pipelined_is_bitwise_reproducible(B):
    """Every reduction of the pipelined schedule has a fixed order: two calls
    on the same inputs give identical bits."""
    import torch
    cfg = (32, 3, 8.0, 8.0, 1.0, 4, 38)
    V = np.asarray(W.hermite_maxwellian_basis(32, 3, 8.0, 6, seed=6), dtype=np.float32)
    pairs = [(j, l) for j in range(6) for l in range(6)]
    g = B.boltz_grid_init(*cfg)
    try:
        spec = B.boltz_spectrum(g, torch.tensor(V, device="cuda"))
        pj, pl = [p[0] for p in pairs], [p[1] for p in pairs]
        Q1 = B.boltz_collide_batched(g, spec, pj, pl).clone()
        Q2 = B.boltz_collide_batched(g, spec, pj, pl)
        B.boltz_sync_status(g)
        assert torch.equal(Q1, Q2)
    finally:
        g.close()


def test_pipelined_several_chunks_against_oracle(B):
    """40 inputs whose pairs connect groups of at most 16 (diagonal cells, a few
    pairs within groups): chunks of at most 16 inputs, each with its own gain
    slots; here the three chunks differ in shape, so each has a launch."""
    cfg = (32, 3, 8.0, 8.0, 1.0, 2, 14)
    f = as_fp32(W.random_fields(32, 3, 8.0, 40, seed=801))
    pairs = [(x, x) for x in range(40)] + [(0, 1), (1, 0), (5, 7), (30, 31), (39, 38), (12, 12)]
    launches = {}
    Qg = gpu_collide(B, cfg, f, pairs, launches=launches)
    assert launches["pipeline"] == 3 and launches["shift"] == 0        # 40 inputs: chunks of 16, 16, 8
    _, Qo, s = oracle_collide(cfg, f, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL


def test_pipelined_falls_back_for_a_group_of_seventeen(B):
    """A chain of pairs joining 17 inputs cannot be split into chunks of 16:
    the node-block schedule runs it, with the same result."""
    cfg = (32, 3, 8.0, 8.0, 1.0, 1, 6)
    f = as_fp32(W.random_fields(32, 3, 8.0, 17, seed=802))
    pairs = [(x, x + 1) for x in range(16)]
    launches = {}
    Qg = gpu_collide(B, cfg, f, pairs, launches=launches)
    assert launches["pipeline"] == 0 and launches["shift"] > 0
    _, Qo, s = oracle_collide(cfg, f, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL


@pytest.mark.parametrize("n_rho,diag", [(1, True), (3, True), (3, False)])
def test_pipelined_chunks_of_one_shape_share_a_launch(B, n_rho, diag):
    """48 inputs in three chunks of one shape (diagonal pairs only, or pairs
    (2i, 2i+1) both ways plus the diagonal): one persistent launch runs the
    node lists of all three chunks one after another, so with N_rho = 3 the
    node buffers are reused across chunk boundaries."""
    cfg = (32, 3, 8.0, 8.0, 1.0, n_rho, 14)
    f = as_fp32(W.random_fields(32, 3, 8.0, 48, seed=803 + n_rho))
    if diag:
        pairs = [(x, x) for x in range(48)]
    else:
        pairs = [p for i in range(24) for p in ((2 * i, 2 * i + 1), (2 * i + 1, 2 * i), (2 * i, 2 * i))]
    launches = {}
    Qg = gpu_collide(B, cfg, f, pairs, launches=launches)
    assert launches["pipeline"] == 1 and launches["shift"] == 0
    _, Qo, s = oracle_collide(cfg, f, pairs)
    assert rel_err(Qg, Qo, s).max() < TOL


def test_pipelined_caps_the_chunks_of_a_launch(B):
    """1056 diagonal pairs: 66 chunks of one shape, at most 64 in a launch, so
    two launches; the result equals the node-block schedule's."""
    cfg = (32, 3, 8.0, 8.0, 1.0, 1, 6)
    f = as_fp32(W.random_fields(32, 3, 8.0, 1056, seed=804))
    pairs = [(x, x) for x in range(1056)]
    lp, ln = {}, {}
    Qp = gpu_collide(B, cfg, f, pairs, launches=lp)
    Qn = gpu_collide(B, cfg, f, pairs, schedule=1, launches=ln)
    assert lp["pipeline"] == 2 and ln["pipeline"] == 0
    scale = np.max(np.abs(Qn), axis=(1, 2, 3))
    assert (np.max(np.abs(Qp - Qn), axis=(1, 2, 3)) / scale).max() < TOL
