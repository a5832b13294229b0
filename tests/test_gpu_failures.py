"""Failure paths of the C ABI, caused on the host or by ordinary inputs (no
GPU fault, trap or hang): non-finite inputs reported as BOLTZ_ENONFINITE, a
workspace cap too small for the batch (BOLTZ_ENOMEM), and the host-side fault
injection of the BOLTZ_FAULT environment variable (alloc, badplan, nan).
After every failure the grid is used again and must work."""
import numpy as np
import pytest

from gpu_helpers import require_gpu
from paper_2112_02695_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PAIRS = ([0, 1, 2, 1, 0], [0, 2, 1, 1, 2])
GRIDS = {
    "3d16": (16, 3, 8.0, 8.0, 1.0, 4, 14),      # single-CTA field kernels
    "3d32": (32, 3, 8.0, 8.0, 1.0, 2, 14),      # pipelined schedule
    "2d32": (32, 2, 8.0, 8.0, 0.0, 4, 8),
}


@pytest.fixture(scope="module")
def B():
    return require_gpu()


def _spectra(B, g, cfg, nan=False):
    import torch
    N, d = cfg[0], cfg[1]
    V = np.asarray(W.hermite_maxwellian_basis(N, d, 8.0, 3, seed=3), dtype=np.float32)
    if nan:
        V[1].flat[V[1].size // 3] = np.nan
    return B.boltz_spectrum(g, torch.tensor(V, device="cuda"))


def _status(B, fn):
    try:
        fn()
    except B.BoltzError as e:
        return e.status
    return B.BOLTZ_OK


@pytest.mark.parametrize("name", sorted(GRIDS))
@pytest.mark.parametrize("form", [0, 3])
def test_nonfinite_input_is_reported(B, name, form):
    """A NaN in one input: the pairs that use it write NaN, boltz_sync_status
    reports BOLTZ_ENONFINITE once, and the next finite batch is clean."""
    cfg = GRIDS[name]
    if form == 3 and abs(cfg[4] - (cfg[1] - 2)) > 1e-12:
        pytest.skip("the Carleman form needs gamma = d - 2")
    g = B.boltz_grid_init(*cfg)
    try:
        Q = B.boltz_collide_batched(g, _spectra(B, g, cfg, nan=True), *PAIRS, form=form)
        assert _status(B, lambda: B.boltz_sync_status(g)) == B.BOLTZ_ENONFINITE
        q = Q.cpu().numpy()
        assert np.isfinite(q[0]).all() and np.isnan(q[1]).any()
        assert _status(B, lambda: B.boltz_sync_status(g)) == B.BOLTZ_OK
        Q = B.boltz_collide_batched(g, _spectra(B, g, cfg), *PAIRS, form=form)
        B.boltz_sync_status(g)
        assert np.isfinite(Q.cpu().numpy()).all()
    finally:
        g.close()


def test_workspace_cap_reports_enomem(B):
    """workspace_max below the batch's workspace: BOLTZ_ENOMEM, nothing queued,
    and the same batch runs on a grid without the cap."""
    cfg = GRIDS["3d32"]
    g = B.boltz_grid_init(*cfg, workspace_max=1 << 20)
    try:
        spec = _spectra(B, g, cfg)
        need = B.boltz_workspace_size(g, spec.shape[0], *PAIRS)
        assert need > (1 << 20)
        assert _status(B, lambda: B.boltz_collide_batched(g, spec, *PAIRS)) == B.BOLTZ_ENOMEM
        assert _status(B, lambda: B.boltz_sync_status(g)) == B.BOLTZ_OK
    finally:
        g.close()
    g = B.boltz_grid_init(*cfg)
    try:
        B.boltz_collide_batched(g, _spectra(B, g, cfg), *PAIRS)
        B.boltz_sync_status(g)
    finally:
        g.close()


@pytest.mark.parametrize("fault,expect_call,expect_sync", [
    ("alloc", "BOLTZ_ENOMEM", "BOLTZ_OK"),
    ("badplan", "BOLTZ_EINVAL", "BOLTZ_OK"),
    ("nan", "BOLTZ_OK", "BOLTZ_ENONFINITE"),
])
def test_host_fault_injection(B, monkeypatch, fault, expect_call, expect_sync):
    cfg = GRIDS["3d16"]
    g = B.boltz_grid_init(*cfg)
    try:
        spec = _spectra(B, g, cfg)
        monkeypatch.setenv("BOLTZ_FAULT", fault)
        assert _status(B, lambda: B.boltz_collide_batched(g, spec, *PAIRS)) == getattr(B, expect_call)
        assert _status(B, lambda: B.boltz_sync_status(g)) == getattr(B, expect_sync)
        monkeypatch.delenv("BOLTZ_FAULT")
        Q = B.boltz_collide_batched(g, spec, *PAIRS)
        B.boltz_sync_status(g)
        assert np.isfinite(Q.cpu().numpy()).all()
    finally:
        g.close()
