"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded (FP32-rounded) inputs."""
import numpy as np
import pytest


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU parity tests need a CUDA device")
    from paper_2112_02695_gb300 import build
    build.build()
    from paper_2112_02695_gb300 import boltz
    return boltz


def as_fp32(x):
    """Inputs are generated in FP64 and rounded once to FP32; both sides get these values."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def gpu_collide(B, cfg, fields, pairs, form=0, return_T=False, schedule=0, launches=None, loss=0):
    """Q (and T) from the library.  `launches`, when a dict, receives the
    per-class launch counts of the call (to check which schedule ran)."""
    import torch
    N, d, L, R, gamma, n_rho, M = cfg
    g = B.boltz_grid_init(N, d, L, R, gamma, n_rho, M, schedule=schedule, loss=loss)
    try:
        f = torch.tensor(np.asarray(fields, dtype=np.float32), device="cuda")
        spec = B.boltz_spectrum(g, f)
        pj = [p[0] for p in pairs]
        pl = [p[1] for p in pairs]
        Q = B.boltz_collide_batched(g, spec, pj, pl, form=form)
        T = B.boltz_project(g, f, Q) if return_T else None
        B.boltz_sync_status(g)
        if launches is not None:
            launches.update({k: c for k, (c, _) in B.boltz_profile_read(g, reset=True).items()})
        torch.cuda.synchronize()
        out = Q.cpu().numpy().astype(np.float64)
        return (out, T.cpu().numpy().astype(np.float64)) if return_T else out
    finally:
        g.close()


def oracle_collide(cfg, fields, pairs, loss="exact"):
    from oracle import collision as C
    N, d, L, R, gamma, n_rho, M = cfg
    prob = C.Problem(N=N, d=d, L=L, R=R, gamma=gamma, n_rho=n_rho, M=M, loss=loss)
    Q, Qp, Qm = C.collide_fields(prob, fields, pairs, return_parts=True)
    return prob, Q, C.scale(Q, Qp, Qm)


def rel_err(gpu, ref, s):
    """Per-result relative L-infinity error, normalised by the oracle scale s."""
    ax = tuple(range(1, np.ndim(ref)))
    return np.max(np.abs(gpu - ref), axis=ax) / s
