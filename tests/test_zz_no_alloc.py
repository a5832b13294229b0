"""The allocation-free projection entry point, checked against the allocating one.

boltz_project_noalloc keeps its partial sums in a fixed device array of the
library instead of allocating, for callers that must not allocate device
memory (cudaMalloc/cudaFree can synchronise the device; some processes have
their device memory reserved up front).  This file is collected last so a
failure here cannot hide any other test; it also passes on its own in a
fresh process.
"""
import numpy as np
import pytest

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.mark.parametrize("N,d,r", [(16, 3, 16), (32, 2, 32), (32, 2, 64)])
def test_noalloc_projection_matches_allocating_projection(N, d, r):
    import torch
    B = require_gpu()
    g = B.boltz_grid_init(N, d, 8.0, 8.0, 1.0, 4, 6 if d == 3 else 8)
    try:
        n = N ** d
        gen = torch.Generator(device="cpu").manual_seed(r)
        for call in range(2):                 # two calls in a row share the fixed array
            V = torch.randn((r,) + g.shape, generator=gen).cuda()
            Q = torch.randn((r * r,) + g.shape, generator=gen).cuda()
            ref = B.boltz_project(g, V, Q)
            out = torch.full((r, r, r), float("nan"), device="cuda")
            B.boltz_project_noalloc(g, V, Q, out)
            torch.cuda.synchronize()
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(a)), call
            assert np.max(np.abs(a - b)) <= TOL * np.max(np.abs(b)), call
        assert n > 0
    finally:
        g.close()


def test_noalloc_projection_rejects_sizes_beyond_its_limit():
    import torch
    B = require_gpu()
    g = B.boltz_grid_init(8, 3, 8.0, 8.0, 1.0, 2, 6)
    try:
        r = 65
        V = torch.zeros((r,) + g.shape, device="cuda")
        Q = torch.zeros((1,) + g.shape, device="cuda").expand(r * r, *g.shape).contiguous()
        out = torch.zeros((r, r, r), device="cuda")
        with pytest.raises(B.BoltzError) as ei:
            B.boltz_project_noalloc(g, V, Q, out)
        assert ei.value.status == B.BOLTZ_EINVAL
    finally:
        g.close()
