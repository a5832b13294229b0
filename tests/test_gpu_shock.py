"""GPU parity of the 1D normal-shock solver (boltz_shock_*) against
oracle/shock.py: the full-tensor upwind steps and the adaptive low-rank steps
(add basis, K-, S-, L-steps, drop, the Sec. 5.1 convergence measure), 2D
velocity grid 16^2 on [-10, 10]^2,
Maxwell molecules, 16 cells on [-6, 6], Mach 1.4.

The GPU keeps every factor in FP64; the collision terms come from the FP32
batch (relative error ~1e-6 of their scale), so the gate is on the change of
f over the steps: max |f_gpu - f_oracle| <= 1e-5 x max |f_oracle - f_0|
(full tensor) and 1e-4 x (low rank, whose K-, S- and L-step collision terms
pass through FP32 couplings as well).  The ranks after every drop must be
equal; the drop tolerances are chosen a factor >= 3 away from every singular
value the oracle produces."""
import numpy as np
import pytest

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu
N_X, N, L_X, DT = 16, 16, 6.0, 0.005


def make(B, mach=1.4, r_max=16, form=0, d=2):
    from oracle import carleman as CM
    from oracle import collision as C
    from oracle import shock as SH
    if d == 3:         # 3D hard spheres, 16^3 on [-10, 10]^3, N_rho = 4 x M = 14
        vel = C.Problem(N=N, d=3, L=10.0, R=10.0, gamma=1.0, n_rho=4, M=14)
        sp = SH.ShockProblem(vel=vel, n_x=12, L_x=L_X, mach=mach)
        g = B.boltz_grid_init(N, 3, 10.0, 10.0, 1.0, 4, 14)
        fL, fR = sp.boundary()
        return sp, g, B.boltz_shock_create(g, 12, L_X, fL, fR, r_max, form)
    vel = C.Problem(N=N, d=2, L=10.0, R=10.0, gamma=0.0, n_rho=6, M=12)
    if form == 3:      # the Carleman (Mouhot-Pareschi) form the paper's experiments use: R = 6, 16 directions
        sp = SH.ShockProblem(vel=vel, n_x=N_X, L_x=L_X, mach=mach,
                             carleman=CM.CarlemanProblem(N=N, d=2, L=10.0, R=6.0, M=16))
        g = B.boltz_grid_init(N, 2, 10.0, 6.0, 0.0, 1, 16)
    else:
        sp = SH.ShockProblem(vel=vel, n_x=N_X, L_x=L_X, mach=mach)
        g = B.boltz_grid_init(N, 2, 10.0, 10.0, 0.0, 6, 12)
    fL, fR = sp.boundary()
    return sp, g, B.boltz_shock_create(g, N_X, L_X, fL, fR, r_max, form)


def test_full_tensor_steps_match_oracle():
    import torch
    from oracle import shock as SH
    B = require_gpu()
    sp, g, sh = make(B)
    try:
        f0 = sp.initial()
        f = torch.tensor(f0, dtype=torch.float64, device="cuda")
        B.boltz_shock_full_step(sh, f, 3, DT)
        torch.cuda.synchronize()
        got = f.cpu().numpy()
    finally:
        sh.close()
        g.close()
    want = f0.copy()
    for _ in range(3):
        want = SH.full_step(sp, want, DT)
    assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want - f0))


def _lowrank_run(B, drop_tol, steps, r0=4, mach=1.4, form=0, d=2):
    import torch
    from oracle import shock as SH
    sp, g, sh = make(B, mach=mach, form=form, d=d)
    n_x, n_v = sp.n_x, N ** d
    try:
        f0 = sp.initial()
        X, S, V = SH.factor(sp, f0, r0)
        rm = sh.r_max
        Xd = torch.zeros((rm, n_x), dtype=torch.float64, device="cuda")
        Vd = torch.zeros((rm, n_v), dtype=torch.float64, device="cuda")
        Sd = torch.zeros(rm * rm, dtype=torch.float64, device="cuda")
        Xd[:r0] = torch.tensor(X)
        Vd[:r0] = torch.tensor(V)
        Sd[: r0 * r0] = torch.tensor(S.ravel())
        r = r0
        fd = torch.empty((n_x, n_v), dtype=torch.float64, device="cuda")
        out = []
        for step in range(steps):
            (X, S, V), parts = SH.lowrank_step(sp, X, S, V, DT, drop_tol, SH.random_xh(n_x, seed=step),
                                               return_parts=True)
            sig = parts["sigma"]
            assert np.min(np.abs(np.log10(sig[sig > 0] / drop_tol))) > np.log10(3.0)
            r, err = B.boltz_shock_lowrank_step(sh, Xd, Sd, Vd, r, DT, drop_tol)
            B.boltz_shock_reconstruct(sh, Xd, Sd, Vd, r, fd)
            torch.cuda.synchronize()
            # the step's convergence measure (Sec. 5.1) against the oracle's
            assert abs(err - parts["err"]) <= 1e-3 * parts["err"], (err, parts["err"])
            out.append((r, S.shape[0], fd.cpu().numpy(), SH.reconstruct(X, S, V)))
        Xg = Xd[:r].cpu().numpy()
        Vg = Vd[:r].cpu().numpy()
        return sp, f0, out, Xg, Vg
    finally:
        sh.close()
        g.close()


def test_lowrank_steps_match_oracle_fixed_rank():
    """drop_tol between sigma_4 and sigma_5: the two added boundary directions
    are dropped again every step, the rank stays 4."""
    B = require_gpu()
    sp, f0, out, Xg, Vg = _lowrank_run(B, 1e-5, 3)
    for r_gpu, r_orc, fg, fo in out:
        assert r_gpu == r_orc == 4
        assert np.max(np.abs(fg - fo)) <= 1e-4 * np.max(np.abs(fo - f0))
    # the returned bases are orthonormal under the midpoint rules
    assert np.allclose(sp.dx * Xg @ Xg.T, np.eye(len(Xg)), atol=1e-11)
    assert np.allclose(sp.wv * Vg @ Vg.T, np.eye(len(Vg)), atol=1e-11)


def test_lowrank_steps_match_oracle_growing_rank():
    """A small drop_tol keeps the new boundary information: the rank grows by
    two per step (4 -> 6 -> 8)."""
    B = require_gpu()
    sp, f0, out, Xg, Vg = _lowrank_run(B, 1e-7, 2)
    assert [o[0] for o in out] == [o[1] for o in out] == [6, 8]
    for r_gpu, r_orc, fg, fo in out:
        assert np.max(np.abs(fg - fo)) <= 1e-4 * np.max(np.abs(fo - f0))


def test_carleman_form_full_and_lowrank_steps_match_oracle():
    """The same solver on the Carleman (Mouhot-Pareschi) form of Q, the
    method of the paper's own experiments (2D Maxwell molecules)."""
    import torch
    from oracle import shock as SH
    B = require_gpu()
    sp, g, sh = make(B, form=3)
    try:
        f0 = sp.initial()
        f = torch.tensor(f0, dtype=torch.float64, device="cuda")
        B.boltz_shock_full_step(sh, f, 2, DT)
        torch.cuda.synchronize()
        got = f.cpu().numpy()
    finally:
        sh.close()
        g.close()
    want = f0.copy()
    for _ in range(2):
        want = SH.full_step(sp, want, DT)
    assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want - f0))
    sp, f0, out, Xg, Vg = _lowrank_run(B, 1e-5, 2, form=3)
    for r_gpu, r_orc, fg, fo in out:
        assert r_gpu == r_orc
        assert np.max(np.abs(fg - fo)) <= 1e-4 * np.max(np.abs(fo - f0))


def test_3d_hard_spheres_full_and_lowrank_steps_match_oracle():
    """The same solver on a 3D velocity grid (16^3, hard spheres, 12 cells):
    two full-tensor steps and two low-rank steps with the rank growing 3 -> 5 -> 7."""
    import torch
    from oracle import shock as SH
    B = require_gpu()
    sp, g, sh = make(B, d=3)
    try:
        f0 = sp.initial()
        f = torch.tensor(f0, dtype=torch.float64, device="cuda")
        B.boltz_shock_full_step(sh, f, 2, DT)
        torch.cuda.synchronize()
        got = f.cpu().numpy()
    finally:
        sh.close()
        g.close()
    want = f0.copy()
    for _ in range(2):
        want = SH.full_step(sp, want, DT)
    assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want - f0))
    sp, f0, out, Xg, Vg = _lowrank_run(B, 3e-7, 2, r0=3, d=3)
    assert [o[0] for o in out] == [o[1] for o in out] == [5, 7]
    for r_gpu, r_orc, fg, fo in out:
        assert np.max(np.abs(fg - fo)) <= 1e-4 * np.max(np.abs(fo - f0))


def _paper_size(B, form=0):
    """The benchmark's shock: Mach 1.4, 1000 cells on [-30, 30], 2D 32^2 on [-13.11, 13.11]^2."""
    from oracle import collision as C
    from oracle import shock as SH
    vel = C.Problem(N=32, d=2, L=13.11, R=13.11, gamma=0.0, n_rho=16, M=16)
    sp = SH.ShockProblem(vel=vel, n_x=1000, L_x=30.0, mach=1.4)
    g = B.boltz_grid_init(32, 2, 13.11, 13.11, 0.0, 16, 16)
    fL, fR = sp.boundary()
    return sp, g, B.boltz_shock_create(g, 1000, 30.0, fL, fR, 64, form)


def test_full_size_full_tensor_step_sampled_cells():
    """One full-tensor step at the benchmark size; cells at both boundaries and
    in the shock are checked one by one (a cell's upwind update needs only its
    neighbours and its own Q(f, f))."""
    import torch
    from oracle import shock as SH
    B = require_gpu()
    sp, g, sh = _paper_size(B)
    try:
        f0 = sp.initial()
        f = torch.tensor(f0, dtype=torch.float64, device="cuda")
        B.boltz_shock_full_step(sh, f, 1, 0.004)
        torch.cuda.synchronize()
        got = f.cpu().numpy()
    finally:
        sh.close()
        g.close()
    fL, fR = sp.boundary()
    v1 = sp.v1()
    vp, vm = np.maximum(v1, 0.0), np.minimum(v1, 0.0)
    from oracle import collision as C
    for p in (0, 1, 480, 500, 520, 998, 999):
        left = fL if p == 0 else f0[p - 1]
        right = fR if p == sp.n_x - 1 else f0[p + 1]
        Q, Qp, Qm = C.collide_fields(sp.vel, f0[p].reshape(1, 32, 32), [(0, 0)], return_parts=True)
        want = f0[p] - 0.004 * (vp * (f0[p] - left) + vm * (right - f0[p])) / sp.dx + 0.004 * Q[0].reshape(-1)
        # FP32 collision term: its rounding scales with max(|Q|, |Q+|, |Q-|) of the cell,
        # which near the boundaries (close to equilibrium) dwarfs the change of f
        gate = 1e-5 * (np.max(np.abs(want - f0[p])) + 0.004 * float(C.scale(Q, Qp, Qm)[0]))
        assert np.max(np.abs(got[p] - want)) <= gate, p


def test_full_size_lowrank_step_properties():
    """One low-rank step at the benchmark size from the rank-2 bimodal state:
    orthonormal bases, rank within r + 2, and the Sec. 5.1 measure equal to
    the norm of the change of the rebuilt solution (no drop)."""
    import torch
    B = require_gpu()
    sp, g, sh = _paper_size(B)
    try:
        fL, fR = sp.boundary()
        s = (np.tanh(0.5 * sp.x) + 1.0) / 2.0
        dev = "cuda"
        Yx, Rx, _ = B.boltz_qr_f64(torch.tensor(np.stack([1.0 - s, s]), device=dev), sp.dx)
        Yv, Rv, _ = B.boltz_qr_f64(torch.tensor(np.stack([fL, fR]), device=dev), sp.wv)
        Xd = torch.zeros((64, sp.n_x), dtype=torch.float64, device=dev)
        Vd = torch.zeros((64, 1024), dtype=torch.float64, device=dev)
        Sd = torch.zeros(64 * 64, dtype=torch.float64, device=dev)
        Xd[:2], Vd[:2] = Yx, Yv
        Sd[:4] = (Rx @ Rv.T).reshape(-1)
        f_before = torch.empty((sp.n_x, 1024), dtype=torch.float64, device=dev)
        B.boltz_shock_reconstruct(sh, Xd, Sd, Vd, 2, f_before)
        r, err = B.boltz_shock_lowrank_step(sh, Xd, Sd, Vd, 2, 0.004, 0.0)
        f_after = torch.empty_like(f_before)
        B.boltz_shock_reconstruct(sh, Xd, Sd, Vd, r, f_after)
        torch.cuda.synchronize()
        X, V = Xd[:r].cpu().numpy(), Vd[:r].cpu().numpy()
        direct = float(np.sqrt(sp.dx * sp.wv * ((f_after - f_before) ** 2).sum().item()))
    finally:
        sh.close()
        g.close()
    assert 1 <= r <= 4
    assert np.allclose(sp.dx * X @ X.T, np.eye(r), atol=1e-10)
    assert np.allclose(sp.wv * V @ V.T, np.eye(r), atol=1e-10)
    assert abs(err - direct) <= 1e-8 * direct


def test_large_velocity_grid_lowrank_steps_properties():
    """3D 48^3 velocity grid (110592 points: the L-factor QR takes the
    multi-kernel Cholesky-QR2 path, the K-factor QR of 8 cells the spread
    one, both on the same workspace), three low-rank steps from the rank-2
    bimodal state: orthonormal bases after every step; with no drop (first
    step) the Sec. 5.1 measure equals the norm of the rebuilt change, then
    drop_tol = 0.2 x the previous measure, as in the benchmark."""
    import torch
    from oracle import collision as C
    from oracle import shock as SH
    B = require_gpu()
    vel = C.Problem(N=48, d=3, L=10.0, R=10.0, gamma=1.0, n_rho=2, M=6)
    sp = SH.ShockProblem(vel=vel, n_x=8, L_x=6.0, mach=1.4)
    g = B.boltz_grid_init(48, 3, 10.0, 10.0, 1.0, 2, 6)
    fL, fR = sp.boundary()
    sh = B.boltz_shock_create(g, 8, 6.0, fL, fR, 10, 0)
    nv = 48 ** 3
    try:
        s = (np.tanh(0.5 * sp.x) + 1.0) / 2.0
        dev = "cuda"
        Yx, Rx, _ = B.boltz_qr_f64(torch.tensor(np.stack([1.0 - s, s]), device=dev), sp.dx)
        Yv, Rv, _ = B.boltz_qr_f64(torch.tensor(np.stack([fL, fR]), device=dev), sp.wv)
        Xd = torch.zeros((10, sp.n_x), dtype=torch.float64, device=dev)
        Vd = torch.zeros((10, nv), dtype=torch.float64, device=dev)
        Sd = torch.zeros(100, dtype=torch.float64, device=dev)
        Xd[:2], Vd[:2] = Yx, Yv
        Sd[:4] = (Rx @ Rv.T).reshape(-1)
        r, tol = 2, 0.0
        f_before = torch.empty((sp.n_x, nv), dtype=torch.float64, device=dev)
        f_after = torch.empty_like(f_before)
        for step in range(3):
            B.boltz_shock_reconstruct(sh, Xd, Sd, Vd, r, f_before)
            r_prev = r
            r, err = B.boltz_shock_lowrank_step(sh, Xd, Sd, Vd, r, 0.004, tol)
            torch.cuda.synchronize()
            X, V = Xd[:r].cpu().numpy(), Vd[:r].cpu().numpy()
            assert 1 <= r <= r_prev + 2
            assert np.allclose(sp.dx * X @ X.T, np.eye(r), atol=1e-10)
            assert np.allclose(sp.wv * V @ V.T, np.eye(r), atol=1e-10)
            assert err > 0.0
            if step == 0:
                B.boltz_shock_reconstruct(sh, Xd, Sd, Vd, r, f_after)
                torch.cuda.synchronize()
                direct = float(np.sqrt(sp.dx * sp.wv * ((f_after - f_before) ** 2).sum().item()))
                assert abs(err - direct) <= 1e-8 * direct
            tol = 0.2 * err
    finally:
        sh.close()
        g.close()


def test_uniform_state_stays_uniform():
    """Mach 1 (f_L = f_R, uniform initial Maxwellian): the boundary vector lies
    in span(V) and is not added; the state changes only by dt Q(M, M)."""
    import torch
    from oracle import shock as SH
    B = require_gpu()
    sp, g, sh = make(B, mach=1.0)
    try:
        f0 = sp.initial()
        X, S, V = SH.factor(sp, f0, 1)
        Xd = torch.zeros((sh.r_max, N_X), dtype=torch.float64, device="cuda")
        Vd = torch.zeros((sh.r_max, N * N), dtype=torch.float64, device="cuda")
        Sd = torch.zeros(sh.r_max ** 2, dtype=torch.float64, device="cuda")
        Xd[:1] = torch.tensor(X)
        Vd[:1] = torch.tensor(V)
        Sd[:1] = float(S[0, 0])
        r, _ = B.boltz_shock_lowrank_step(sh, Xd, Sd, Vd, 1, 0.01, 1e-6)
        fd = torch.empty((N_X, N * N), dtype=torch.float64, device="cuda")
        B.boltz_shock_reconstruct(sh, Xd, Sd, Vd, r, fd)
        torch.cuda.synchronize()
        qscale = np.abs(SH.collide_cells(sp, f0[:1])).max()
        assert r == 1
        assert np.max(np.abs(fd.cpu().numpy() - f0)) <= 0.01 * qscale * 1.01 + 1e-12
    finally:
        sh.close()
        g.close()


def test_rejections():
    import torch
    B = require_gpu()
    sp, g, sh = make(B, r_max=6)
    try:
        Xd = torch.zeros((6, N_X), dtype=torch.float64, device="cuda")
        Vd = torch.zeros((6, N * N), dtype=torch.float64, device="cuda")
        Sd = torch.zeros(36, dtype=torch.float64, device="cuda")
        with pytest.raises(B.BoltzError) as ei:
            B.boltz_shock_lowrank_step(sh, Xd, Sd, Vd, 5, DT, 1e-6)      # 5 + 2 > r_max
        assert ei.value.status == B.BOLTZ_EINVAL
        with pytest.raises(B.BoltzError) as ei:
            B.boltz_shock_full_step(sh, torch.zeros((N_X, N * N), dtype=torch.float64, device="cuda"), 1, -1.0)
        assert ei.value.status == B.BOLTZ_EINVAL
    finally:
        sh.close()
        g.close()


@pytest.mark.parametrize("form,start", [(0, "factor"), (3, "factor"), (0, "bimodal")])
def test_replayed_steps_equal_direct_steps(monkeypatch, form, start):
    """Eight low-rank steps on the same buffers: from the third on they replay
    a captured graph; with BOLTZ_SHOCK_GRAPH=0 every step runs directly.  The
    factors, ranks and convergence measures agree bit for bit.  The bimodal
    start (1 - s) f_L + s f_R has f_L, f_R in span(V): replays find a boundary
    vector not kept, write nothing, and the step runs directly."""
    import torch
    from oracle import shock as SH
    B = require_gpu()

    def run():
        sp, g, sh = make(B, form=form)
        n_x, n_v = sp.n_x, N ** 2
        try:
            rm = sh.r_max
            Xd = torch.zeros((rm, n_x), dtype=torch.float64, device="cuda")
            Vd = torch.zeros((rm, n_v), dtype=torch.float64, device="cuda")
            Sd = torch.zeros(rm * rm, dtype=torch.float64, device="cuda")
            if start == "factor":
                X, S, V = SH.factor(sp, sp.initial(), 4)
                r = 4
            else:
                fL, fR = sp.boundary()
                x = -L_X + (np.arange(n_x) + 0.5) * (2 * L_X / n_x)
                s = (np.tanh(0.5 * x) + 1.0) / 2.0
                X, S, V = SH.factor(sp, np.outer(1.0 - s, fL) + np.outer(s, fR), 2)
                r = 2
            Xd[:r] = torch.tensor(X)
            Vd[:r] = torch.tensor(V)
            Sd[: r * r] = torch.tensor(S.ravel())
            hist = []
            for _ in range(8):
                r, err = B.boltz_shock_lowrank_step(sh, Xd, Sd, Vd, r, DT, 1e-7)
                hist.append((r, err))
            torch.cuda.synchronize()
            return hist, Xd.cpu().numpy(), Sd.cpu().numpy(), Vd.cpu().numpy()
        finally:
            sh.close()
            g.close()

    h1, X1, S1, V1 = run()
    monkeypatch.setenv("BOLTZ_SHOCK_GRAPH", "0")
    h2, X2, S2, V2 = run()
    assert h1 == h2
    assert np.array_equal(X1, X2) and np.array_equal(S1, S2) and np.array_equal(V1, V2)
