"""GPU parity of the low-rank step consumers against oracle/lowrank.py.

FP32 contractions (K-step and L-step collision terms): relative error <= 1e-5
of the per-output magnitude scale sum |terms| (the sums cancel, so the scale
is that of the summands).  FP64 steps (QR, SVD truncation, rotation): 1e-11,
plus the defining properties (orthonormality, reconstruction, ordering)."""
import numpy as np
import pytest

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    return require_gpu()


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("r,nx", [(16, 1000), (5, 257), (33, 300), (64, 129), (1, 1)])
def test_kstep_collision(B, r, nx):
    import torch
    from oracle import lowrank as LR
    rng = np.random.default_rng(100 + r)
    T = f32(rng.standard_normal((r, r, r)))
    K = f32(rng.standard_normal((r, nx)))
    got = B.boltz_kstep_collision(torch.tensor(T, dtype=torch.float32, device="cuda"),
                                  torch.tensor(K, dtype=torch.float32, device="cuda")).cpu().numpy()
    want = LR.kstep_collision(T, K)
    scale = LR.kstep_collision(np.abs(T), np.abs(K))
    assert np.max(np.abs(got - want) / scale) < 1e-5


@pytest.mark.parametrize("r,nv", [(16, 32768), (7, 1000), (40, 515), (64, 256)])
def test_lstep_collision(B, r, nv):
    import torch
    from oracle import lowrank as LR
    rng = np.random.default_rng(200 + r)
    Q = f32(rng.standard_normal((r * r, nv)))
    C = f32(rng.standard_normal((r, r, r)))
    got = B.boltz_lstep_collision(torch.tensor(Q, dtype=torch.float32, device="cuda"),
                                  torch.tensor(C, dtype=torch.float32, device="cuda")).cpu().numpy()
    want = LR.lstep_collision(Q, C)
    scale = LR.lstep_collision(np.abs(Q), np.abs(C))
    assert np.max(np.abs(got - want) / scale) < 1e-5


def test_lstep_from_a_real_batch(B):
    """The L-step term built from a real collision batch (3D 16^3, rank 4) and
    a coupling from random X, S equals the oracle's sum_{m,n} E_imn Q(L_m, L_n)."""
    import torch
    from gpu_helpers import as_fp32, gpu_collide
    from oracle import collision as C
    from oracle import lowrank as LR
    from paper_2112_02695_gb300 import workloads as W
    cfg = (16, 3, 8.0, 8.0, 1.0, 4, 14)
    r = 4
    V = as_fp32(W.hermite_maxwellian_basis(16, 3, 8.0, r, seed=11))
    pairs = [(p, q) for p in range(r) for q in range(r)]
    Qg = gpu_collide(B, cfg, V, pairs)
    rng = np.random.default_rng(12)
    S = rng.standard_normal((r, r))
    X = rng.standard_normal((r, 50))
    Cc = f32(LR.lstep_coupling(LR.triple_products(X, 0.02), S))
    G = B.boltz_lstep_collision(torch.tensor(Qg, dtype=torch.float32, device="cuda"),
                                torch.tensor(Cc, dtype=torch.float32, device="cuda")).cpu().numpy()
    prob = C.Problem(N=16, d=3, L=8.0, R=8.0, gamma=1.0, n_rho=4, M=14)
    Lf = np.einsum("mp,p...->m...", S, V)
    QL = C.collide_fields(prob, Lf, [(m, n) for m in range(r) for n in range(r)]).reshape(r, r, -1)
    want = np.einsum("imn,mnv->iv", LR.triple_products(X, 0.02), QL)
    assert np.max(np.abs(G - want)) / np.max(np.abs(want)) < 1e-4


@pytest.mark.parametrize("r,n", [(16, 32768), (16, 1000), (64, 4096), (1, 8), (7, 7)])
def test_qr_f64(B, r, n):
    import torch
    from oracle import lowrank as LR
    rng = np.random.default_rng(300 + r + n)
    W = rng.standard_normal((r, n)) * np.exp(0.5 * rng.standard_normal((r, 1)))
    w = 0.125
    Y, R, info = B.boltz_qr_f64(torch.tensor(W, device="cuda"), w)
    Y, R = Y.cpu().numpy(), R.cpu().numpy()
    assert int(info.item()) == 0
    Yo, Ro = LR.qr_weighted(W, w)
    assert np.max(np.abs(R - Ro)) / np.max(np.abs(Ro)) < 1e-11
    assert np.max(np.abs(Y - Yo)) / np.max(np.abs(Yo)) < 1e-11
    assert np.max(np.abs(w * Y @ Y.T - np.eye(r))) < 1e-12
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)


def test_qr_f64_in_place_and_rank_deficient(B):
    import torch
    from oracle import lowrank as LR
    rng = np.random.default_rng(7)
    W = rng.standard_normal((6, 500))
    Wd = torch.tensor(W, device="cuda")
    Y, R, info = B.boltz_qr_f64(Wd, 0.5, Y=Wd)          # in place
    assert int(info.item()) == 0
    Yo, _ = LR.qr_weighted(W, 0.5)
    assert np.max(np.abs(Y.cpu().numpy() - Yo)) < 1e-11 * np.max(np.abs(Yo))
    Wbad = W.copy()
    Wbad[3] = 2.0 * Wbad[1] - Wbad[0]                   # linearly dependent
    _, _, info = B.boltz_qr_f64(torch.tensor(Wbad, device="cuda"), 0.5)
    assert int(info.item()) > 0


@pytest.mark.parametrize("r", [16, 6, 7, 64, 1])
def test_svd_truncate_f64(B, r):
    import torch
    from oracle import lowrank as LR
    rng = np.random.default_rng(400 + r)
    U0, _ = np.linalg.qr(rng.standard_normal((r, r)))
    Q0, _ = np.linalg.qr(rng.standard_normal((r, r)))
    s0 = np.sort(10.0 ** rng.uniform(-12, 1, r))[::-1]
    S = U0 @ np.diag(s0) @ Q0.T
    drop = 1e-6
    U, sig, Qm, rk, info = B.boltz_svd_truncate_f64(torch.tensor(S, device="cuda"), drop)
    U, sig, Qm = U.cpu().numpy(), sig.cpu().numpy(), Qm.cpu().numpy()
    assert int(info.item()) == 0
    _, so, _, rko = LR.svd_truncate(S, drop)
    assert int(rk.item()) == rko
    assert np.max(np.abs(sig - so)) <= 1e-12 * so[0]
    assert np.all(np.diff(sig) <= 0)
    assert np.max(np.abs(U @ np.diag(sig) @ Qm.T - S)) <= 1e-12 * so[0]
    assert np.max(np.abs(Qm.T @ Qm - np.eye(r))) < 1e-12
    big = sig > 1e-9 * sig[0]
    assert np.max(np.abs(U[:, big].T @ U[:, big] - np.eye(int(big.sum())))) < 1e-10


@pytest.mark.parametrize("r,n", [(16, 38912), (16, 38913), (5, 17), (3, 3000), (9, 1000), (2, 2)])
def test_qr_f64_sizes_at_the_path_limits(B, r, n):
    """Cholesky-QR2 at the edges of the spread path (r <= 16, n <= 152 x 256 =
    38912: entries per CTA = max(16, ceil(n / 152)), a ragged last CTA) and
    just past it (the multi-kernel path), against the oracle."""
    import torch
    from oracle import lowrank as LR
    rng = np.random.default_rng(500 + r + n)
    W = rng.standard_normal((r, n)) * np.exp(0.5 * rng.standard_normal((r, 1)))
    w = 0.03
    Y, R, info = B.boltz_qr_f64(torch.tensor(W, device="cuda"), w)
    Y, R = Y.cpu().numpy(), R.cpu().numpy()
    assert int(info.item()) == 0
    Yo, Ro = LR.qr_weighted(W, w)
    assert np.max(np.abs(R - Ro)) / np.max(np.abs(Ro)) < 1e-11
    assert np.max(np.abs(Y - Yo)) / np.max(np.abs(Yo)) < 1e-11
    assert np.max(np.abs(w * Y @ Y.T - np.eye(r))) < 1e-12


@pytest.mark.parametrize("r,spectrum", [(8, "repeated"), (16, "repeated"), (5, "clustered"), (12, "clustered"),
                                        (2, "repeated"), (3, "rank1")])
def test_svd_truncate_f64_repeated_and_clustered_values(B, r, spectrum):
    """Equal and nearly equal singular values (Jacobi pairs of equal norms,
    rotations of about 45 degrees), and a rank-one matrix: the one-warp SVD's
    FP32-derived angles and its early end of the FP64 sweeps still give
    orthonormal factors, sigma to 1e-12 and U Sigma Q^T = S to 1e-12."""
    import torch
    rng = np.random.default_rng(600 + r)
    U0, _ = np.linalg.qr(rng.standard_normal((r, r)))
    Q0, _ = np.linalg.qr(rng.standard_normal((r, r)))
    if spectrum == "repeated":
        s0 = np.array([3.0] * (r // 2) + [1.0] * (r - r // 2))
    elif spectrum == "clustered":
        s0 = 2.0 + 1e-9 * np.arange(r)[::-1]
    else:
        s0 = np.array([5.0] + [0.0] * (r - 1))
    S = U0 @ np.diag(s0) @ Q0.T
    U, sig, Qm, rk, info = B.boltz_svd_truncate_f64(torch.tensor(S, device="cuda"), 0.5)
    U, sig, Qm = U.cpu().numpy(), sig.cpu().numpy(), Qm.cpu().numpy()
    assert int(info.item()) == 0
    so = np.sort(s0)[::-1]
    assert np.max(np.abs(sig - so)) <= 1e-12 * so[0]
    assert int(rk.item()) == int(np.sum(so >= 0.5))
    assert np.max(np.abs(U @ np.diag(sig) @ Qm.T - S)) <= 1e-12 * so[0]
    assert np.max(np.abs(Qm.T @ Qm - np.eye(r))) < 1e-12
    big = sig > 1e-9 * sig[0]
    assert np.max(np.abs(U[:, big].T @ U[:, big] - np.eye(int(big.sum())))) < 1e-11


def test_drop_step_end_to_end(B):
    """Sec. 3.2 on the GPU: SVD of S, keep sigma >= drop_tol, rotate X and V;
    the truncated factorisation X_bar S_bar V_bar^T differs from X S V^T by at
    most the largest dropped singular value (orthonormal bases)."""
    import torch
    from oracle import lowrank as LR
    rng = np.random.default_rng(9)
    r, nx, nv, wx, wv = 8, 300, 4096, 0.2, 0.125
    X, _ = LR.qr_weighted(rng.standard_normal((r, nx)), wx)
    V, _ = LR.qr_weighted(rng.standard_normal((r, nv)), wv)
    s0 = np.array([5, 2, 1, 0.3, 1e-2, 1e-7, 1e-9, 1e-11])
    U0, _ = np.linalg.qr(rng.standard_normal((r, r)))
    Q0, _ = np.linalg.qr(rng.standard_normal((r, r)))
    S = U0 @ np.diag(s0) @ Q0.T
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    U, sig, Qm, rk, info = B.boltz_svd_truncate_f64(d(S), 1e-6)
    k = int(rk.item())
    assert k == 5 and int(info.item()) == 0
    Xb = B.boltz_basis_rotate_f64(d(X), U, k).cpu().numpy()
    Vb = B.boltz_basis_rotate_f64(d(V), Qm, k).cpu().numpy()
    assert np.max(np.abs(Xb - LR.rotate(X, U.cpu().numpy(), k))) < 1e-12
    full = X.T @ S @ V              # f(x, v) on the grids
    trunc = Xb.T @ np.diag(sig.cpu().numpy()[:k]) @ Vb
    # sup-norm bound through the orthonormal bases' scaling: ||X^T (S - S_k) V||_F = ||S - S_k||_F / sqrt(wx wv)
    err_f = np.linalg.norm(full - trunc) * np.sqrt(wx * wv)
    assert err_f <= 1.0001 * np.linalg.norm(s0[k:])
    assert np.allclose(wx * Xb @ Xb.T, np.eye(k), atol=1e-12)


@pytest.mark.parametrize("r", [16, 5, 64])
def test_coupling_and_sstep_term(B, r):
    import torch
    from oracle import lowrank as LR
    rng = np.random.default_rng(500 + r)
    X = rng.standard_normal((r, 40))
    E = f32(LR.triple_products(X, 0.05))
    S = f32(rng.standard_normal((r, r)))
    T = f32(rng.standard_normal((r, r, r)))
    d = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    Cg, Dg = B.boltz_lowrank_coupling(d(E), d(S), d(T))
    Co = LR.lstep_coupling(E, S)
    Do = LR.sstep_collision(T, E, S)
    Cs = LR.lstep_coupling(np.abs(E), np.abs(S))
    assert np.max(np.abs(Cg.cpu().numpy() - Co) / Cs) < 1e-5
    Ds = LR.sstep_collision(np.abs(T), np.abs(E), np.abs(S))
    assert np.max(np.abs(Dg.cpu().numpy() - Do) / Ds) < 1e-5
    C2, D2 = B.boltz_lowrank_coupling(d(E), d(S))
    assert D2 is None and np.array_equal(C2.cpu().numpy(), Cg.cpu().numpy())


def test_mott_smith_alpha_beta(B):
    """Sec. 4.2 closure on the GPU (Mach-3 Rankine-Hugoniot states, 32^3,
    hard spheres) against the oracle's alpha and beta."""
    import torch
    from gpu_helpers import as_fp32
    from oracle import collision as C
    from oracle import mott_smith as MS
    from paper_2112_02695_gb300 import workloads as W
    cfg = (32, 3, 8.0, 8.0, 1.0, 6, 14)
    (rL, uL, TL), (rR, uR, TR) = W.rankine_hugoniot(3, 3.0)
    fL, fR = (as_fp32(f) for f in W.shock_states_fields(32, 3, 8.0))
    g = B.boltz_grid_init(*cfg)
    try:
        spec = B.boltz_spectrum(g, torch.tensor(np.stack([fL, fR]), dtype=torch.float32, device="cuda"))
        al, be, _ = B.boltz_mott_smith(g, spec, rL, uL, TL, TR)
    finally:
        g.close()
    prob = C.Problem(N=32, d=3, L=8.0, R=8.0, gamma=1.0, n_rho=6, M=14)
    al_o = MS.alpha(prob, fL, fR)
    assert abs(al - al_o) <= 1e-4 * abs(al_o)
    assert abs(be - MS.beta(al_o, 3, rL, uL, TL, TR)) <= 1e-4 * abs(be)
    assert al < 0 and be > 0
