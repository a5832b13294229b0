"""Pins of the low-rank oracle (oracle/lowrank.py) against the mathematics it
restates: the K- and L-step collision terms against direct collision
evaluations of the reconstructed functions (bilinearity, paper Sec. 2),
closed forms, a textbook Gram-Schmidt, and a matrix of known singular values."""
import numpy as np
import pytest

from oracle import collision as C
from oracle import lowrank as LR


def small_problem():
    return C.Problem(N=8, d=2, L=6.0, R=6.0, gamma=1.0, n_rho=3, M=8)


def basis(prob, r, seed):
    rng = np.random.default_rng(seed)
    x = -prob.L + np.arange(prob.N) * (2 * prob.L / prob.N)
    v0, v1 = np.meshgrid(x, x, indexing="ij")
    g = np.exp(-0.5 * (v0 ** 2 + v1 ** 2))
    return np.stack([g * (1 + 0.3 * rng.standard_normal() * v0 + 0.2 * rng.standard_normal() * v1 ** 2)
                     for _ in range(r)])


def all_pairs_Q(prob, V):
    r = V.shape[0]
    pairs = [(p, q) for p in range(r) for q in range(r)]
    return C.collide_fields(prob, V, pairs)


def test_kstep_term_equals_projection_of_the_cell_collision():
    """C_j(x) = <V_j, Q(f_x, f_x)>_v with f_x = sum_m K_m(x) V_m (Sec. 2 K-step)."""
    prob = small_problem()
    r, nx = 3, 4
    V = basis(prob, r, 1)
    Q = all_pairs_Q(prob, V)
    T = C.project(prob, V, Q).reshape(r, r, r)
    K = np.random.default_rng(2).standard_normal((r, nx))
    got = LR.kstep_collision(T, K)
    fx = np.einsum("mx,m...->x...", K, V)
    Qx = C.collide_fields(prob, fx, [(x, x) for x in range(nx)])
    want = np.stack([C.project(prob, V[j][None], Qx)[0] for j in range(r)])   # [r][nx]
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_kstep_term_closed_form():
    r, nx = 4, 7
    T = np.zeros((r, r, r))
    for j in range(r):
        T[j, j, j] = 1.0
    K = np.random.default_rng(3).standard_normal((r, nx))
    assert np.allclose(LR.kstep_collision(T, K), K ** 2, rtol=0, atol=1e-15)


def test_lstep_term_equals_collision_of_the_l_functions():
    """sum_{p,q} C_ipq Q(V_p, V_q) = sum_{m,n} E_imn Q(L_m, L_n), L_m = sum_p S_mp V_p."""
    prob = small_problem()
    r = 3
    V = basis(prob, r, 4)
    rng = np.random.default_rng(5)
    S = rng.standard_normal((r, r))
    X = rng.standard_normal((r, 9))
    E = LR.triple_products(X, 0.25)
    Q = all_pairs_Q(prob, V)
    got = LR.lstep_collision(Q, LR.lstep_coupling(E, S))
    Lf = np.einsum("mp,p...->m...", S, V)
    QL = C.collide_fields(prob, Lf, [(m, n) for m in range(r) for n in range(r)]).reshape(r, r, -1)
    want = np.einsum("imn,mnv->iv", E, QL)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_triple_products_closed_form():
    n, w = 10, 0.3
    X = np.ones((2, n))
    X[1] = np.arange(n)
    E = LR.triple_products(X, w)
    assert E[0, 0, 0] == pytest.approx(w * n)
    assert E[1, 1, 0] == pytest.approx(w * np.sum(np.arange(n) ** 2))
    assert E[0, 1, 1] == E[1, 0, 1] == E[1, 1, 0]


def test_qr_matches_gram_schmidt_and_reconstructs():
    rng = np.random.default_rng(6)
    r, n, w = 5, 40, 0.125
    W = rng.standard_normal((r, n))
    Y, R = LR.qr_weighted(W, w)
    # textbook modified Gram-Schmidt under <a, b> = w sum a b
    Yg = np.zeros_like(W)
    Rg = np.zeros((r, r))
    for j in range(r):
        u = W[j].copy()
        for i in range(j):
            Rg[i, j] = w * np.dot(Yg[i], u)
            u -= Rg[i, j] * Yg[i]
        Rg[j, j] = np.sqrt(w * np.dot(u, u))
        Yg[j] = u / Rg[j, j]
    assert np.allclose(Y, Yg, atol=1e-12) and np.allclose(R, Rg, atol=1e-12)
    assert np.allclose(R.T @ Y, W, atol=1e-12)                      # W_j = sum_i Y_i R_ij
    assert np.allclose(w * Y @ Y.T, np.eye(r), atol=1e-12)
    assert np.allclose(np.tril(R, -1), 0) and np.all(np.diag(R) > 0)


def test_svd_truncation_of_known_spectrum():
    rng = np.random.default_rng(7)
    r = 6
    U0, _ = np.linalg.qr(rng.standard_normal((r, r)))
    Q0, _ = np.linalg.qr(rng.standard_normal((r, r)))
    s0 = np.array([3.0, 1.0, 0.5, 1e-3, 1e-8, 1e-12])
    S = U0 @ np.diag(s0) @ Q0.T
    U, s, Qm, rk = LR.svd_truncate(S, 1e-6)
    assert np.allclose(s, s0, rtol=1e-9, atol=1e-14)
    assert rk == 4
    assert np.allclose(U @ np.diag(s) @ Qm.T, S, atol=1e-13)
    assert np.allclose(U.T @ U, np.eye(r), atol=1e-13) and np.allclose(Qm.T @ Qm, np.eye(r), atol=1e-13)
    # singular vectors agree with the construction up to sign for distinct values
    assert np.allclose(np.abs(np.diag(U.T @ U0)), 1.0, atol=1e-6)


def test_rotation_keeps_orthonormality_and_identity():
    rng = np.random.default_rng(8)
    r, n, w = 4, 30, 0.5
    Y, _ = LR.qr_weighted(rng.standard_normal((r, n)), w)
    U, _ = np.linalg.qr(rng.standard_normal((r, r)))
    Z = LR.rotate(Y, U, 3)
    assert np.allclose(w * Z @ Z.T, np.eye(3), atol=1e-12)
    assert np.allclose(LR.rotate(Y, np.eye(r), r), Y)


def test_sstep_term_equals_projection_of_the_kstep_term():
    """D_ij = <X_i V_j, Q(f, f)>_{x,v} with f = sum X_k S_kl V_l, i.e.
    w_x sum_x X_i(x) C_j(x) with C the K-step term of K_m = sum_k X_k S_km."""
    rng = np.random.default_rng(10)
    r, nx, w = 4, 11, 0.3
    T = rng.standard_normal((r, r, r))
    X = rng.standard_normal((r, nx))
    S = rng.standard_normal((r, r))
    E = LR.triple_products(X, w)
    got = LR.sstep_collision(T, E, S)
    K = S.T @ X                                # K_m(x) = sum_k X_k(x) S_km
    Ck = LR.kstep_collision(T, K)              # [r][nx]
    want = w * X @ Ck.T                        # D_ij = w sum_x X_i(x) C_j(x)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_coupling_closed_form():
    """With E_imn = delta_im delta_in and S = identity, C_ipq = delta_ip delta_iq."""
    r = 5
    E = np.zeros((r, r, r))
    for i in range(r):
        E[i, i, i] = 1.0
    C = LR.lstep_coupling(E, np.eye(r))
    assert np.array_equal(C, E)
