"""FP64 oracle of the low-rank step pieces that consume the collision batch.

TEST INFRASTRUCTURE ONLY (see the package docstring): imported by tests, the
smoke check and the benchmark's CPU leg, never by the CUDA library, with
which it shares no code.

What is computed (paper Sec. 2, eqs. "eqn:K-step detailed" and
"eqn:L-step detailed"; Sec. 2.4, the fully discrete scheme; Sec. 3.2,
dropping basis).  Functions of x or v are stored as rows: K is [r][n_x],
V is [r][n_v]; the r^3 tensor T[j][m][n] = <V_j Q(V_m, V_n)>_v is the
projection the collision library returns.

  K-step collision term (Sec. 2.4, K-step (b)):
      C_j(x) = sum_{m,n} T_jmn K_m(x) K_n(x)
  S-step collision term (Sec. 2.4, S-step (a)):
      D_ij = sum_{m,n} T_jmn sum_l ( sum_k E_ikl S_km ) S_ln
  L-step coupling and collision term (Sec. 2.4, L-step (b)):
      C_ipq = sum_n ( sum_m E_imn S_mp ) S_nq,   E_imn = <X_i X_m X_n>_x
      G_i(v) = sum_{p,q} Q(V_p, V_q)(v) C_ipq
  QR of the K- and L-steps (Sec. 2.4, K-step (c), L-step (c)): the r
      functions W_j become Y_i, orthonormal under <a, b> = w sum a b (w the
      midpoint-rule cell volume), with W_j = sum_i Y_i R_ij, R upper
      triangular with a positive diagonal
  Dropping basis (Sec. 3.2): S = U Sigma Q^T with descending singular values;
      the r' values >= drop_tol are kept (values below drop_tol are dropped),
      U_bar = U[:, :r'], Q_bar = Q[:, :r'], S_bar = Sigma[:r', :r'], and the
      bases rotate as X_bar_k = sum_i X_i U_bar_ik, V_bar_k = sum_j V_j Q_bar_jk.

The steps use plain loops and numpy's dense LAPACK routines (QR, SVD) as the
paper's linear algebra; the only readings are the storage order above and
the sign normalisation of the QR (positive diagonal of R).
"""
from __future__ import annotations

import numpy as np


def kstep_collision(T: np.ndarray, K: np.ndarray) -> np.ndarray:
    """C_j(x) = sum_{m,n} T_jmn K_m(x) K_n(x).  T [r][r][r], K [r][n_x]."""
    T = np.asarray(T, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    r = K.shape[0]
    out = np.zeros_like(K)
    for j in range(r):
        for m in range(r):
            for n in range(r):
                out[j] += T[j, m, n] * K[m] * K[n]
    return out


def lstep_coupling(E: np.ndarray, S: np.ndarray) -> np.ndarray:
    """C_ipq = sum_n (sum_m E_imn S_mp) S_nq.  E [r][r][r], S [r][r]."""
    E = np.asarray(E, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    r = S.shape[0]
    inner = np.zeros((r, r, r))            # inner[i, p, n] = sum_m E_imn S_mp
    for i in range(r):
        for p in range(r):
            for m in range(r):
                inner[i, p] += E[i, m] * S[m, p]
    C = np.zeros((r, r, r))
    for i in range(r):
        for p in range(r):
            for q in range(r):
                C[i, p, q] = np.dot(inner[i, p], S[:, q])
    return C


def sstep_collision(T: np.ndarray, E: np.ndarray, S: np.ndarray) -> np.ndarray:
    """S-step collision term (Sec. 2.4, S-step (a)), in the paper's order:
    D_ij = sum_{m,n} T_jmn sum_l ( sum_k E_ikl S_km ) S_ln."""
    T = np.asarray(T, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    r = S.shape[0]
    D = np.zeros((r, r))
    for i in range(r):
        inner = np.zeros((r, r))               # inner[m, l] = sum_k E_ikl S_km
        for m in range(r):
            for l in range(r):
                inner[m, l] = np.dot(E[i, :, l], S[:, m])
        M = inner @ S                          # M[m, n] = sum_l inner[m, l] S_ln
        for j in range(r):
            D[i, j] = np.sum(T[j] * M)
    return D


def triple_products(X: np.ndarray, w: float) -> np.ndarray:
    """E_imn = <X_i X_m X_n>_x = w sum_x X_i X_m X_n (midpoint rule)."""
    X = np.asarray(X, dtype=np.float64)
    r = X.shape[0]
    E = np.zeros((r, r, r))
    for i in range(r):
        for m in range(r):
            for n in range(r):
                E[i, m, n] = w * np.sum(X[i] * X[m] * X[n])
    return E


def lstep_collision(Q: np.ndarray, C: np.ndarray) -> np.ndarray:
    """G_i(v) = sum_{p,q} C_ipq Q(V_p, V_q)(v).  Q [r*r][n_v] (pair p*r+q), C [r][r][r]."""
    Q = np.asarray(Q, dtype=np.float64).reshape(Q.shape[0], -1)
    C = np.asarray(C, dtype=np.float64)
    r = C.shape[0]
    out = np.zeros((r, Q.shape[1]))
    for i in range(r):
        for p in range(r):
            for q in range(r):
                out[i] += C[i, p, q] * Q[p * r + q]
    return out


def qr_weighted(W: np.ndarray, w: float):
    """W [r][n] -> (Y [r][n], R [r][r]): W_j = sum_i Y_i R_ij, w Y Y^T = I,
    R upper triangular with a positive diagonal."""
    A = np.asarray(W, dtype=np.float64).T * np.sqrt(w)      # n x r
    Qn, R = np.linalg.qr(A, mode="reduced")
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    Qn = Qn * sgn[None, :]
    R = sgn[:, None] * R
    return (Qn / np.sqrt(w)).T, R


def svd_truncate(S: np.ndarray, drop_tol: float):
    """S = U Sigma Q^T (descending); keep the singular values >= drop_tol.
    Returns U [r][r], sigma [r], Q [r][r] (columns are the singular vectors)
    and r' (the number kept)."""
    U, s, Qt = np.linalg.svd(np.asarray(S, dtype=np.float64))
    r_keep = int(np.sum(s >= drop_tol))
    return U, s, Qt.T, r_keep


def rotate(X: np.ndarray, U: np.ndarray, r_new: int) -> np.ndarray:
    """X_bar_k = sum_i X_i U_ik for k < r_new.  X [r][n], U [r][r]."""
    X = np.asarray(X, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    out = np.zeros((r_new, X.shape[1]))
    for k in range(r_new):
        for i in range(X.shape[0]):
            out[k] += U[i, k] * X[i]
    return out
