"""Dictionary update and the alternating learning loop in FP64 (Sec. 2.1, Eq. 1).

Eq. 1 minimises sum_i ||x_i - D alpha_i||^2 subject to ||alpha_i||_0 <= k and
unit-norm atoms; the paper solves it by alternating minimisation, updating the
codes with D fixed and D with the codes fixed.  It does not name the D-update
rule.  Reading taken: MOD, the least-squares minimiser of the objective in D
with the codes held fixed, with a small ridge term so that it is defined when
some atom is unused:

    G = A A^T (K x K),  B = X A^T (d x K),  lambda = 1e-6 * trace(G) / K
    D~ = (B + lambda D_old) (G + lambda I)^-1        (Cholesky of G + lambda I)
    d_j <- d~_j / ||d~_j||                           (unit-norm constraint of Eq. 1)
    dead atoms (alpha_j. all zero, or d~_j = 0) are refilled, in increasing j,
    with the normalised signals of largest residual ||x_i - D_old alpha_i||,
    taken in decreasing-residual order, ties to the smallest signal index.

If trace(G) = 0 (no codes at all) lambda falls back to 1e-6.

Learning loop: D_0 = the normalised signals at K given distinct indices (the
random draw is an input); then `iters` times {codes = OMP(D, X); D = MOD(...)}
and a final OMP pass; RMSE_t = sqrt(sum_i ||x_i - D alpha_i||^2 / (N d)) after
every coding pass.

Pins (tests/test_oracle_mod.py): stationarity (X - D~ A) A^T = lambda (D~ - D_old)
of the ridge problem; exact recovery of a planted dictionary from exact codes in
one step; the update never increases ||X - D A||_F before normalisation; dead-atom
refill order on a hand-built case.  Learning quality beyond matching this loop is
reported, not pinned (parity unpinned for planted-atom recovery rates).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .omp import omp

RIDGE_REL = 1e-6


def code_matrix(idx, coef, nnz, K: int) -> sp.csr_matrix:
    """Sparse A (K x N) from ELL codes (only the first nnz_i slots of row i count)."""
    idx = np.asarray(idx, dtype=np.int64)
    coef = np.asarray(coef, dtype=np.float64)
    N, s = idx.shape
    keep = np.arange(s)[None, :] < np.asarray(nnz)[:, None]
    rows = idx[keep]
    cols = np.repeat(np.arange(N), s).reshape(N, s)[keep]
    return sp.csr_matrix((coef[keep], (rows, cols)), shape=(K, N))


def normal_equations(X, idx, coef, nnz, K: int):
    """G = A A^T (K, K) and B = X A^T (d, K), dense FP64."""
    A = code_matrix(idx, coef, nnz, K)
    G = (A @ A.T).toarray()
    B = (A @ np.asarray(X, dtype=np.float64)).T  # (d, K)
    return G, np.asarray(B)


def ridge_lambda(G: np.ndarray) -> float:
    tr = float(np.trace(G))
    K = G.shape[0]
    return RIDGE_REL * tr / K if tr > 0.0 else RIDGE_REL


def mod_solve(G, B, D_old):
    """D~^T (K, d) solving (G + lambda I) D~^T = (B + lambda D_old^T)^T."""
    D_old = np.asarray(D_old, dtype=np.float64)  # (K, d) rows = atoms
    K = G.shape[0]
    lam = ridge_lambda(G)
    M = G + lam * np.eye(K)
    rhs = B.T + lam * D_old  # (K, d)
    L = np.linalg.cholesky(M)
    # forward then backward substitution with the Cholesky factor
    z = np.linalg.solve(L, rhs)
    return np.linalg.solve(L.T, z), lam


def refill_order(resid_sq: np.ndarray, xnorm: np.ndarray) -> np.ndarray:
    """Signal indices by decreasing residual, ties to the smallest index, x != 0."""
    order = np.lexsort((np.arange(resid_sq.size), -resid_sq))
    return order[xnorm[order] > 0.0]


def mod_update(X, D_old, idx, coef, nnz, resid_sq=None):
    """One MOD step: returns (D_new (K, d), info dict)."""
    X = np.asarray(X, dtype=np.float64)
    D_old = np.asarray(D_old, dtype=np.float64)
    K = D_old.shape[0]
    G, B = normal_equations(X, idx, coef, nnz, K)
    Dt, lam = mod_solve(G, B, D_old)
    norms = np.linalg.norm(Dt, axis=1)
    counts = np.bincount(np.asarray(idx)[np.arange(idx.shape[1])[None, :] < np.asarray(nnz)[:, None]],
                         minlength=K)
    dead = np.nonzero((counts == 0) | (norms == 0.0))[0]
    D_new = Dt / np.where(norms > 0.0, norms, 1.0)[:, None]
    if dead.size:
        if resid_sq is None:
            from .sh import reconstruct
            r = X - reconstruct(D_old, idx, coef, nnz)
            resid_sq = np.sum(r * r, axis=1)
        xn = np.linalg.norm(X, axis=1)
        order = refill_order(np.asarray(resid_sq, dtype=np.float64), xn)
        for j, i in zip(dead, order):
            D_new[j] = X[i] / xn[i]
    return D_new, {"G": G, "B": B, "lambda": lam, "dead": dead, "D_tilde": Dt}


def init_dictionary(X, init_idx):
    X = np.asarray(X, dtype=np.float64)
    D0 = X[np.asarray(init_idx)]
    return D0 / np.linalg.norm(D0, axis=1, keepdims=True)


def rmse(resid_sq, d: int) -> float:
    r = np.asarray(resid_sq, dtype=np.float64)
    return float(np.sqrt(r.sum() / (r.size * d)))


def learn(X, K: int, s: int, iters: int, init_idx, eps: float = 0.0):
    """Alternating minimisation of Eq. 1 with OMP codes and MOD updates."""
    X = np.asarray(X, dtype=np.float64)
    d = X.shape[1]
    D = init_dictionary(X, init_idx)
    hist = []
    for _ in range(iters):
        codes = omp(D, X, s, eps)
        hist.append(rmse(codes["resid_sq"], d))
        D, _ = mod_update(X, D, codes["idx"], codes["coef"], codes["nnz"], codes["resid_sq"])
    codes = omp(D, X, s, eps)
    hist.append(rmse(codes["resid_sq"], d))
    return D, codes, hist
