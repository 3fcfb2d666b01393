"""Pins for oracle.mod: the MOD dictionary update and the alternating loop (Eq. 1)."""
import numpy as np

from oracle import mod as M, omp as O
from paper_2605_30396_gb300 import synth


def _codes(rng, N, K, s):
    idx = synth.distinct_supports(rng, N, K, s)
    coef = rng.laplace(0, 1, size=(N, s))
    return idx, coef, np.full(N, s)


def test_normal_equations_match_dense():
    rng = np.random.default_rng(0)
    N, K, s = 80, 12, 3
    idx, coef, nnz = _codes(rng, N, K, s)
    nnz[:5] = 1
    X = rng.standard_normal((N, 45))
    A = np.zeros((K, N))
    for i in range(N):
        for t in range(nnz[i]):
            A[idx[i, t], i] = coef[i, t]
    G, B = M.normal_equations(X, idx, coef, nnz, K)
    np.testing.assert_allclose(G, A @ A.T, atol=1e-12)
    np.testing.assert_allclose(B, X.T @ A.T, atol=1e-12)


def test_stationarity_of_ridge_solution():
    """(X - D~ A) A^T = lambda (D~ - D_old): gradient of the ridge objective is zero."""
    rng = np.random.default_rng(1)
    N, K, s = 300, 20, 4
    idx, coef, nnz = _codes(rng, N, K, s)
    X = rng.standard_normal((N, 45))
    D_old = synth.hidden_dictionary(K, 2)
    G, B = M.normal_equations(X, idx, coef, nnz, K)
    Dt, lam = M.mod_solve(G, B, D_old)
    A = np.zeros((K, N))
    for i in range(N):
        A[idx[i], i] = coef[i]
    lhs = (X.T - Dt.T @ A) @ A.T
    np.testing.assert_allclose(lhs, lam * (Dt.T - D_old.T), atol=1e-9)


def test_planted_recovery_one_step():
    rng = np.random.default_rng(3)
    N, K, s = 2000, 16, 3
    Dtrue = synth.hidden_dictionary(K, 4)
    idx, coef, nnz = _codes(rng, N, K, s)
    X = np.einsum("ns,nsd->nd", coef, Dtrue[idx])
    D_old = synth.hidden_dictionary(K, 99)
    Dn, info = M.mod_update(X, D_old, idx, coef, nnz)
    # up to the tiny ridge pull towards D_old, the true atoms come back
    cos = np.abs(np.sum(Dn * Dtrue, axis=1))
    assert cos.min() > 1 - 1e-9


def test_update_never_increases_objective():
    rng = np.random.default_rng(5)
    N, K, s = 500, 24, 4
    Dh = synth.hidden_dictionary(K, 6)
    X = synth.signals(N, Dh, s, 7, dtype=np.float64)
    D = synth.hidden_dictionary(K, 8)
    codes = O.omp(D, X, s)
    A = np.zeros((K, N))
    for i in range(N):
        A[codes["idx"][i, :codes["nnz"][i]], i] = codes["coef"][i, :codes["nnz"][i]]
    before = np.linalg.norm(X.T - D.T @ A)
    G, B = M.normal_equations(X, codes["idx"], codes["coef"], codes["nnz"], K)
    Dt, lam = M.mod_solve(G, B, D)
    after = np.linalg.norm(X.T - Dt.T @ A)
    assert after <= before + 1e-12


def test_dead_atom_refill_order():
    rng = np.random.default_rng(9)
    N, K = 10, 4
    X = rng.standard_normal((N, 45))
    D_old = synth.hidden_dictionary(K, 1)
    # atoms 1 and 3 unused; signal residuals chosen by hand via resid_sq
    idx = np.zeros((N, 1), dtype=np.int64)
    idx[::2, 0] = 0
    idx[1::2, 0] = 2
    coef = np.ones((N, 1))
    nnz = np.ones(N, dtype=np.int64)
    resid = np.array([1, 5, 3, 5, 2, 0.5, 9, 1, 1, 1], dtype=float)
    Dn, info = M.mod_update(X, D_old, idx, coef, nnz, resid_sq=resid)
    np.testing.assert_array_equal(info["dead"], [1, 3])
    xn = X / np.linalg.norm(X, axis=1, keepdims=True)
    np.testing.assert_allclose(Dn[1], xn[6])  # largest residual
    np.testing.assert_allclose(Dn[3], xn[1])  # tie 5 vs 5 -> smaller index 1
    np.testing.assert_allclose(np.linalg.norm(Dn, axis=1), 1.0)


def test_learn_loop_reduces_rmse_and_recovers_atoms():
    N, K, s = 3000, 32, 3
    Dh = synth.hidden_dictionary(K, 10)
    X = synth.signals(N, Dh, s, 11, dtype=np.float64)
    init = synth.init_atom_indices(N, K, 0)
    D, codes, hist = M.learn(X, K, s, 8, init)
    assert hist[-1] < hist[0]
    assert len(hist) == 9
    cos = np.abs(D @ Dh.T).max(axis=1)
    assert np.mean(cos > 0.99) > 0.5


def test_ridge_lambda_reading():
    """lambda = 1e-6 trace(G) / K (the mean diagonal), 1e-6 when G is zero."""
    assert M.ridge_lambda(2.0 * np.eye(7)) == 2e-6
    assert M.ridge_lambda(np.zeros((5, 5))) == 1e-6
