"""Pins for oracle.ksvd: the approximate K-SVD sweep (one power step per atom)."""
import numpy as np

from oracle import ksvd as KS
from paper_2605_30396_gb300 import synth


def _problem(seed, N=400, K=24, s=4):
    rng = np.random.default_rng(seed)
    D = synth.hidden_dictionary(K, seed + 1)
    idx = synth.distinct_supports(rng, N, K, s)
    coef = rng.laplace(0, 1, (N, s))
    nnz = rng.integers(1, s + 1, N)
    coef[np.arange(s)[None, :] >= nnz[:, None]] = 0.0
    X = rng.standard_normal((N, 45))
    return X, D, idx, coef, nnz


def _objective(X, D, idx, coef, nnz):
    R = np.array(X, dtype=np.float64)
    for i in range(X.shape[0]):
        for t in range(nnz[i]):
            R[i] -= coef[i, t] * D[idx[i, t]]
    return float(np.sum(R * R))


def test_objective_non_increasing_and_consistent():
    X, D, idx, coef, nnz = _problem(0)
    D1, c1, info = KS.ksvd_update(X, D, idx, coef, nnz, trace=True)
    obj = info["objective"]
    np.testing.assert_allclose(obj[0], _objective(X, D, idx, coef, nnz), rtol=1e-12)
    assert np.all(np.diff(obj) <= 1e-9 * obj[0])
    assert obj[-1] < obj[0]
    np.testing.assert_allclose(obj[-1], _objective(X, D1, idx, c1, nnz), rtol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(D1, axis=1), 1.0, rtol=1e-12)
    # the support never changes; coefficients outside nnz stay zero
    assert np.all(c1[np.arange(idx.shape[1])[None, :] >= nnz[:, None]] == 0.0)


def test_rank_one_error_recovered_exactly():
    # one atom per signal: atom j's restricted error is X_w = c u^T, rank one
    rng = np.random.default_rng(3)
    K, N = 6, 120
    U = synth.hidden_dictionary(K, 4)
    assign = np.arange(N) % K
    c = rng.uniform(0.5, 2.0, N) * rng.choice([-1.0, 1.0], N)
    X = c[:, None] * U[assign]
    D0 = synth.hidden_dictionary(K, 5)
    g0 = rng.uniform(0.5, 2.0, N)
    idx = assign[:, None]
    D1, c1, info = KS.ksvd_update(X, D0, idx, g0[:, None], np.ones(N, dtype=np.int64))
    for j in range(K):
        w = assign == j
        sign = np.sign(np.dot(c[w], g0[w]))
        np.testing.assert_allclose(D1[j], sign * U[j], atol=1e-12)
        np.testing.assert_allclose(c1[w, 0], sign * c[w], atol=1e-12)
    assert np.max(info["resid_sq"]) < 1e-24


def test_start_at_top_singular_vector_returns_svd_pair():
    rng = np.random.default_rng(7)
    N = 50
    X = rng.standard_normal((N, 45))
    U, S, Vt = np.linalg.svd(X, full_matrices=False)
    D0 = synth.hidden_dictionary(1, 8)
    g0 = 3.0 * U[:, 0]
    D1, c1, info = KS.ksvd_update(X, D0, np.zeros((N, 1), dtype=np.int64), g0[:, None],
                                  np.ones(N, dtype=np.int64), trace=True)
    np.testing.assert_allclose(D1[0], Vt[0], atol=1e-12)
    np.testing.assert_allclose(c1[:, 0], S[0] * U[:, 0], atol=1e-12)
    np.testing.assert_allclose(info["objective"][-1], np.sum(S[1:] ** 2), rtol=1e-12)


def test_signal_order_does_not_matter():
    X, D, idx, coef, nnz = _problem(11, N=300)
    perm = np.random.default_rng(12).permutation(X.shape[0])
    D1, c1, _ = KS.ksvd_update(X, D, idx, coef, nnz)
    D2, c2, _ = KS.ksvd_update(X[perm], D, idx[perm], coef[perm], nnz[perm])
    np.testing.assert_allclose(D2, D1, atol=1e-12)
    np.testing.assert_allclose(c2, c1[perm], atol=1e-12)


def test_unused_atoms_refilled_with_worst_signals():
    X, D, idx, coef, nnz = _problem(21, N=200, K=10, s=3)
    K = 14  # atoms 10..13 unused
    D_big = np.vstack([D, synth.hidden_dictionary(4, 22)])
    rng = np.random.default_rng(23)
    resid = rng.random(X.shape[0])
    resid[[5, 9]] = 10.0  # a tie: the smaller index first
    D1, _, info = KS.ksvd_update(X, D_big, idx, coef, nnz, resid_sq=resid)
    assert list(info["unused"]) == [10, 11, 12, 13]
    order = np.lexsort((np.arange(resid.size), -resid))[:4]
    assert list(order[:2]) == [5, 9]
    for j, i in zip(range(10, 14), order):
        np.testing.assert_allclose(D1[j], X[i] / np.linalg.norm(X[i]), atol=1e-12)
