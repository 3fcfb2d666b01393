"""Pins for oracle.omp (OMP of Sec. 2.1) against closed forms, library LS and brute force."""
import itertools

import numpy as np
import pytest

from oracle import brute, omp as O
from paper_2605_30396_gb300 import synth


@pytest.mark.parametrize("n,s", [(16, 2), (64, 4)])
def test_exact_recovery_erc(n, s):
    """D = [I | H/sqrt n]: coherence mu = 1/sqrt n, and mu (2s-1) < 1 guarantees
    OMP recovers every s-sparse support exactly (Tropp's exact recovery condition)."""
    D = synth.erc_dictionary(n)
    mu = np.max(np.abs(D @ D.T - np.eye(2 * n)))
    assert mu * (2 * s - 1) < 1
    rng = np.random.default_rng(11)
    x, sup, coef = synth.planted_sparse(rng, D, 300, s)
    out = O.omp(D, x, s)
    assert (out["nnz"] == s).all()
    np.testing.assert_array_equal(np.sort(out["idx"], 1), np.sort(sup, 1))
    assert out["resid_sq"].max() < 1e-24
    # coefficients equal the planted ones (matched by atom)
    for i in range(20):
        got = dict(zip(out["idx"][i], out["coef"][i]))
        for j, c in zip(sup[i], coef[i]):
            assert abs(got[j] - c) < 1e-12


def test_orthonormal_is_hard_thresholding():
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    D = Q.T  # rows orthonormal
    X = rng.standard_normal((100, 12))
    s = 5
    out = O.omp(D, X, s)
    c = X @ D.T
    top = np.argsort(-np.abs(c), axis=1, kind="stable")[:, :s]
    np.testing.assert_array_equal(out["idx"], top)
    np.testing.assert_allclose(out["coef"], np.take_along_axis(c, top, 1), atol=1e-12)


def test_s1_is_best_single_atom():
    rng = np.random.default_rng(4)
    D = synth.hidden_dictionary(20, 3)
    X = rng.standard_normal((40, 45))
    out = O.omp(D, X, 1)
    for i in range(40):
        sup, g, r = brute.best_subset(D, X[i], 1)
        assert out["idx"][i, 0] == sup[0]
        assert abs(np.sqrt(out["resid_sq"][i]) - r) < 1e-12


def test_never_beats_brute_force_small_d():
    rng = np.random.default_rng(6)
    d, K, s = 6, 10, 3
    D = rng.standard_normal((K, d))
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    X = rng.standard_normal((30, d))
    out = O.omp(D, X, s)
    for i in range(30):
        _, _, r = brute.best_subset(D, X[i], s)
        assert np.sqrt(out["resid_sq"][i]) >= r - 1e-12


def test_brute_force_equality_on_erc():
    D = synth.erc_dictionary(8)
    rng = np.random.default_rng(8)
    x, sup, _ = synth.planted_sparse(rng, D, 10, 1)
    out = O.omp(D, x, 1)
    for i in range(10):
        bs, _, r = brute.best_subset(D, x[i], 1)
        assert out["idx"][i, 0] == bs[0] and r < 1e-12


def test_residual_orthogonal_and_lstsq():
    rng = np.random.default_rng(1)
    D = synth.hidden_dictionary(64, 2)
    X = synth.signals(50, D, 6, 3, dtype=np.float64)
    s = 8
    out = O.omp(D, X, s)
    for i in range(50):
        I = out["idx"][i, :out["nnz"][i]]
        DI = D[I].T
        r = out["resid"][i]
        assert np.max(np.abs(DI.T @ r)) < 1e-12 * max(1, np.linalg.norm(X[i]))
        g, *_ = np.linalg.lstsq(DI, X[i], rcond=None)
        np.testing.assert_allclose(out["coef"][i, :len(I)], g, rtol=1e-10, atol=1e-12)
        assert len(set(I.tolist())) == len(I)


def test_residual_nonincreasing():
    rng = np.random.default_rng(12)
    D = synth.hidden_dictionary(32, 5)
    X = rng.standard_normal((60, 45))
    prev = np.sum(X * X, axis=1)
    for s in range(1, 9):
        r = O.omp(D, X, s)["resid_sq"]
        assert (r <= prev + 1e-12).all()
        prev = r


def test_tolerance_stop_and_zero_signal():
    D = synth.erc_dictionary(16)
    rng = np.random.default_rng(5)
    x, sup, coef = synth.planted_sparse(rng, D, 20, 2)
    X = np.concatenate([x, np.zeros((1, 16))])
    out = O.omp(D, X, 6, eps=1e-9)
    assert (out["nnz"][:20] == 2).all()  # exact after 2 atoms, stops by tolerance
    assert out["nnz"][20] == 0 and out["resid_sq"][20] == 0


def test_tie_break_smallest_index():
    D = np.eye(4)
    X = np.array([[1.0, -1.0, 1.0, 0.5]])
    out = O.omp(D, X, 2)
    np.testing.assert_array_equal(out["idx"][0], [0, 1])


def test_degenerate_duplicate_atom_guard():
    """A repeated atom is never added: c = 0 on it after selection of its twin."""
    a = np.array([1.0, 0.0, 0.0])
    D = np.stack([a, a, [0, 1.0, 0]])
    X = np.array([[2.0, 0.0, 0.0]])
    out = O.omp(D, X, 3)
    assert out["nnz"][0] == 1 and out["idx"][0, 0] == 0


def test_restricted_equals_plain_when_candidates_are_all_atoms():
    rng = np.random.default_rng(21)
    D = synth.hidden_dictionary(24, 7)
    X = synth.signals(40, D, 4, 8, dtype=np.float64)
    cand = np.tile(np.arange(24), (40, 1))
    a = O.omp(D, X, 5)
    b = O.omp_restricted(D, X, cand, 5)
    np.testing.assert_array_equal(a["idx"], b["idx"])
    np.testing.assert_allclose(a["coef"], b["coef"], atol=1e-12)


def test_tolerance_boundary_is_inclusive():
    """The stop test is ||r||_2 <= eps: a residual exactly at eps stops."""
    D = np.eye(4)
    X = np.array([[3.0, 4.0, 0.0, 0.0]])  # ||x|| = 5 exactly
    assert O.omp(D, X, 2, eps=5.0)["nnz"][0] == 0
    out = O.omp(D, X, 2, eps=4.0)  # after atom 1 (coefficient 4), ||r|| = 3 <= 4
    assert out["nnz"][0] == 1 and out["idx"][0, 0] == 1


def _shuffled_subsets(rng, K, m, must):
    """Per row: m distinct atoms in random order, containing the atoms of must[i]."""
    out = np.empty((len(must), m), dtype=np.int64)
    for i, sup in enumerate(must):
        rest = np.setdiff1d(np.arange(K), sup)
        extra = rng.choice(rest, m - len(sup), replace=False)
        out[i] = rng.permutation(np.concatenate([sup, extra]))
    return out


def test_restricted_equals_plain_omp_on_the_candidate_subdictionary():
    """Restricted OMP over a shuffled strict subset is plain OMP on the
    sub-dictionary D[cand_i], its positions mapped back to atom ids through
    cand_i (generic real-valued atoms, so no ties arise)."""
    rng = np.random.default_rng(31)
    K, m, s = 40, 12, 5
    D = synth.hidden_dictionary(K, 9)
    X = synth.signals(60, D, 4, 10, dtype=np.float64)
    cand = np.stack([rng.choice(K, m, replace=False) for _ in range(60)])
    got = O.omp_restricted(D, X, cand, s)
    for i in range(60):
        ref = O.omp(D[cand[i]], X[i:i + 1], s)
        n = int(ref["nnz"][0])
        assert got["nnz"][i] == n
        np.testing.assert_array_equal(got["idx"][i, :n], cand[i][ref["idx"][0, :n]])
        np.testing.assert_allclose(got["coef"][i, :n], ref["coef"][0, :n], atol=1e-12)
        np.testing.assert_allclose(got["resid_sq"][i], ref["resid_sq"][0], rtol=1e-10, atol=1e-14)


def test_restricted_recovers_planted_atom_ids_from_shuffled_candidates():
    """Under the exact recovery condition, OMP over any candidate set that holds
    the planted support returns the planted atom ids (not candidate positions)."""
    D = synth.erc_dictionary(64)  # 128 atoms, mu = 1/8
    rng = np.random.default_rng(12)
    x, sup, coef = synth.planted_sparse(rng, D, 200, 4)
    cand = _shuffled_subsets(rng, D.shape[0], 16, sup)
    out = O.omp_restricted(D, x, cand, 4)
    assert (out["nnz"] == 4).all()
    np.testing.assert_array_equal(np.sort(out["idx"], 1), np.sort(sup, 1))
    assert out["resid_sq"].max() < 1e-24
    for i in range(200):
        got = dict(zip(out["idx"][i], out["coef"][i]))
        for j, c in zip(sup[i], coef[i]):
            assert abs(got[j] - c) < 1e-12


def test_restricted_tie_goes_to_smallest_atom_id_not_first_position():
    """Candidates listed in decreasing atom order: equal correlations must pick
    the smallest atom id, which sits at the largest candidate position."""
    D = np.eye(6)
    X = np.array([[0.0, 1.0, 0.0, 1.0, 0.0, 1.0]])  # atoms 1, 3, 5 tie
    cand = np.array([[5, 4, 3, 2, 1, 0]])
    out = O.omp_restricted(D, X, cand, 3)
    np.testing.assert_array_equal(out["idx"][0], [1, 3, 5])
    # the same tie over a candidate list in a shuffled order
    out = O.omp_restricted(D, X, np.array([[3, 0, 5, 2, 1, 4]]), 2)
    np.testing.assert_array_equal(out["idx"][0], [1, 3])


@pytest.mark.parametrize("d,K,m,s", [(6, 10, 6, 2), (8, 12, 7, 3)])
def test_restricted_never_beats_brute_force_over_the_candidates(d, K, m, s):
    """Greedy over the candidates never beats the best s-subset of the
    candidates; for s = 1 both are the single best candidate atom."""
    rng = np.random.default_rng(40 + d)
    D = rng.standard_normal((K, d))
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    X = rng.standard_normal((25, d))
    cand = np.stack([rng.choice(K, m, replace=False) for _ in range(25)])
    out = O.omp_restricted(D, X, cand, s)
    one = O.omp_restricted(D, X, cand, 1)
    for i in range(25):
        sub = D[cand[i]]
        sup, _, rbest = brute.best_subset(sub, X[i], s)
        assert np.sqrt(out["resid_sq"][i]) >= rbest - 1e-12
        sup1, _, r1 = brute.best_subset(sub, X[i], 1)
        assert one["idx"][i, 0] == cand[i][sup1[0]]
        assert abs(np.sqrt(one["resid_sq"][i]) - r1) < 1e-12
