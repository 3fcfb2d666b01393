"""Approximate K-SVD sweep on the GPU vs the FP64 oracle, on the same codes."""
import numpy as np
import pytest
import torch

from gpu_common import close_rel
from oracle import ksvd as oks, omp as oomp
from paper_2605_30396_gb300 import synth

pytestmark = pytest.mark.gpu


def _inputs(N, K, s, seed=0, K_used=None):
    Ku = K if K_used is None else K_used
    Dh = synth.hidden_dictionary(Ku, seed + 1)
    X = synth.signals(N, Dh, s, seed + 2)
    D0 = synth.hidden_dictionary(K, seed + 3).astype(np.float32)
    ref = oomp.omp(D0[:Ku].astype(np.float64), X.astype(np.float64), s)
    return (X, D0, ref["idx"].astype(np.uint16), ref["coef"].astype(np.float32), ref["nnz"].astype(np.uint8),
            ref["resid_sq"].astype(np.float32))


def _gpu(lib, X, D0, idx, coef, nnz, resid):
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    cf = c(coef)
    Dn = lib.ksvd_update(c(X), c(D0), c(idx.view(np.int16)), cf, c(nnz), c(resid) if resid is not None else None,
                         sync=True)
    return Dn.cpu().numpy(), cf.cpu().numpy()


def _oracle(X, D0, idx, coef, nnz, resid):
    return oks.ksvd_update(X.astype(np.float64), D0.astype(np.float64), idx.astype(np.int64),
                           coef.astype(np.float64), nnz.astype(np.int64),
                           None if resid is None else resid.astype(np.float64), trace=True)


@pytest.mark.parametrize("N,K,s", [(3000, 64, 4), (6000, 128, 8), (20000, 96, 6), (500, 16, 1), (800, 40, 12)])
def test_ksvd_matches_oracle(lib, N, K, s):
    X, D0, idx, coef, nnz, resid = _inputs(N, K, s)
    Dg, cg = _gpu(lib, X, D0, idx, coef, nnz, resid)
    Do, co, info = _oracle(X, D0, idx, coef, nnz, resid)
    ok, worst = close_rel(Dg, Do)
    assert ok, ("D", worst)
    ok, worst = close_rel(cg, co)
    assert ok, ("coef", worst)
    # the objective after the sweep, from the GPU's outputs, matches the oracle's
    obj_g = np.sum((X.astype(np.float64) - _recon(Dg, idx, cg, nnz)) ** 2)
    np.testing.assert_allclose(obj_g, info["objective"][-1], rtol=1e-4)
    assert obj_g <= info["objective"][0]


def _recon(D, idx, coef, nnz):
    out = np.zeros((idx.shape[0], 45))
    for t in range(idx.shape[1]):
        m = t < nnz
        out[m] += coef[m, t, None].astype(np.float64) * D[idx[m, t].astype(np.int64)].astype(np.float64)
    return out


def test_unused_atoms_refilled_and_entries_spread_over_ctas(lib):
    # 40 of 56 atoms used; about 4,000 entries per used atom span many CTAs
    N, K, s = 40000, 56, 4
    X, D0, idx, coef, nnz, resid = _inputs(N, K, s, seed=5, K_used=40)
    Dg, cg = _gpu(lib, X, D0, idx, coef, nnz, resid)
    Do, co, info = _oracle(X, D0, idx, coef, nnz, resid)
    assert list(info["unused"]) == list(range(40, 56))
    ok, worst = close_rel(Dg, Do)
    assert ok, ("D", worst)
    ok, worst = close_rel(cg, co)
    assert ok, ("coef", worst)
    # without residuals, unused atoms keep their old values
    Dg2, _ = _gpu(lib, X, D0, idx, coef, nnz, None)
    np.testing.assert_array_equal(Dg2[40:], D0[40:])


def test_rank_one_recovery_and_reproducibility(lib):
    rng = np.random.default_rng(3)
    K, N = 6, 3000
    U = synth.hidden_dictionary(K, 4)
    assign = np.arange(N) % K
    c = rng.uniform(0.5, 2.0, N) * rng.choice([-1.0, 1.0], N)
    X = (c[:, None] * U[assign]).astype(np.float32)
    D0 = synth.hidden_dictionary(K, 5).astype(np.float32)
    g0 = rng.uniform(0.5, 2.0, N).astype(np.float32)
    idx = assign[:, None].astype(np.uint16)
    nnz = np.ones(N, dtype=np.uint8)
    Dg, cg = _gpu(lib, X, D0, idx, g0[:, None], nnz, None)
    for j in range(K):
        w = assign == j
        sign = np.sign(np.dot(c[w], g0[w]))
        # FP32 sums over 500 entries (and X rounded to FP32): a few ulps of drift
        np.testing.assert_allclose(Dg[j], sign * U[j], atol=1e-5)
        np.testing.assert_allclose(cg[w, 0], sign * c[w], rtol=3e-5, atol=1e-5)
    Dg2, cg2 = _gpu(lib, X, D0, idx, g0[:, None], nnz, None)
    np.testing.assert_array_equal(Dg, Dg2)
    np.testing.assert_array_equal(cg, cg2)


def test_ksvd_rejects_aliasing_and_bad_sizes(lib):
    D = torch.from_numpy(synth.hidden_dictionary(8, 1).astype(np.float32)).cuda()
    from paper_2605_30396_gb300 import _lib
    L = _lib.lib()
    assert L.dlsh_ksvd_workspace_size(8, 44, 4, 10) == 0
    assert L.dlsh_ksvd_workspace_size(5000, 45, 4, 10) == 0
    X = torch.zeros((10, 45), device="cuda")
    idx = torch.zeros((10, 4), dtype=torch.int16, device="cuda")
    coef = torch.zeros((10, 4), device="cuda")
    nnz = torch.zeros(10, dtype=torch.uint8, device="cuda")
    ws = torch.empty(L.dlsh_ksvd_workspace_size(8, 45, 4, 10), dtype=torch.uint8, device="cuda")
    import ctypes
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = L.dlsh_ksvd_update(p(X), 10, 45, 8, p(idx), p(coef), p(nnz), 4, p(D), None, p(D), p(ws), ws.numel(),
                            None, 1)
    assert rc != 0


def test_ksvd_k1024_random_codes(lib):
    """K = 1024, s = 8 (the scene's dictionary size) on 200,000 signals with
    random distinct supports: every atom's entries spread over many CTAs."""
    N, K, s = 200_000, 1024, 8
    rng = np.random.default_rng(31)
    X = synth.signals(N, synth.hidden_dictionary(K, 32), s, 33)
    D0 = synth.hidden_dictionary(K, 34).astype(np.float32)
    idx = synth.distinct_supports(rng, N, K, s).astype(np.uint16)
    coef = rng.laplace(0, 1, (N, s)).astype(np.float32)
    nnz = np.full(N, s, dtype=np.uint8)
    Dg, cg = _gpu(lib, X, D0, idx, coef, nnz, None)
    Do, co, info = _oracle(X, D0, idx, coef, nnz, None)
    ok, worst = close_rel(Dg, Do)
    assert ok, ("D", worst)
    ok, worst = close_rel(cg, co)
    assert ok, ("coef", worst)


def test_ksvd_empty(lib):
    D0 = synth.hidden_dictionary(12, 2).astype(np.float32)
    X = np.zeros((0, 45), dtype=np.float32)
    Dg, cg = _gpu(lib, X, D0, np.zeros((0, 4), dtype=np.uint16), np.zeros((0, 4), dtype=np.float32),
                  np.zeros(0, dtype=np.uint8), np.zeros(0, dtype=np.float32))
    np.testing.assert_array_equal(Dg, D0)  # every atom unused, nothing to refill from
    assert cg.shape == (0, 4)
