"""Orthogonal Matching Pursuit in FP64 (Sec. 2.1).

The paper codes every signal with OMP against the dictionary D, adding the most
relevant atom one at a time until a target sparsity k and/or an error tolerance
epsilon is reached.  This module takes the algorithm's steps in order, for each
signal x independently (rows of a batch are processed side by side with numpy,
but every row follows exactly the sequence below; no step is fused, reordered or
made incremental):

    r = x, I = {}
    for t = 1..s:
        if ||r||_2 <= eps: stop
        c = D^T r, with c_j = 0 for j in I
        j* = argmax_j |c_j|            (ties: smallest j)
        if |c_j*| <= 1e-12 ||x||: stop
        I = I + {j*}
        Householder QR of D_I, recomputed from scratch;
        if |R_tt| <= 1e-10: drop j*, stop
        gamma = argmin ||x - D_I gamma|| = R^-1 Q^T x
        r = x - D_I gamma

Readings of the paper (it names OMP but none of these details): the tolerance is
the absolute L2 norm of the residual over the 45-vector, checked before each
selection; ties go to the smallest atom index; an atom is never selected twice.

Layout: D has atoms as ROWS, shape (K, d) (the paper's D is its transpose);
X is (N, d).  Outputs: idx (N, s) in selection order (pad 0), coef (N, s) (pad 0),
nnz (N,), and residual norms.  Diagnostics: for each step, the sorted top-5 |c|
divided by ||r||, used by the parity tests to tell well-separated selections.

Pins (tests/test_oracle_omp.py): exact support recovery under Tropp's exact
recovery condition; orthonormal D gives hard thresholding; s = 1 is the best
1-subset; for d <= 8 the OMP residual never beats brute force; residual
orthogonality to the selected atoms; gamma equals numpy.linalg.lstsq on D_I;
the residual norm never increases.  omp_restricted: over a shuffled strict
candidate subset it equals omp on the sub-dictionary with positions mapped back
to atom ids; it recovers planted atom ids under the exact recovery condition;
equal correlations go to the smallest atom id wherever it sits in the candidate
list; it never beats the best s-subset of the candidates (d <= 8).
"""
from __future__ import annotations

import numpy as np

CORR_STOP_REL = 1e-12
QR_PIVOT_MIN = 1e-10


def _back_substitute(R: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve R g = b for upper-triangular R, batched: R (n, t, t), b (n, t)."""
    n, t, _ = R.shape
    g = np.zeros((n, t))
    for k in range(t - 1, -1, -1):
        acc = b[:, k] - np.einsum("nj,nj->n", R[:, k, k + 1:], g[:, k + 1:])
        g[:, k] = acc / R[:, k, k]
    return g


def omp(D, X, s: int, eps: float = 0.0, top: int = 5):
    """Batch of independent OMP runs.  Returns a dict of numpy arrays."""
    D = np.asarray(D, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    N, d = X.shape
    K = D.shape[0]
    idx = np.zeros((N, s), dtype=np.int64)
    coef = np.zeros((N, s))
    nnz = np.zeros(N, dtype=np.int64)
    R = X.copy()
    xnorm = np.linalg.norm(X, axis=1)
    active = np.ones(N, dtype=bool)
    topc = np.full((N, s, top), np.nan)  # sorted |c| / ||r|| at each step
    for t in range(s):
        act = np.nonzero(active)[0]
        if act.size == 0:
            break
        rnorm = np.linalg.norm(R[act], axis=1)
        stop = rnorm <= eps
        C = R[act] @ D.T
        if t > 0:
            np.put_along_axis(C, idx[act, :t], 0.0, axis=1)
        A = np.abs(C)
        jstar = np.argmax(A, axis=1)
        cmax = A[np.arange(act.size), jstar]
        stop |= cmax <= CORR_STOP_REL * xnorm[act]
        ntop = min(top, K)
        srt = -np.sort(-A, axis=1)[:, :ntop]
        with np.errstate(divide="ignore", invalid="ignore"):
            topc[act, t, :ntop] = srt / rnorm[:, None]
        active[act[stop]] = False
        go = act[~stop]
        if go.size == 0:
            break
        idx[go, t] = jstar[~stop]
        DI = np.transpose(D[idx[go, :t + 1]], (0, 2, 1))  # (n, d, t+1)
        Q, Rr = np.linalg.qr(DI)  # Householder QR (LAPACK geqrf) per signal
        piv = np.abs(Rr[:, t, t])
        bad = piv <= QR_PIVOT_MIN
        if bad.any():
            idx[go[bad], t] = 0
            active[go[bad]] = False
        ok = ~bad
        g = go[ok]
        if g.size == 0:
            continue
        qtx = np.einsum("ndt,nd->nt", Q[ok], X[g])
        gamma = _back_substitute(Rr[ok], qtx)
        R[g] = X[g] - np.einsum("ndt,nt->nd", DI[ok], gamma)
        coef[g, :t + 1] = gamma
        nnz[g] = t + 1
    res = X - np.einsum("ns,nsd->nd", np.where(np.arange(s)[None, :] < nnz[:, None], coef, 0.0),
                        D[idx])
    return {"idx": idx, "coef": coef, "nnz": nnz, "resid_sq": np.sum(res * res, axis=1),
            "resid": res, "topc": topc}


def omp_restricted(D, X, cand, s: int, eps: float = 0.0):
    """OMP run separately for each signal over its own candidate atoms only.

    cand (N, m): candidate atom indices per signal (distinct).  The steps are the
    ones of `omp` with the argmax taken over the candidates; returned indices are
    global atom indices in selection order.
    """
    D = np.asarray(D, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    cand = np.asarray(cand, dtype=np.int64)
    N, m = cand.shape
    idx = np.zeros((N, s), dtype=np.int64)
    coef = np.zeros((N, s))
    nnz = np.zeros(N, dtype=np.int64)
    chosen = np.zeros((N, m), dtype=bool)
    R = X.copy()
    xnorm = np.linalg.norm(X, axis=1)
    active = np.ones(N, dtype=bool)
    for t in range(s):
        act = np.nonzero(active)[0]
        if act.size == 0:
            break
        rnorm = np.linalg.norm(R[act], axis=1)
        stop = rnorm <= eps
        C = np.einsum("nd,nmd->nm", R[act], D[cand[act]])
        C[chosen[act]] = 0.0
        A = np.abs(C)
        # ties: smallest global atom index among the candidates with the max
        best = A.max(axis=1)
        tie = A == best[:, None]
        gidx = np.where(tie, cand[act], np.iinfo(np.int64).max)
        jglob = gidx.min(axis=1)
        jloc = np.argmax(cand[act] == jglob[:, None], axis=1)
        stop |= best <= CORR_STOP_REL * xnorm[act]
        active[act[stop]] = False
        go = act[~stop]
        if go.size == 0:
            break
        jl = jloc[~stop]
        chosen[go, jl] = True
        idx[go, t] = cand[go, jl]
        DI = np.transpose(D[idx[go, :t + 1]], (0, 2, 1))
        Q, Rr = np.linalg.qr(DI)
        piv = np.abs(Rr[:, t, t])
        bad = piv <= QR_PIVOT_MIN
        if bad.any():
            idx[go[bad], t] = 0
            active[go[bad]] = False
        ok = ~bad
        g = go[ok]
        if g.size == 0:
            continue
        qtx = np.einsum("ndt,nd->nt", Q[ok], X[g])
        gamma = _back_substitute(Rr[ok], qtx)
        R[g] = X[g] - np.einsum("ndt,nt->nd", DI[ok], gamma)
        coef[g, :t + 1] = gamma
        nnz[g] = t + 1
    res = X - np.einsum("ns,nsd->nd", np.where(np.arange(s)[None, :] < nnz[:, None], coef, 0.0),
                        D[idx])
    return {"idx": idx, "coef": coef, "nnz": nnz, "resid_sq": np.sum(res * res, axis=1)}
