"""Approximate K-SVD dictionary update in FP64 (an alternative D-update for the
alternating minimisation of Eq. 1, Sec. 2.1).

Test infrastructure only: the tests, smoke() and bench.py's CPU legs use it; the
library never does.

The paper names only "alternating minimisation".  Besides MOD (oracle/mod.py)
the K-SVD family reads the D-step as a sweep over the atoms in which atom j and
the coefficients that use it are refitted together, with every other atom and
coefficient held at its current value.  The approximate variant (Rubinstein,
Zibulevsky and Elad, 2008) replaces the rank-1 SVD of each atom's restricted
error by one power iteration started from the current coefficients.  Steps, for
j = 0, 1, ..., K-1 in order, with D and A the current values (atoms < j already
updated):

    w      = {i : atom j is in the first nnz_i code slots of signal i}
    g      = A[j, w]                                  (current coefficients)
    E      = X[w] - (D A)[w] + g d_j                  (error without atom j)
    d      = E^T g  (a d-vector),   d <- d / ||d||     (one power step)
    g_new  = E d
    D[j] = d,  A[j, w] = g_new

An atom with w empty is unused; an atom whose d is zero is left as it was (atom
and coefficients).  After the sweep, unused atoms are refilled, in increasing j,
with the normalised signals of largest residual under the input codes (resid_sq,
the encoder's), ties to the smaller index, zero signals skipped: the same rule
as the MOD update.  The support (indices, nnz) never changes; the coefficients
do.  Within a signal the atom indices are distinct (as OMP produces them).

Each atom step is a block-coordinate minimisation of ||X - D A||_F^2: with g
fixed, d ~ E^T g is the least-squares direction; with the unit d fixed, E d is
the least-squares coefficient row.  So the objective never increases from one
atom step to the next.

Pins (tests/test_oracle_ksvd.py): the objective is non-increasing over the
atom steps and its last value equals ||X - D_new A_new||_F^2 computed from the
outputs; an exactly rank-1 restricted error is recovered exactly in one step;
started from the top right singular vector of E, the step returns the top
singular pair (numpy's SVD); the result does not depend on how the signals are
ordered.
"""
from __future__ import annotations

import numpy as np

from .mod import refill_order


def ksvd_update(X, D_old, idx, coef, nnz, resid_sq=None, trace: bool = False):
    """One sweep.  Returns (D_new (K, d), coef_new (N, s), info dict)."""
    X = np.asarray(X, dtype=np.float64)
    D = np.array(D_old, dtype=np.float64)
    idx = np.asarray(idx, dtype=np.int64)
    A = np.array(coef, dtype=np.float64)
    nnz = np.asarray(nnz, dtype=np.int64)
    N, s = idx.shape
    K = D.shape[0]
    live = np.arange(s)[None, :] < nnz[:, None]
    # current residual R = X - D A, kept up to date through the sweep
    R = X.copy()
    for t in range(s):
        m = live[:, t]
        R[m] -= A[m, t][:, None] * D[idx[m, t]]
    objective = [float(np.sum(R * R))] if trace else None
    unused = []
    for j in range(K):
        rows, slots = np.nonzero(live & (idx == j))
        if rows.size == 0:
            unused.append(j)
            continue
        g = A[rows, slots]
        E = R[rows] + np.outer(g, D[j])
        d = E.T @ g
        nd = np.linalg.norm(d)
        if nd == 0.0:
            continue
        d /= nd
        g_new = E @ d
        R[rows] = E - np.outer(g_new, d)
        D[j] = d
        A[rows, slots] = g_new
        if trace:
            objective.append(float(np.sum(R * R)))
    if unused:
        if resid_sq is None:
            r = X.copy()
            c0 = np.asarray(coef, dtype=np.float64)
            D0 = np.asarray(D_old, dtype=np.float64)
            for t in range(s):
                m = live[:, t]
                r[m] -= c0[m, t][:, None] * D0[idx[m, t]]
            resid_sq = np.sum(r * r, axis=1)
        xn = np.linalg.norm(X, axis=1)
        order = refill_order(np.asarray(resid_sq, dtype=np.float64), xn)
        for j, i in zip(unused, order):
            D[j] = X[i] / xn[i]
    info = {"unused": np.asarray(unused, dtype=np.int64), "resid_sq": np.sum(R * R, axis=1)}
    if trace:
        info["objective"] = np.asarray(objective)
    return D, A, info
