"""Learned support proposal in FP64: MLP forward/backward, BCE loss, Adam, and the
candidate-restricted OMP with its fallback to plain OMP.

The network maps a signal to one logit per atom; trained on (signal, OMP support)
pairs produced by the codec itself, its top-2s logits name candidate atoms, and
OMP restricted to those candidates gives an s-sparse code.  Plain OMP (Sec. 2.1)
remains the reference: a signal falls back to it when the restricted code's
residual is worse.  This extends the paper's pipeline (the paper itself uses plain
OMP only); the definitions below are the textbook ones.

    xn  = x / ||x||            (x = 0 gives xn = 0)
    z1  = W1 xn + b1,  h1 = gelu(z1)      W1: (256, 45)
    z2  = W2 h1 + b2,  h2 = gelu(z2)      W2: (256, 256)
    z3  = W3 h2 + b3                      W3: (K, 256)
    gelu(z) = z * Phi(z) = 0.5 z (1 + erf(z / sqrt 2))        (exact erf form)
    loss = mean over batch and atoms of BCE-with-logits(z3, y),
           y = multi-hot OMP support;  BCE(z, y) = max(z, 0) - z y + log(1 + e^-|z|)
    Adam: m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
          p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)

Fallback rule ("exact" mode): fall back iff ||r_learned|| > ||r_omp|| (1 + 1e-6).

Pins (tests/test_oracle_mlp.py): central finite differences of the loss against
the analytic gradients; BCE against its closed form at hand-picked logits; gelu
against math.erf; Adam against a hand-worked first step.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from .omp import omp, omp_restricted

FALLBACK_REL = 1e-6


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def normalise_input(X):
    X = np.asarray(X, dtype=np.float64)
    n = np.linalg.norm(X, axis=1, keepdims=True)
    return np.where(n > 0.0, X / np.where(n > 0.0, n, 1.0), 0.0)


def forward(p, X):
    xn = normalise_input(X)
    z1 = xn @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    z3 = h2 @ p["W3"].T + p["b3"]
    return {"xn": xn, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "z3": z3}


def bce_with_logits(z, y):
    z = np.asarray(z, dtype=np.float64)
    return np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))


def loss(p, X, Y):
    return float(bce_with_logits(forward(p, X)["z3"], Y).mean())


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def backward(p, X, Y):
    """Gradients of `loss` with respect to every parameter."""
    f = forward(p, X)
    n, K = f["z3"].shape
    dz3 = (sigmoid(f["z3"]) - Y) / (n * K)
    g = {"W3": dz3.T @ f["h2"], "b3": dz3.sum(axis=0)}
    dh2 = dz3 @ p["W3"]
    dz2 = dh2 * gelu_grad(f["z2"])
    g["W2"] = dz2.T @ f["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * gelu_grad(f["z1"])
    g["W1"] = dz1.T @ f["xn"]
    g["b1"] = dz1.sum(axis=0)
    return g, f


def adam_step(p, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (p, m, v)."""
    p2, m2, v2 = {}, {}, {}
    for k in p:
        m2[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
        v2[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k]
        mh = m2[k] / (1.0 - beta1 ** t)
        vh = v2[k] / (1.0 - beta2 ** t)
        p2[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p2, m2, v2


def support_targets(idx, nnz, K: int):
    """Multi-hot (N, K) target from ELL supports."""
    idx = np.asarray(idx)
    N, s = idx.shape
    Y = np.zeros((N, K))
    keep = np.arange(s)[None, :] < np.asarray(nnz)[:, None]
    rows = np.repeat(np.arange(N), s).reshape(N, s)
    Y[rows[keep], idx[keep]] = 1.0
    return Y


def top_candidates(z3, m: int):
    """Indices of the m largest logits per row, by decreasing logit, ties to smaller index."""
    z3 = np.asarray(z3)
    order = np.lexsort((np.broadcast_to(np.arange(z3.shape[1]), z3.shape), -z3), axis=1)
    return order[:, :m]


def encode_learned(p, D, X, s: int, eps: float = 0.0):
    """Learned proposal + restricted OMP + exact-mode fallback to plain OMP."""
    cand = top_candidates(forward(p, X)["z3"], 2 * s)
    lr = omp_restricted(D, X, cand, s, eps)
    pl = omp(D, X, s, eps)
    fb = np.sqrt(lr["resid_sq"]) > np.sqrt(pl["resid_sq"]) * (1.0 + FALLBACK_REL)
    out = {k: np.where(fb[:, None] if lr[k].ndim == 2 else fb, pl[k], lr[k])
           for k in ("idx", "coef", "nnz", "resid_sq")}
    out["fallback"] = fb
    out["cand"] = cand
    return out
