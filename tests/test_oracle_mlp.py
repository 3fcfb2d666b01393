"""Pins for oracle.mlp: gradients by finite differences, BCE/GELU closed forms, Adam."""
import math

import numpy as np

from oracle import mlp as P
from paper_2605_30396_gb300 import synth


def _small():
    rng = np.random.default_rng(0)
    p = synth.mlp_params(12, 1, hidden=7)
    p = {k: v + 0.05 * rng.standard_normal(v.shape) for k, v in p.items()}
    X = rng.standard_normal((5, 45))
    Y = (rng.random((5, 12)) < 0.3).astype(float)
    return p, X, Y


def test_gradients_finite_difference():
    p, X, Y = _small()
    g, _ = P.backward(p, X, Y)
    h = 1e-6
    rng = np.random.default_rng(1)
    for k in p:
        flat = p[k].reshape(-1)
        for e in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[e]
            flat[e] = old + h
            lp = P.loss(p, X, Y)
            flat[e] = old - h
            lm = P.loss(p, X, Y)
            flat[e] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[e]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)) + 1e-9, (k, e, fd, an)


def test_bce_closed_form():
    z = np.array([-30.0, -2.0, 0.0, 1.5, 40.0])
    for y in (0.0, 1.0):
        ref = [-(y * math.log(1 / (1 + math.exp(-v))) + (1 - y) * math.log(1 - 1 / (1 + math.exp(-v))))
               if abs(v) < 20 else (max(v, 0) - v * y + math.log1p(math.exp(-abs(v)))) for v in z]
        np.testing.assert_allclose(P.bce_with_logits(z, y), ref, rtol=1e-12)


def test_gelu_and_grad():
    z = np.linspace(-5, 5, 21)
    ref = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in z])
    np.testing.assert_allclose(P.gelu(z), ref, rtol=1e-14, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(P.gelu_grad(z), (P.gelu(z + h) - P.gelu(z - h)) / (2 * h), atol=1e-8)


def test_adam_first_step_is_sign_step():
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -0.25, 0.0])}
    z = {"w": np.zeros(3)}
    p2, m, v = P.adam_step(p, g, z, z, 1, lr=0.1)
    # bias-corrected m/sqrt(v) = g/|g| at t = 1
    np.testing.assert_allclose(p2["w"], [0.9, -1.9, 3.0], atol=1e-7)
    np.testing.assert_allclose(m["w"], 0.1 * g["w"])
    np.testing.assert_allclose(v["w"], 0.001 * g["w"] ** 2)


def test_top_candidates_ties():
    z = np.array([[0.5, 2.0, 2.0, -1.0, 0.5]])
    np.testing.assert_array_equal(P.top_candidates(z, 3), [[1, 2, 0]])


def test_encode_learned_never_worse_than_plain():
    D = synth.hidden_dictionary(32, 3)
    X = synth.signals(60, D, 3, 4, dtype=np.float64)
    p = synth.mlp_params(32, 5, hidden=16)
    out = P.encode_learned(p, D, X, 3)
    from oracle.omp import omp
    pl = omp(D, X, 3)
    assert (np.sqrt(out["resid_sq"]) <= np.sqrt(pl["resid_sq"]) * (1 + 1e-6) + 1e-15).all()


def test_input_is_normalised():
    """The network sees x / ||x||: scaling a signal leaves the logits unchanged,
    and a zero signal gives the biases' forward pass."""
    K = 32
    p = synth.mlp_params(K, 3)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((5, 45))
    np.testing.assert_allclose(P.forward(p, 3.7 * X)["z3"], P.forward(p, X)["z3"], rtol=1e-12)
    z0 = P.forward(p, np.zeros((1, 45)))
    np.testing.assert_allclose(z0["z1"], p["b1"][None, :], atol=0)


def test_adam_epsilon_outside_the_root():
    """eps is added to sqrt(v_hat): with g = 1e-9 the first step is
    lr * 1e-9 / (1e-9 + 1e-8) = lr / 11."""
    p = {"w": np.zeros(1)}
    g = {"w": np.array([1e-9])}
    z = {"w": np.zeros(1)}
    p2, _, _ = P.adam_step(p, g, z, z, 1, lr=1.0)
    np.testing.assert_allclose(p2["w"], [-1.0 / 11.0], rtol=1e-12)


def test_support_targets_ignore_padding_slots():
    Y = P.support_targets(np.array([[3, 5], [1, 2]]), np.array([1, 0]), 8)
    want = np.zeros((2, 8))
    want[0, 3] = 1.0
    np.testing.assert_array_equal(Y, want)
