"""The on-device signal generator follows the same recipe as the host one
(drawn here on the CPU device of torch, so no GPU is needed)."""
import numpy as np
import torch

from paper_2605_30396_gb300 import synth


def test_supports_are_s_distinct_atoms_with_laplace_coefficients():
    # identity atoms and no noise: each row is its coefficients at its support
    X = synth.signals_device(100_000, np.eye(45), 6, 3, noise_std=0.0, device="cpu").numpy()
    nz = X != 0
    assert (nz.sum(axis=1) == 6).all()
    c = X[nz]
    # Laplace(0, 1): E|c| = 1, Var = 2, median |c| = ln 2
    assert abs(np.abs(c).mean() - 1.0) < 0.01
    assert abs(c.var() - 2.0) < 0.04
    assert abs(np.median(np.abs(c)) - np.log(2.0)) < 0.01
    # every atom equally likely
    freq = nz.sum(axis=0) / nz.sum()
    assert np.abs(freq - 1 / 45).max() < 0.1 / 45


def test_matches_the_host_generator_in_distribution():
    D = synth.hidden_dictionary(64, 0)
    Xh = synth.signals(200_000, D, 4, 1)
    Xd = synth.signals_device(200_000, D, 4, 1, device="cpu").numpy()
    for q in (50, 90, 99):
        a, b = np.percentile(np.abs(Xh), q), np.percentile(np.abs(Xd), q)
        assert abs(a - b) <= 0.02 * a, (q, a, b)
    assert abs(Xh.std() - Xd.std()) <= 0.01 * Xh.std()


def test_noise_level_and_seed():
    X = synth.signals_device(50_000, np.zeros((8, 45)), 3, 5, noise_std=1e-3, device="cpu")
    assert abs(float(X.std()) - 1e-3) < 2e-5
    Y = synth.signals_device(50_000, np.zeros((8, 45)), 3, 5, noise_std=1e-3, device="cpu")
    assert torch.equal(X, Y)
