"""Pins for oracle.sh: real SH of degree 1..3 and decode-from-codes."""
import math

import numpy as np
import pytest
from scipy.special import sph_harm_y

from oracle import sh
from paper_2605_30396_gb300 import synth


def _dirs(n=64, seed=5):
    return synth.unit_directions(n, seed, dtype=np.float64)


def test_closed_forms_textbook():
    """Closed-form real SH (Condon-Shortley phase) written out in Cartesian form."""
    v = _dirs()
    x, y, z = v[:, 0], v[:, 1], v[:, 2]
    pi = math.pi
    ref = np.stack([
        -math.sqrt(3 / (4 * pi)) * y,
        math.sqrt(3 / (4 * pi)) * z,
        -math.sqrt(3 / (4 * pi)) * x,
        0.5 * math.sqrt(15 / pi) * x * y,
        -0.5 * math.sqrt(15 / pi) * y * z,
        0.25 * math.sqrt(5 / pi) * (3 * z * z - 1),
        -0.5 * math.sqrt(15 / pi) * x * z,
        0.25 * math.sqrt(15 / pi) * (x * x - y * y),
        -0.25 * math.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y),
        0.5 * math.sqrt(105 / pi) * x * y * z,
        -0.25 * math.sqrt(21 / (2 * pi)) * y * (5 * z * z - 1),
        0.25 * math.sqrt(7 / pi) * z * (5 * z * z - 3),
        -0.25 * math.sqrt(21 / (2 * pi)) * x * (5 * z * z - 1),
        0.25 * math.sqrt(105 / pi) * z * (x * x - y * y),
        -0.25 * math.sqrt(35 / (2 * pi)) * x * (x * x - 3 * y * y),
    ], axis=1)
    np.testing.assert_allclose(sh.sh_basis(v), ref, rtol=0, atol=1e-13)


def test_against_scipy_complex_sh():
    """Real form of scipy's complex Y_l^m: sqrt2 Re (m>0), sqrt2 Im (m<0), Y_l^0."""
    v = _dirs(200, 9)
    theta = np.arccos(np.clip(v[:, 2], -1, 1))
    phi = np.arctan2(v[:, 1], v[:, 0])
    B = sh.sh_basis(v)
    for l in range(1, 4):
        for m in range(-l, l + 1):
            Yc = sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                ref = math.sqrt(2) * Yc.real
            elif m < 0:
                ref = math.sqrt(2) * Yc.imag
            else:
                ref = Yc.real
            np.testing.assert_allclose(B[:, sh.basis_index(l, m)], ref, atol=1e-12)


def test_orthonormal_on_sphere():
    """Gauss-Legendre in cos(theta) x uniform phi is exact for these degree-<=6 products."""
    zq, wq = np.polynomial.legendre.leggauss(8)
    nphi = 16
    phi = 2 * np.pi * np.arange(nphi) / nphi
    Z, P = np.meshgrid(zq, phi, indexing="ij")
    W = np.repeat(wq[:, None], nphi, axis=1) * (2 * np.pi / nphi)
    r = np.sqrt(1 - Z ** 2)
    dirs = np.stack([r * np.cos(P), r * np.sin(P), Z], axis=-1).reshape(-1, 3)
    B = sh.sh_basis(dirs)
    gram = B.T @ (B * W.reshape(-1)[:, None])
    np.testing.assert_allclose(gram, np.eye(15), atol=1e-12)


def test_decode_linearity_and_one_sparse():
    rng = np.random.default_rng(3)
    K, n, s = 16, 50, 3
    D = synth.hidden_dictionary(K, 1)
    idx = synth.distinct_supports(rng, n, K, s)
    coef = rng.standard_normal((n, s))
    nnz = np.full(n, s)
    dirs = _dirs(n, 4)
    rgb = sh.decode(D, idx, coef, nnz, dirs=dirs)
    # sum of 1-sparse decodes (linearity in the code)
    acc = np.zeros((n, 3))
    for t in range(s):
        acc += coef[:, t:t + 1] * sh.sh_eval(D[idx[:, t]], dirs)
    np.testing.assert_allclose(rgb, acc, atol=1e-12)
    # nnz masks trailing slots
    nnz2 = np.full(n, 1)
    rgb1 = sh.decode(D, idx, coef, nnz2, dirs=dirs)
    np.testing.assert_allclose(rgb1, coef[:, :1] * sh.sh_eval(D[idx[:, 0]], dirs), atol=1e-12)


def test_view_directions_from_camera():
    cam = np.array([0.0, 0.0, 4.0])
    mu = np.array([[0.0, 0.0, 0.0], [4.0, 0.0, 4.0]])
    v = sh.view_directions(mu, cam)
    np.testing.assert_allclose(v, [[0, 0, -1], [1, 0, 0]], atol=1e-15)


@pytest.mark.parametrize("l", [1, 2, 3])
def test_legendre_recurrence_closed_form(l):
    z = np.linspace(-1, 1, 11)
    s2 = np.sqrt(1 - z * z)
    table = {
        (1, 0): z, (1, 1): -s2,
        (2, 0): 0.5 * (3 * z * z - 1), (2, 1): -3 * z * s2, (2, 2): 3 * (1 - z * z),
        (3, 0): 0.5 * (5 * z ** 3 - 3 * z), (3, 1): -1.5 * (5 * z * z - 1) * s2,
        (3, 2): 15 * z * (1 - z * z), (3, 3): -15 * s2 ** 3,
    }
    for m in range(l + 1):
        np.testing.assert_allclose(sh.assoc_legendre(l, m, z), table[(l, m)], atol=1e-13)


def test_channel_major_layout():
    """Coefficient c*15 + b belongs to channel c and basis b: a single unit
    coefficient at (c, b = 1, the l = 1, m = 0 basis sqrt(3/(4 pi)) z) lights
    channel c only."""
    v = np.array([[0.36, -0.48, 0.8]])
    for c in range(3):
        y = np.zeros((1, 45))
        y[0, c * 15 + 1] = 1.0
        rgb = sh.sh_eval(y, v)[0]
        want = np.zeros(3)
        want[c] = math.sqrt(3.0 / (4.0 * math.pi)) * 0.8
        np.testing.assert_allclose(rgb, want, atol=1e-15)
