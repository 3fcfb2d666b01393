"""Pins of the splatting preprocess oracle (closed forms, finite differences,
symmetries); no GPU."""
import math

import numpy as np

from oracle import sh, splat

FX = FY = 800.0
W, H = 1280, 720
NEAR = 0.2


def _run(mu, scales, quats, Rv=np.eye(3), tv=np.zeros(3), dc=None, y=None):
    n = len(mu)
    dc = np.zeros((n, 3)) if dc is None else dc
    y = np.zeros((n, 45)) if y is None else y
    return splat.preprocess(np.asarray(mu, float), np.asarray(scales, float), np.asarray(quats, float), Rv, tv,
                            FX, FY, W, H, NEAR, dc, y=y)


def test_jacobian_matches_central_differences():
    rng = np.random.default_rng(0)
    pc = np.column_stack([rng.uniform(-1, 1, 50), rng.uniform(-0.5, 0.5, 50), rng.uniform(2, 6, 50)])
    J = splat.jacobian(pc, FX, FY, W, H)

    def proj(p):
        return np.stack([FX * p[:, 0] / p[:, 2], FY * p[:, 1] / p[:, 2]], axis=1)

    h = 1e-6
    for k in range(3):
        d = np.zeros(3)
        d[k] = h
        num = (proj(pc + d) - proj(pc - d)) / (2 * h)
        np.testing.assert_allclose(J[:, :, k], num, rtol=1e-6, atol=1e-6)


def test_isotropic_gaussian_on_axis_closed_form():
    z0, sig = 4.0, 0.05
    out = _run([[0.0, 0.0, z0]], [[sig, sig, sig]], [[1.0, 0.0, 0.0, 0.0]])
    v = (FX / z0) ** 2 * sig * sig + splat.LOWPASS
    np.testing.assert_allclose(out["xy"][0], [W / 2, H / 2])
    np.testing.assert_allclose(out["conic"][0], [1 / v, 0.0, 1 / v], rtol=1e-12)
    # lambda_max = v (mid^2 - det = 0 < 0.1, so sqrt(0.1) is added)
    assert out["radius"][0] == math.ceil(3 * math.sqrt(v + math.sqrt(0.1)))
    assert out["depth"][0] == z0


def test_isotropic_projection_ignores_rotation():
    rng = np.random.default_rng(1)
    mu = np.column_stack([rng.uniform(-1, 1, 20), rng.uniform(-0.5, 0.5, 20), rng.uniform(2, 5, 20)])
    s = np.full((20, 3), 0.03)
    a = _run(mu, s, np.tile([1.0, 0, 0, 0], (20, 1)))
    b = _run(mu, s, rng.standard_normal((20, 4)))
    np.testing.assert_allclose(a["conic"], b["conic"], rtol=1e-10)
    np.testing.assert_array_equal(a["radius"], b["radius"])


def test_quarter_turn_swaps_axes():
    # a 90-degree turn about z maps the x scale onto y
    q = np.array([[math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)]])
    S = splat.covariance3d(np.array([[0.3, 0.1, 0.2]]), q)[0]
    np.testing.assert_allclose(S, np.diag([0.01, 0.09, 0.04]), atol=1e-12)


def test_clamp_far_off_axis():
    pc = np.array([[10.0, 0.0, 2.0]])  # x/z = 5, beyond 1.3 * W / (2 fx) = 1.04
    J = splat.jacobian(pc, FX, FY, W, H)
    assert J[0, 0, 2] == -FX * (1.3 * 0.5 * W / FX) * 2.0 / 4.0


def test_culling():
    out = _run([[0.0, 0.0, -1.0], [0.0, 0.0, 0.1], [50.0, 0.0, 2.0], [0.0, 0.0, 3.0]],
               np.full((4, 3), 0.02), np.tile([1.0, 0, 0, 0], (4, 1)))
    assert list(out["radius"][:3]) == [0, 0, 0]  # behind, before the near plane, off screen
    assert out["radius"][3] > 0
    assert np.all(out["rgb"][:3] == 0) and np.all(out["conic"][:3] == 0)


def test_colour_of_zero_sh_and_codes_path():
    rng = np.random.default_rng(2)
    mu = np.column_stack([rng.uniform(-1, 1, 30), rng.uniform(-0.5, 0.5, 30), rng.uniform(2, 5, 30)])
    dc = rng.standard_normal((30, 3))
    out = _run(mu, np.full((30, 3), 0.02), np.tile([1.0, 0, 0, 0], (30, 1)), dc=dc)
    vis = out["radius"] > 0
    np.testing.assert_allclose(out["rgb"][vis], np.maximum(0, splat.Y00 * dc + 0.5)[vis])
    # colour from codes equals colour from the dense reconstruction
    K, s = 16, 3
    D = rng.standard_normal((K, 45))
    idx = np.stack([rng.choice(K, s, replace=False) for _ in range(30)])
    coef = rng.standard_normal((30, s))
    nnz = rng.integers(0, s + 1, 30)
    a = splat.preprocess(mu, np.full((30, 3), 0.02), np.tile([1.0, 0, 0, 0], (30, 1)), np.eye(3), np.zeros(3),
                         FX, FY, W, H, NEAR, dc, D=D, idx=idx, coef=coef, nnz=nnz)
    b = splat.preprocess(mu, np.full((30, 3), 0.02), np.tile([1.0, 0, 0, 0], (30, 1)), np.eye(3), np.zeros(3),
                         FX, FY, W, H, NEAR, dc, y=sh.reconstruct(D, idx, coef, nnz))
    np.testing.assert_allclose(a["rgb"], b["rgb"], rtol=1e-12)
    assert splat.Y00 == sh.norm_lm(0, 0)
    # the decode's full colour: Y00 = 1 / (2 sqrt(pi)) = 0.28209479177..., the
    # +0.5 offset and the clamp at zero
    np.testing.assert_allclose(sh.full_colour(np.zeros(3), [1.0, -3.0, 0.0]), [0.78209479177387814, 0.0, 0.5],
                               rtol=1e-15)
