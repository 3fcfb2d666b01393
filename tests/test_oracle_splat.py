"""Pins of the splatting preprocess oracle (closed forms, finite differences,
symmetries); no GPU."""
import math

import numpy as np

from oracle import sh, splat
from paper_2605_30396_gb300 import synth

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
    pc = np.array([[0.0, -10.0, 2.0]])  # y/z = -5, beyond -1.3 * H / (2 fy) = -0.585
    J = splat.jacobian(pc, FX, FY, W, H)
    assert J[0, 1, 2] == FY * (1.3 * 0.5 * H / FY) * 2.0 / 4.0
    assert J[0, 0, 2] == 0.0


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


def _scipy_rot():
    from scipy.spatial.transform import Rotation
    return Rotation


def test_quaternion_rotation_matches_scipy():
    Rotation = _scipy_rot()
    rng = np.random.default_rng(5)
    q = rng.standard_normal((40, 4))  # (w, x, y, z), unnormalised
    ref = Rotation.from_quat(np.column_stack([q[:, 1:], q[:, :1]])).as_matrix()  # scipy: (x, y, z, w)
    np.testing.assert_allclose(splat.quat_to_rot(q), ref, atol=1e-12)


def test_geometry_invariant_under_a_joint_rotation_of_scene_and_camera():
    """Rotating the means, the Gaussians' orientations and the camera by the same
    rotation Q (R_v -> R_v Q^T) leaves every camera-space quantity unchanged."""
    Rotation = _scipy_rot()
    rng = np.random.default_rng(6)
    n = 200
    mu = np.column_stack([rng.uniform(-1, 1, n), rng.uniform(-0.5, 0.5, n), rng.uniform(2, 5, n)])
    sc = np.exp(rng.normal(np.log(0.05), 0.5, (n, 3)))
    q = rng.standard_normal((n, 4))
    Rv = Rotation.from_euler("xyz", [0.1, -0.2, 0.3]).as_matrix()
    tv = np.array([0.2, -0.1, 0.5])
    Q = Rotation.from_euler("zyx", [0.7, 0.4, -1.1])
    a = splat.preprocess(mu, sc, q, Rv, tv, FX, FY, W, H, NEAR, np.zeros((n, 3)), y=np.zeros((n, 45)))
    rq = Q * Rotation.from_quat(np.column_stack([q[:, 1:], q[:, :1]]))
    q2 = rq.as_quat()
    q2 = np.column_stack([q2[:, 3:], q2[:, :3]])  # back to (w, x, y, z)
    Qm = Q.as_matrix()
    b = splat.preprocess(mu @ Qm.T, sc, q2, Rv @ Qm.T, tv, FX, FY, W, H, NEAR, np.zeros((n, 3)),
                         y=np.zeros((n, 45)))
    assert (a["radius"] > 0).sum() > 100
    np.testing.assert_array_equal(a["radius"], b["radius"])
    for k in ("xy", "depth", "conic"):
        np.testing.assert_allclose(b[k], a[k], rtol=1e-9, atol=1e-9)


def test_conic_inverts_the_screen_covariance():
    """conic, read as [[c0, c1], [c1, c2]], times J R_v Sigma R_v^T J^T + 0.3 I is
    the identity (J and Sigma from the functions pinned above)."""
    Rotation = _scipy_rot()
    rng = np.random.default_rng(8)
    n = 100
    mu = np.column_stack([rng.uniform(-1, 1, n), rng.uniform(-0.5, 0.5, n), rng.uniform(2, 5, n)])
    sc = np.exp(rng.normal(np.log(0.05), 0.7, (n, 3)))
    q = rng.standard_normal((n, 4))
    Rv = Rotation.from_euler("xyz", [0.05, 0.1, -0.2]).as_matrix()
    tv = np.array([0.1, 0.0, 0.3])
    out = splat.preprocess(mu, sc, q, Rv, tv, FX, FY, W, H, NEAR, np.zeros((n, 3)), y=np.zeros((n, 45)))
    vis = out["radius"] > 0
    assert vis.sum() > 50
    J = splat.jacobian(mu @ Rv.T + tv, FX, FY, W, H)
    T = J @ Rv
    S2 = T @ splat.covariance3d(sc, q) @ np.transpose(T, (0, 2, 1)) + splat.LOWPASS * np.eye(2)
    c = out["conic"]
    C = np.stack([np.stack([c[:, 0], c[:, 1]], -1), np.stack([c[:, 1], c[:, 2]], -1)], 1)
    np.testing.assert_allclose((C @ S2)[vis], np.broadcast_to(np.eye(2), (vis.sum(), 2, 2)), atol=1e-9)


def test_colour_uses_the_direction_from_the_camera_centre():
    """With the camera built at a known eye position, the colour of a Gaussian is
    evaluated along (mu - eye) / |mu - eye|."""
    from oracle import sh as osh
    rng = np.random.default_rng(9)
    n = 60
    eye = np.array([0.3, -2.5, 0.8])
    R, t = synth.look_at(eye, (0.0, 0.0, 0.0))
    mu = rng.uniform(-0.5, 0.5, (n, 3))
    y = rng.standard_normal((n, 45))
    dc = rng.standard_normal((n, 3))
    out = splat.preprocess(mu, np.full((n, 3), 0.02), np.tile([1.0, 0, 0, 0], (n, 1)), R, t, FX, FY, W, H, NEAR,
                           dc, y=y)
    assert (out["radius"] > 0).all()
    v = (mu - eye) / np.linalg.norm(mu - eye, axis=1, keepdims=True)
    ref = np.maximum(0.0, splat.Y00 * dc + osh.sh_eval(y, v) + 0.5)
    np.testing.assert_allclose(out["rgb"], ref, rtol=1e-12, atol=1e-12)
