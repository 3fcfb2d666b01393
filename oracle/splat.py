"""Gaussian-splatting preprocess with colour from SH or from sparse codes (FP64).

Test infrastructure only: the tests, smoke() and bench.py's CPU legs use it; the
library never does.

The paper's rendering claim (Sec. 2.2, Eqs. 2-3) is that the colour step reads
the small shared dictionary and a Gaussian's nonzeros instead of its 45 SH
coefficients.  The colour step sits in the renderer's per-Gaussian preprocess,
which this module spells out in the usual splatting form (the paper does not
restate it; the reading is listed in the design notes):

  camera      world -> camera p_c = Rv p + tv; focal lengths fx, fy in pixels;
              image W x H with the principal point at its centre; near plane
              z_near.  The camera centre is c = -Rv^T tv.
  visibility  z_c > z_near, a positive-definite screen covariance, and a
              3-sigma square that meets the image.
  covariance  Sigma = R(q) diag(s^2) R(q)^T for unit quaternion q = (w, x, y, z)
  projection  J = [[fx/z, 0, -fx tx/z^2], [0, fy/z, -fy ty/z^2]] with
              tx = clamp(x/z, +-1.3 W/(2 fx)) z (likewise ty), and
              Sigma_2D = J Rv Sigma Rv^T J^T + 0.3 I (the low-pass term)
  outputs     pixel centre (fx x/z + W/2, fy y/z + H/2), depth z,
              conic = Sigma_2D^-1 as (a, b, c) for [[a, b], [b, c]],
              radius = ceil(3 sqrt(lambda_max)) with
              lambda_max = mid + sqrt(max(0.1, mid^2 - det)), mid = trace/2
  colour      rgb = max(0, Y00 dc + sum_b Y_b(v) y_{c,b} + 0.5) along
              v = (mu - c)/||mu - c||, with y the dense SH (45 per Gaussian) or
              D alpha from the sparse codes; Y00 = 1/(2 sqrt(pi)).
Invisible Gaussians get radius 0 and zeros elsewhere.

Pins (tests/test_oracle_splat.py): the Jacobian against central differences of
the projection, an isotropic Gaussian on the optical axis in closed form,
rotation invariance of isotropic Gaussians, a 90-degree quaternion that swaps
two axes, the quaternion rotation against scipy's, invariance of the geometry
under a joint rotation of scene and camera, the conic as the inverse of the
screen covariance, the clamp far off-axis in x and y, culling behind the
camera and off-screen, the colour of zero SH, and the colour along the
direction from a camera built at a known position.
"""
from __future__ import annotations

import math

import numpy as np

from . import sh

Y00 = 0.5 / math.sqrt(math.pi)
LOWPASS = 0.3
CLAMP = 1.3


def quat_to_rot(q: np.ndarray) -> np.ndarray:
    """(N, 4) quaternions (w, x, y, z), normalised here -> (N, 3, 3) rotations."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def covariance3d(scales: np.ndarray, quats: np.ndarray) -> np.ndarray:
    R = quat_to_rot(quats)
    S2 = np.asarray(scales, dtype=np.float64) ** 2
    return np.einsum("nij,nj,nkj->nik", R, S2, R)


def jacobian(pc: np.ndarray, fx: float, fy: float, W: int, H: int) -> np.ndarray:
    """(N, 2, 3) Jacobian of the perspective projection at camera points pc,
    with the view-frustum clamp of the x/z and y/z ratios."""
    x, y, z = pc[:, 0], pc[:, 1], pc[:, 2]
    limx = CLAMP * 0.5 * W / fx
    limy = CLAMP * 0.5 * H / fy
    tx = np.clip(x / z, -limx, limx) * z
    ty = np.clip(y / z, -limy, limy) * z
    J = np.zeros((pc.shape[0], 2, 3))
    J[:, 0, 0] = fx / z
    J[:, 0, 2] = -fx * tx / (z * z)
    J[:, 1, 1] = fy / z
    J[:, 1, 2] = -fy * ty / (z * z)
    return J


def preprocess(means, scales, quats, Rv, tv, fx, fy, W, H, z_near, dc, y=None, D=None, idx=None,
               coef=None, nnz=None):
    """Per-Gaussian preprocess.  Colour from dense SH y (N, 45) or from codes
    (D, idx, coef, nnz).  Returns dict of xy (N, 2), depth (N,), conic (N, 3),
    radius (N,) int, rgb (N, 3), and under "raw" the unmasked z, pixel centre,
    det and 3 sqrt(lambda_max) from which visibility and the radius were decided."""
    mu = np.asarray(means, dtype=np.float64)
    N = mu.shape[0]
    Rv = np.asarray(Rv, dtype=np.float64)
    tv = np.asarray(tv, dtype=np.float64)
    pc = mu @ Rv.T + tv
    z = pc[:, 2]
    front = z > z_near
    zs = np.where(front, z, 1.0)
    pcs = np.where(front[:, None], pc, np.array([0.0, 0.0, 1.0]))
    J = jacobian(pcs, fx, fy, W, H)
    T = J @ Rv
    S3 = covariance3d(scales, quats)
    S2 = T @ S3 @ np.transpose(T, (0, 2, 1))
    a = S2[:, 0, 0] + LOWPASS
    b = S2[:, 0, 1]
    c = S2[:, 1, 1] + LOWPASS
    det = a * c - b * b
    ok = front & (det > 0.0)
    dets = np.where(ok, det, 1.0)
    mid = 0.5 * (a + c)
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - det))
    radius = np.ceil(3.0 * np.sqrt(np.maximum(lam, 0.0)))
    px = fx * pcs[:, 0] / zs + 0.5 * W
    py = fy * pcs[:, 1] / zs + 0.5 * H
    onscreen = (px + radius > 0) & (px - radius < W) & (py + radius > 0) & (py - radius < H)
    vis = ok & onscreen
    out = {
        "xy": np.where(vis[:, None], np.stack([px, py], axis=1), 0.0),
        "depth": np.where(vis, z, 0.0),
        "conic": np.where(vis[:, None], np.stack([c / dets, -b / dets, a / dets], axis=1), 0.0),
        "radius": np.where(vis, radius, 0).astype(np.int64),
        "raw": {"z": z, "px": px, "py": py, "det": det, "extent": 3.0 * np.sqrt(np.maximum(lam, 0.0)),
                "front": front},
    }
    cam = -Rv.T @ tv
    dirs = sh.view_directions(mu, cam)
    if y is None:
        y = sh.reconstruct(np.asarray(D, dtype=np.float64), idx, coef, nnz)
    view = sh.sh_eval(np.asarray(y, dtype=np.float64), dirs)
    rgb = np.maximum(0.0, Y00 * np.asarray(dc, dtype=np.float64) + view + 0.5)
    out["rgb"] = np.where(vis[:, None], rgb, 0.0)
    return out
