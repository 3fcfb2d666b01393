"""Real spherical harmonics of degree 1..3 and radiance from sparse codes (FP64).

Sec. 2.2: the 45 non-DC SH coefficients of a Gaussian (15 basis functions x RGB)
are replaced by a shared dictionary and sparse codes, and the radiance step reads
the dictionary and the nonzeros directly.  The colour of Gaussian i seen along
unit direction v is, per channel c,

    rgb_c(v) = sum_{b=0..14} Y_b(v) * y[c*15 + b],     y = D alpha_i   (dense)

which the oracle evaluates literally: reconstruct y densely, then evaluate.

Basis convention: real SH with the Condon-Shortley phase, degree l = 1..3,
m = -l..l, basis index b = l*l + l + m - 1 (DC dropped), and
    Y_lm = sqrt(2) N_lm P_l^|m|(z) sin(|m| phi)   for m < 0
    Y_l0 = N_l0 P_l^0(z)
    Y_lm = sqrt(2) N_lm P_l^m(z) cos(m phi)       for m > 0
    N_lm = sqrt((2l+1)/(4 pi) * (l-|m|)! / (l+|m|)!)
with z = cos(theta) the direction's z component and phi = atan2(y, x).  The
constants are derived here from the Legendre recurrence, never typed in.

Pins (tests/test_oracle_sh.py): closed-form textbook values of the real SH,
scipy's complex spherical harmonics, orthonormality on the sphere under an exact
product quadrature, and decode linearity / 1-sparse special cases.
"""
from __future__ import annotations

import math

import numpy as np

LMAX = 3
N_BASIS = 15


def _double_factorial(n: int) -> int:
    out = 1
    while n > 1:
        out *= n
        n -= 2
    return out


def assoc_legendre(l: int, m: int, z: np.ndarray) -> np.ndarray:
    """P_l^m(z), 0 <= m <= l, including the Condon-Shortley phase (-1)^m."""
    z = np.asarray(z, dtype=np.float64)
    pmm = ((-1) ** m) * _double_factorial(2 * m - 1) * np.power(
        np.clip(1.0 - z * z, 0.0, None), 0.5 * m)
    if l == m:
        return pmm
    pm1 = z * (2 * m + 1) * pmm
    if l == m + 1:
        return pm1
    prev, cur = pmm, pm1
    for ll in range(m + 2, l + 1):
        nxt = ((2 * ll - 1) * z * cur - (ll + m - 1) * prev) / (ll - m)
        prev, cur = cur, nxt
    return cur


def norm_lm(l: int, m: int) -> float:
    am = abs(m)
    return math.sqrt((2 * l + 1) / (4.0 * math.pi)
                     * math.factorial(l - am) / math.factorial(l + am))


def basis_index(l: int, m: int) -> int:
    return l * l + l + m - 1


def sh_basis(dirs: np.ndarray) -> np.ndarray:
    """(n, 3) unit directions -> (n, 15) real SH values of degree 1..3."""
    dirs = np.asarray(dirs, dtype=np.float64)
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    phi = np.arctan2(y, x)
    out = np.empty((dirs.shape[0], N_BASIS))
    for l in range(1, LMAX + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            p = assoc_legendre(l, am, z)
            if m < 0:
                val = math.sqrt(2.0) * norm_lm(l, m) * p * np.sin(am * phi)
            elif m == 0:
                val = norm_lm(l, 0) * p
            else:
                val = math.sqrt(2.0) * norm_lm(l, m) * p * np.cos(m * phi)
            out[:, basis_index(l, m)] = val
    return out


def sh_eval(y: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    """Dense evaluation: y (n, 45) channel-major coefficients -> rgb (n, 3)."""
    y = np.asarray(y, dtype=np.float64)
    Y = sh_basis(dirs)  # (n, 15)
    return np.einsum("nb,ncb->nc", Y, y.reshape(-1, 3, N_BASIS))


def view_directions(means: np.ndarray, cam: np.ndarray) -> np.ndarray:
    """Unit view directions v_i = (mu_i - cam) / ||mu_i - cam||."""
    v = np.asarray(means, dtype=np.float64) - np.asarray(cam, dtype=np.float64)[None, :]
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def reconstruct(D: np.ndarray, idx: np.ndarray, coef: np.ndarray, nnz: np.ndarray) -> np.ndarray:
    """Dense y_i = sum_{t < nnz_i} coef[i,t] * D[idx[i,t]]  (D rows are atoms)."""
    D = np.asarray(D, dtype=np.float64)
    idx = np.asarray(idx, dtype=np.int64)
    coef = np.asarray(coef, dtype=np.float64)
    s = idx.shape[1]
    keep = np.arange(s)[None, :] < np.asarray(nnz)[:, None]
    c = np.where(keep, coef, 0.0)
    return np.einsum("ns,nsd->nd", c, D[idx])


def decode(D, idx, coef, nnz, dirs=None, means=None, cam=None) -> np.ndarray:
    """Radiance of each Gaussian from its sparse code: dense SH eval of D alpha."""
    if dirs is None:
        dirs = view_directions(means, cam)
    return sh_eval(reconstruct(D, idx, coef, nnz), dirs)


def full_colour(view, dc):
    """A Gaussian's colour with its DC term, in the usual 3DGS convention (the
    paper leaves the DC coefficient outside the dictionary, Sec. 2.2):
    max(0, Y00 dc + view-dependent part + 0.5), Y00 = N_00 = 1/(2 sqrt(pi))."""
    return np.maximum(0.0, norm_lm(0, 0) * np.asarray(dc, dtype=np.float64) + np.asarray(view, dtype=np.float64)
                      + 0.5)
