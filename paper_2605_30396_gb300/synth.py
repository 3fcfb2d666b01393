"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the bench.

This module holds only input generation (random draws and their packing); none of
the codec's arithmetic (sparse coding, dictionary update, SH evaluation) lives
here, so both sides of every parity test can take their inputs from it.

Signal model (stand-in for the 45 non-DC SH coefficients per Gaussian of a
trained 3DGS model, Sec. 2.2): a hidden unit-norm dictionary of K atoms whose
entries have per-SH-degree standard deviations 0.15 / 0.08 / 0.04 (degree 1, 2,
3), optionally with correlation rho between the R, G, B entries of the same
basis function; each signal is s distinct hidden atoms with Laplace(b=1)
coefficients plus N(0, sigma_noise^2) noise.  Layout is channel-major:
x[c*15 + b], c in {R, G, B}, b = SH basis index 0..14 (degree 1..3).
"""
from __future__ import annotations

import numpy as np

D_SH = 45
N_BASIS = 15
# SH degree of basis b (0-based over degrees 1..3): 3 of degree 1, 5 of 2, 7 of 3.
BASIS_DEGREE = np.array([1] * 3 + [2] * 5 + [3] * 7)
DEGREE_STD = {1: 0.15, 2: 0.08, 3: 0.04}


def hidden_dictionary(K: int, seed: int, rho: float = 0.0, dtype=np.float64) -> np.ndarray:
    """Hidden unit-norm atoms, shape (K, 45), row j = atom j (channel-major)."""
    rng = np.random.default_rng(seed)
    std_b = np.array([DEGREE_STD[int(l)] for l in BASIS_DEGREE])  # (15,)
    # (R,G,B) triple of each basis entry ~ N(0, Sigma), Sigma = (1-rho) I + rho 11^T
    cov = (1.0 - rho) * np.eye(3) + rho * np.ones((3, 3))
    chol = np.linalg.cholesky(cov)
    z = rng.standard_normal((K, N_BASIS, 3)) @ chol.T  # (K, 15, 3)
    z = z * std_b[None, :, None]
    atoms = np.transpose(z, (0, 2, 1)).reshape(K, D_SH)  # channel-major
    atoms /= np.linalg.norm(atoms, axis=1, keepdims=True)
    return atoms.astype(dtype)


def distinct_supports(rng: np.random.Generator, N: int, K: int, s: int) -> np.ndarray:
    """(N, s) int64 array of s distinct atom indices per row, uniform."""
    sup = rng.integers(0, K, size=(N, s))
    while True:
        srt = np.sort(sup, axis=1)
        bad = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0]
        if bad.size == 0:
            return sup
        sup[bad] = rng.integers(0, K, size=(bad.size, s))


def signals(N: int, atoms: np.ndarray, s: int, seed: int, noise_std: float = 1e-3,
            dtype=np.float32, chunk: int = 1 << 18) -> np.ndarray:
    """(N, 45) signals: s-sparse Laplace(1) combinations of hidden atoms + noise."""
    rng = np.random.default_rng(seed)
    K = atoms.shape[0]
    out = np.empty((N, D_SH), dtype=dtype)
    for lo in range(0, N, chunk):
        n = min(chunk, N - lo)
        sup = distinct_supports(rng, n, K, s)
        coef = rng.laplace(0.0, 1.0, size=(n, s))
        x = np.einsum("ns,nsd->nd", coef, atoms[sup])
        x += noise_std * rng.standard_normal((n, D_SH))
        out[lo:lo + n] = x
    return out


def unit_directions(N: int, seed: int, dtype=np.float32) -> np.ndarray:
    """(N, 3) uniform unit vectors (normalised N(0, I3))."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((N, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v.astype(dtype)


def camera_and_means(N: int, cam_seed: int, mean_seed: int, radius: float = 4.0,
                     dtype=np.float32):
    """Camera position radius*u (u uniform on S^2) and Gaussian means ~ U[-1,1]^3."""
    cam = radius * unit_directions(1, cam_seed, dtype=np.float64)[0]
    rng = np.random.default_rng(mean_seed)
    mu = rng.uniform(-1.0, 1.0, size=(N, 3))
    return cam.astype(dtype), mu.astype(dtype)


def init_atom_indices(N: int, K: int, seed: int) -> np.ndarray:
    """K distinct signal indices whose (normalised) signals seed the dictionary."""
    return np.random.default_rng(seed).choice(N, K, replace=False)


def erc_dictionary(n: int) -> np.ndarray:
    """[I | H/sqrt(n)] (2n atoms of dimension n, rows = atoms), mutual coherence 1/sqrt(n).

    H is the Sylvester Hadamard matrix, so n must be a power of two.
    """
    H = np.array([[1.0]])
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    assert H.shape[0] == n
    return np.concatenate([np.eye(n), H.T / np.sqrt(n)], axis=0)


def planted_sparse(rng: np.random.Generator, atoms: np.ndarray, N: int, s: int,
                   min_abs: float = 0.5):
    """Exactly s-sparse signals (no noise) with coefficient magnitudes >= min_abs."""
    K = atoms.shape[0]
    sup = distinct_supports(rng, N, K, s)
    mag = min_abs + rng.exponential(1.0, size=(N, s))
    sign = rng.choice([-1.0, 1.0], size=(N, s))
    coef = mag * sign
    x = np.einsum("ns,nsd->nd", coef, atoms[sup])
    return x, sup, coef


def mlp_params(K: int, seed: int, d_in: int = D_SH, hidden: int = 256):
    """He-style random init for the 45->256->256->K support-proposal network."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((hidden, d_in)) * np.sqrt(2.0 / d_in)
    W2 = rng.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden)
    W3 = rng.standard_normal((K, hidden)) * np.sqrt(1.0 / hidden)
    b1 = np.zeros(hidden)
    b2 = np.zeros(hidden)
    b3 = np.full(K, -np.log(K / 16.0))
    return {"W1": W1, "b1": b1, "W2": W2, "b2": b2, "W3": W3, "b3": b3}


def splat_gaussians(N: int, seed: int, log_scale_mean: float = float(np.log(0.01)),
                    log_scale_std: float = 0.5, dtype=np.float32):
    """Gaussians of a splatting scene: means ~ U[-1,1]^3, per-axis scales
    exp(N(log_scale_mean, log_scale_std^2)), unnormalised rotations q ~ N(0, I4)
    as (w, x, y, z), and DC colours ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(N, 3))
    scales = np.exp(rng.normal(log_scale_mean, log_scale_std, size=(N, 3)))
    quats = rng.standard_normal((N, 4))
    dc = rng.standard_normal((N, 3))
    return tuple(a.astype(dtype) for a in (means, scales, quats, dc))


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)):
    """World -> camera pose (R, t) of a camera at `eye` looking at `target`,
    camera axes x right, y down, z forward: p_c = R p + t."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, dtype=np.float64)
    if abs(float(f @ up)) > 0.99 * np.linalg.norm(up):
        up = np.array([0.0, 1.0, 0.0]) if abs(f[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    return R, -R @ eye


def random_codes(N: int, K: int, s: int, seed: int, nnz_min: int = 0):
    """Random ELL codes: uniform indices (repeats allowed), N(0,1) coefficients,
    nnz uniform in [nnz_min, s]; slots t >= nnz hold index 0 and coefficient 0."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, K, size=(N, s))
    coef = rng.standard_normal((N, s))
    nnz = rng.integers(nnz_min, s + 1, size=N)
    pad = np.arange(s)[None, :] >= nnz[:, None]
    idx[pad] = 0
    coef[pad] = 0.0
    return idx.astype(np.uint16), coef.astype(np.float32), nnz.astype(np.uint8)


def signals_device(N: int, atoms, s: int, seed: int, noise_std: float = 1e-3,
                   device="cuda", chunk: int = 1 << 20):
    """`signals` drawn on the GPU with torch's seeded generator: the same recipe
    (s distinct uniform atoms per signal, Laplace(b=1) coefficients, N(0,
    noise_std^2) noise), another random stream.  For bench-scale inputs, where
    drawing tens of millions of signals on the host would dominate the run.
    Returns an (N, 45) float32 CUDA tensor."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    A = torch.as_tensor(np.asarray(atoms), dtype=torch.float32, device=device)
    K = A.shape[0]
    out = torch.empty((N, D_SH), dtype=torch.float32, device=device)
    for lo in range(0, N, chunk):
        n = min(chunk, N - lo)
        # s distinct atoms: draw, then redraw every row that holds a repeat
        sup = torch.randint(0, K, (n, s), generator=g, device=device)
        while True:
            srt, _ = torch.sort(sup, dim=1)
            bad = (srt[:, 1:] == srt[:, :-1]).any(dim=1).nonzero().flatten()
            if bad.numel() == 0:
                break
            sup[bad] = torch.randint(0, K, (bad.numel(), s), generator=g, device=device)
        # Laplace(0, 1) by inversion of a uniform on (-1/2, 1/2)
        u = torch.rand((n, s), generator=g, device=device, dtype=torch.float64) - 0.5
        u = u.clamp(-0.5 + 1e-12, 0.5 - 1e-12)
        coef = (-torch.sign(u) * torch.log1p(-2.0 * u.abs())).to(torch.float32)
        x = torch.einsum("ns,nsd->nd", coef, A[sup])
        x += noise_std * torch.randn((n, D_SH), generator=g, device=device)
        out[lo:lo + n] = x
    return out
