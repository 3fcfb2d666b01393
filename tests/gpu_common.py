"""Shared inputs and tolerances for the GPU parity tests."""
import numpy as np

# Element tolerance of the spec reading: |g - o| <= 1e-4 (|o| + rms(o)).
REL = 1e-4


def close_rel(got, ref, rel=REL):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    rms = np.sqrt(np.mean(ref * ref)) if ref.size else 0.0
    err = np.abs(got - ref)
    bound = rel * (np.abs(ref) + rms)
    return bool((err <= bound).all()), float((err / np.maximum(bound, 1e-300)).max() if ref.size else 0)


def embed45(atoms):
    """Pad atoms of dimension n < 45 with zeros to length 45 (norms unchanged)."""
    K, n = atoms.shape
    out = np.zeros((K, 45))
    out[:, :n] = atoms
    return out


def well_separated(topc, nnz, margin):
    """Signals whose every oracle selection step had (|c|_1 - |c|_2)/||r|| > margin."""
    gaps = topc[:, :, 0] - topc[:, :, 1]
    s = topc.shape[1]
    steps = np.arange(s)[None, :] < np.asarray(nnz)[:, None]
    ok = np.where(steps, gaps > margin, True)
    return ok.all(axis=1)
