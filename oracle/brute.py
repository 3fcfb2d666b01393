"""Best s-subset by exhaustive enumeration (FP64; tiny inputs only).

The sparse-coding half of Eq. 1 is min ||x - D alpha||^2 s.t. ||alpha||_0 <= s.
For tiny K this is solved exactly by trying every support of size s and solving
least squares on it; OMP (a greedy method) can never do better.  Used only to pin
`omp` on d <= 8 cases.
"""
from __future__ import annotations

import itertools

import numpy as np


def best_subset(D, x, s: int):
    """Returns (support tuple, coefficients, residual norm) of the best s-subset."""
    D = np.asarray(D, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    best = (None, None, np.inf)
    for sup in itertools.combinations(range(D.shape[0]), s):
        A = D[list(sup)].T
        g, *_ = np.linalg.lstsq(A, x, rcond=None)
        r = float(np.linalg.norm(x - A @ g))
        if r < best[2]:
            best = (sup, g, r)
    return best
