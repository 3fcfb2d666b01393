"""Step a1 alone: C = R D^T on the tcgen05 path vs the FP64 product."""
import numpy as np
import pytest
import torch

from paper_2605_30396_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,K", [(1, 1), (128, 128), (300, 300), (513, 1024), (200, 2100)])
@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("bf16", 1.2e-2), ("fp8", 0.12)])
def test_correlate_matches_fp64(lib, M, K, prec, tol):
    rng = np.random.default_rng(M * 7 + K)
    D = synth.hidden_dictionary(K, 3).astype(np.float32)
    R = (rng.standard_normal((M, 45)) * rng.uniform(0.01, 3.0, (M, 1))).astype(np.float32)
    C = lib.correlate(torch.from_numpy(D), torch.from_numpy(R), precision=prec).cpu().numpy()
    ref = R.astype(np.float64) @ D.astype(np.float64).T
    scale = np.linalg.norm(R.astype(np.float64), axis=1, keepdims=True)  # |d_j| = 1
    err = np.abs(C - ref) / np.maximum(scale, 1e-30)
    assert err.max() <= tol, (prec, err.max())
