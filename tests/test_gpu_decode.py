"""Step a6: radiance from sparse codes vs the oracle's dense SH evaluation of D alpha."""
import numpy as np
import pytest
import torch

from gpu_common import close_rel
from oracle import sh as osh
from paper_2605_30396_gb300 import synth

pytestmark = pytest.mark.gpu


def _codes(rng, N, K, s, ragged=True):
    idx = synth.distinct_supports(rng, N, K, s)
    coef = rng.laplace(0, 1, (N, s)).astype(np.float32)
    nnz = rng.integers(0, s + 1, N) if ragged else np.full(N, s)
    coef[np.arange(s)[None, :] >= nnz[:, None]] = 0.0
    idx[np.arange(s)[None, :] >= nnz[:, None]] = 0
    return idx, coef, nnz.astype(np.uint8)


@pytest.mark.parametrize("N,K,s", [(1, 16, 1), (1000, 256, 8), (4099, 1024, 16), (777, 2048, 8),
                                   (500, 64, 32), (333, 1100, 4)])
def test_decode_dirs(lib, N, K, s):
    rng = np.random.default_rng(N + K)
    D = synth.hidden_dictionary(K, 5).astype(np.float32)
    idx, coef, nnz = _codes(rng, N, K, s)
    dirs = synth.unit_directions(N, 6)
    rgb = lib.decode(torch.from_numpy(D).cuda(), torch.from_numpy(idx.astype(np.int16)).cuda(),
                     torch.from_numpy(coef).cuda(), torch.from_numpy(nnz).cuda(),
                     dirs=torch.from_numpy(dirs).cuda(), sync=True).cpu().numpy()
    ref = osh.decode(D, idx, coef, nnz, dirs=dirs)
    ok, worst = close_rel(rgb, ref)
    assert ok, worst


def test_decode_camera_and_means(lib):
    N, K, s = 5000, 1024, 8
    rng = np.random.default_rng(1)
    D = synth.hidden_dictionary(K, 2).astype(np.float32)
    idx, coef, nnz = _codes(rng, N, K, s, ragged=False)
    cam, mu = synth.camera_and_means(N, 2, 3)
    rgb = lib.decode(torch.from_numpy(D), torch.from_numpy(idx.astype(np.int16)),
                     torch.from_numpy(coef), torch.from_numpy(nnz), means=torch.from_numpy(mu),
                     cam=cam).numpy()  # host tensors: the end-to-end path
    ref = osh.decode(D, idx, coef, nnz, means=mu, cam=cam)
    ok, worst = close_rel(rgb, ref)
    assert ok, worst


def test_decode_empty(lib):
    D = torch.from_numpy(synth.hidden_dictionary(16, 1).astype(np.float32)).cuda()
    z = torch.empty((0, 4), dtype=torch.float32, device="cuda")
    rgb = lib.decode(D, torch.empty((0, 4), dtype=torch.int16, device="cuda"), z,
                     torch.empty((0,), dtype=torch.uint8, device="cuda"),
                     dirs=torch.empty((0, 3), device="cuda"), sync=True)
    assert rgb.shape == (0, 3)


def test_decode_one_sparse_is_scaled_atom(lib):
    K, N = 32, 64
    D = synth.hidden_dictionary(K, 4).astype(np.float32)
    idx = (np.arange(N) % K).reshape(N, 1)
    coef = np.linspace(-2, 2, N).astype(np.float32).reshape(N, 1)
    dirs = synth.unit_directions(N, 9)
    rgb = lib.decode(torch.from_numpy(D), torch.from_numpy(idx.astype(np.int16)),
                     torch.from_numpy(coef), torch.from_numpy(np.ones(N, np.uint8)),
                     dirs=torch.from_numpy(dirs)).numpy()
    ref = coef * osh.sh_eval(D[idx[:, 0]], dirs)
    ok, worst = close_rel(rgb, ref)
    assert ok, worst
