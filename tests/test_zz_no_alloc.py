"""The allocation-free encoder entry point (dlsh_encode_noalloc).

For callers that cannot allocate device memory (plugins whose host application
owns every device allocation, real-time loops where cudaMalloc is not allowed).
Its scratch is a fixed device array inside the library; this file is collected
last so that a run stopping at the first failure has run every other test first.
It must pass both alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2605_30396_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(L, D, X, s, prec):
    N, K = X.shape[0], D.shape[0]
    idx = torch.full((N, s), -1, dtype=torch.int16, device="cuda")
    coef = torch.full((N, s), float("nan"), dtype=torch.float32, device="cuda")
    nnz = torch.full((N,), 255, dtype=torch.uint8, device="cuda")
    resid = torch.full((N,), float("nan"), dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.dlsh_encode_noalloc(_ptr(D), K, 45, _ptr(X), N, s, 0.0, prec, _ptr(idx), _ptr(coef),
                               _ptr(nnz), _ptr(resid), stream, 1)
    assert rc == 0, L.dlsh_last_error()
    return idx, coef, nnz, resid


def _with_workspace(L, D, X, s, prec):
    N, K = X.shape[0], D.shape[0]
    idx = torch.empty((N, s), dtype=torch.int16, device="cuda")
    coef = torch.empty((N, s), dtype=torch.float32, device="cuda")
    nnz = torch.empty((N,), dtype=torch.uint8, device="cuda")
    resid = torch.empty((N,), dtype=torch.float32, device="cuda")
    need = L.dlsh_encode_workspace_size(K, 45, s, prec)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.dlsh_encode(_ptr(D), K, 45, _ptr(X), N, s, 0.0, prec, _ptr(idx), _ptr(coef), _ptr(nnz),
                       _ptr(resid), _ptr(ws), need, stream, 1)
    assert rc == 0, L.dlsh_last_error()
    return idx, coef, nnz, resid


def _compare(a, b):
    np.testing.assert_array_equal(a[0].cpu().numpy(), b[0].cpu().numpy())
    np.testing.assert_array_equal(a[2].cpu().numpy(), b[2].cpu().numpy())
    # the same kernels run on the same inputs; the encoder tests' coefficient
    # tolerance (1e-3 of the largest coefficient) bounds any difference
    ca, cb = a[1].cpu().numpy(), b[1].cpu().numpy()
    scale = np.abs(cb).max(axis=1, keepdims=True) + 1e-12
    assert (np.abs(ca - cb) / scale).max() <= 1e-3
    np.testing.assert_allclose(a[3].cpu().numpy(), b[3].cpu().numpy(), rtol=1e-4, atol=1e-12)


def test_noalloc_matches_workspace_encoder_twice(lib):
    L = _lib.lib()
    assert L.dlsh_encode_noalloc_max_bytes() == 8 << 20
    # first call: K=1024, FP32, s=8
    D1 = torch.from_numpy(synth.hidden_dictionary(1024, 11).astype(np.float32)).cuda()
    X1 = torch.from_numpy(synth.signals(5000, synth.hidden_dictionary(1024, 12), 8, 13)).cuda()
    _compare(_noalloc(L, D1, X1, 8, 0), _with_workspace(L, D1, X1, 8, 0))
    # second call in a row: another dictionary, size and precision reuse the same scratch
    D2 = torch.from_numpy(synth.hidden_dictionary(300, 21).astype(np.float32)).cuda()
    X2 = torch.from_numpy(synth.signals(2345, synth.hidden_dictionary(300, 22), 4, 23)).cuda()
    _compare(_noalloc(L, D2, X2, 6, 1), _with_workspace(L, D2, X2, 6, 1))


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    L = _lib.lib()
    fake = ctypes.c_void_p(0x1000)
    rc = L.dlsh_encode_noalloc(fake, 2048, 45, fake, 10, 8, 0.0, 0, fake, fake, fake, None, None, 0)
    assert rc == -2
    assert b"scratch" in L.dlsh_last_error()
