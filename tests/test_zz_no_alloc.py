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


def _largest_fitting_k(L, s, prec):
    """Largest K whose encoder scratch fits the fixed array (host-side sizes only)."""
    cap = L.dlsh_encode_noalloc_max_bytes()
    K = 1024
    while L.dlsh_encode_workspace_size(K + 1, 45, s, prec) <= cap:
        K += 1
    return K


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_at_the_edges_of_its_scratch(lib, prec):
    """K = 1024 with s = 16, and the largest K whose scratch fits, both against
    the workspace encoder; one atom more must be refused before any launch."""
    L = _lib.lib()
    D = torch.from_numpy(synth.hidden_dictionary(1024, 31 + prec).astype(np.float32)).cuda()
    X = torch.from_numpy(synth.signals(3000, synth.hidden_dictionary(1024, 32), 12, 33)).cuda()
    _compare(_noalloc(L, D, X, 16, prec), _with_workspace(L, D, X, 16, prec))
    Kmax = _largest_fitting_k(L, 8, prec)
    assert Kmax >= 1024
    Dm = torch.from_numpy(synth.hidden_dictionary(Kmax, 41 + prec).astype(np.float32)).cuda()
    Xm = torch.from_numpy(synth.signals(1500, synth.hidden_dictionary(Kmax, 42), 8, 43)).cuda()
    _compare(_noalloc(L, Dm, Xm, 8, prec), _with_workspace(L, Dm, Xm, 8, prec))
    Dn = torch.from_numpy(synth.hidden_dictionary(Kmax + 1, 44).astype(np.float32)).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = Xm.shape[0]
    out = (torch.empty((n, 8), dtype=torch.int16, device="cuda"),
           torch.empty((n, 8), dtype=torch.float32, device="cuda"),
           torch.empty((n,), dtype=torch.uint8, device="cuda"),
           torch.empty((n,), dtype=torch.float32, device="cuda"))
    rc = L.dlsh_encode_noalloc(_ptr(Dn), Kmax + 1, 45, _ptr(Xm), n, 8, 0.0, prec,
                               *[_ptr(t) for t in out], stream, 1)
    assert rc == -2 and b"scratch" in L.dlsh_last_error()
