"""Python binding of the dlsh C ABI (argument marshalling only).

Tensors are torch tensors; every computation runs in libdlsh.so's CUDA kernels on
the current CUDA stream.  Device tensors in give device tensors out.  For the
encoder and decoder, host (CPU) tensors are also accepted: they are copied to the
device (pinned, asynchronous), processed, and the results copied back — the
end-to-end path a user with host data takes.

Layouts follow include/dlsh.h: D (K, 45) rows are atoms, X (N, 45), codes in
padded ELL: idx (N, s) stored as int16 bits of uint16 atom indices (use
`idx_as_long`), coef (N, s) float32, nnz (N,) uint8.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

PRECISION = {"fp32": 0, "bf16": 1, "fp8": 2}
FLAG_SYNC = 1
D_SH = 45


class DlshError(RuntimeError):
    def __init__(self, code: int, call: str):
        self.code = code
        super().__init__(f"{call} failed with status {code}: {_lib.last_error()}")


def _check(rc: int, call: str):
    if rc != 0:
        raise DlshError(rc, call)


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _prec(p) -> int:
    return PRECISION[p] if isinstance(p, str) else int(p)


_WS = {}


def workspace(nbytes: int, device=None, key: str = "default") -> torch.Tensor:
    """A cached uint8 device buffer of at least nbytes (256-byte aligned)."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    k = (key, dev.index)
    buf = _WS.get(k)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        _WS[k] = buf
    return buf


def idx_as_long(idx: torch.Tensor) -> torch.Tensor:
    """uint16 atom indices (held in an int16 tensor) as int64."""
    return idx.to(torch.int32).bitwise_and_(0xFFFF).to(torch.int64)


def _dev_f32(t):
    return t.to(device="cuda", dtype=torch.float32).contiguous()


def _to_device(t, dtype=None):
    if t.is_cuda:
        return t.contiguous() if dtype is None else t.to(dtype).contiguous()
    t = t.contiguous() if dtype is None else t.to(dtype).contiguous()
    if not t.is_pinned():
        t = t.pin_memory()
    return t.to("cuda", non_blocking=True)


def encode_workspace_size(K: int, s: int, precision="fp32") -> int:
    return int(_lib.lib().dlsh_encode_workspace_size(K, D_SH, s, _prec(precision)))


def encode(D, X, s: int, eps: float = 0.0, precision="fp32", sync: bool = False, out=None):
    """OMP sparse codes of X against D.  Returns (idx, coef, nnz, resid_sq)."""
    host = not X.is_cuda
    D = _to_device(D, torch.float32)
    X = _to_device(X, torch.float32)
    N, K = X.shape[0], D.shape[0]
    if out is None:
        idx = torch.empty((N, s), dtype=torch.int16, device=X.device)
        coef = torch.empty((N, s), dtype=torch.float32, device=X.device)
        nnz = torch.empty((N,), dtype=torch.uint8, device=X.device)
        resid = torch.empty((N,), dtype=torch.float32, device=X.device)
    else:
        idx, coef, nnz, resid = out
    L = _lib.lib()
    need = L.dlsh_encode_workspace_size(K, D.shape[1], s, _prec(precision))
    if need == 0:
        raise DlshError(-2, "dlsh_encode_workspace_size")
    ws = workspace(need, key="encode")
    rc = L.dlsh_encode(_p(D), K, D.shape[1], _p(X), N, s, float(eps), _prec(precision), _p(idx),
                       _p(coef), _p(nnz), _p(resid), _p(ws), ws.numel(), _stream(),
                       FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_encode")
    if host:
        return tuple(t.to("cpu", non_blocking=False) for t in (idx, coef, nnz, resid))
    return idx, coef, nnz, resid


def correlate(D, R, precision="fp32", sync: bool = True):
    """C = R D^T on the encoder's tensor-core path."""
    D = _dev_f32(D)
    R = _dev_f32(R)
    M, K = R.shape[0], D.shape[0]
    C = torch.empty((M, K), dtype=torch.float32, device=R.device)
    L = _lib.lib()
    need = L.dlsh_encode_workspace_size(K, D.shape[1], 1, _prec(precision))
    ws = workspace(need, key="correlate")
    rc = L.dlsh_correlate(_p(D), K, D.shape[1], _p(R), M, _prec(precision), _p(C), _p(ws),
                          ws.numel(), _stream(), FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_correlate")
    return C


def decode(D, idx, coef, nnz, dirs=None, means=None, cam=None, sync: bool = False, out=None):
    """View-dependent RGB (N, 3) from sparse codes; either dirs, or means + cam."""
    host = not coef.is_cuda
    D = _to_device(D, torch.float32)
    idx = _to_device(idx)
    coef = _to_device(coef, torch.float32)
    nnz = _to_device(nnz)
    N, s = coef.shape
    if dirs is not None:
        dm = _to_device(dirs, torch.float32)
        cam_arr = None
    else:
        dm = _to_device(means, torch.float32)
        c = [float(v) for v in (cam.tolist() if hasattr(cam, "tolist") else cam)]
        cam_arr = (ctypes.c_float * 3)(*c)
    rgb = out if out is not None else torch.empty((N, 3), dtype=torch.float32, device=coef.device)
    L = _lib.lib()
    rc = L.dlsh_decode(_p(D), D.shape[0], D.shape[1], _p(idx), _p(coef), _p(nnz), s, N, _p(dm),
                       cam_arr, _p(rgb), _stream(), FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_decode")
    return rgb.cpu() if host else rgb


def mod_update(X, D_old, idx, coef, nnz, resid_sq=None, sync: bool = False):
    """One MOD dictionary update; returns D_new (K, 45)."""
    X = _dev_f32(X)
    D_old = _dev_f32(D_old)
    N, s = coef.shape
    K = D_old.shape[0]
    D_new = torch.empty_like(D_old)
    L = _lib.lib()
    need = L.dlsh_mod_workspace_size(K, D_SH, s, N)
    if need == 0:
        raise DlshError(-2, "dlsh_mod_workspace_size")
    ws = workspace(need, key="mod")
    rc = L.dlsh_mod_update(_p(X), N, D_SH, K, _p(idx.contiguous()), _p(coef.contiguous()),
                           _p(nnz.contiguous()), s, _p(D_old),
                           _p(resid_sq.contiguous()) if resid_sq is not None else None, _p(D_new),
                           _p(ws), ws.numel(), _stream(), FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_mod_update")
    return D_new


def init_dictionary(X, init_idx, sync: bool = False):
    """D_0 = normalised rows of X at init_idx (the learning loop's first step)."""
    X = _dev_f32(X)
    init = torch.as_tensor(init_idx, dtype=torch.int64).to("cuda").contiguous()
    K = init.numel()
    D = torch.empty((K, D_SH), dtype=torch.float32, device=X.device)
    rc = _lib.lib().dlsh_init_dictionary(_p(X), X.shape[0], D_SH, _p(init), K, _p(D), _stream(),
                                         FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_init_dictionary")
    return D


def learn_dictionary(X, K: int, s: int, iters: int, init_idx, eps: float = 0.0,
                     precision="fp32", sync: bool = False):
    """Alternating OMP / MOD learning (graph-captured).  Returns
    (D, idx, coef, nnz, rmse[iters+1])."""
    X = _dev_f32(X)
    N = X.shape[0]
    init = torch.as_tensor(init_idx, dtype=torch.int64).to("cuda").contiguous()
    D = torch.empty((K, D_SH), dtype=torch.float32, device=X.device)
    idx = torch.empty((N, s), dtype=torch.int16, device=X.device)
    coef = torch.empty((N, s), dtype=torch.float32, device=X.device)
    nnz = torch.empty((N,), dtype=torch.uint8, device=X.device)
    rmse = torch.empty((iters + 1,), dtype=torch.float32, device=X.device)
    L = _lib.lib()
    need = L.dlsh_learn_workspace_size(K, D_SH, s, N, _prec(precision))
    if need == 0:
        raise DlshError(-2, "dlsh_learn_workspace_size")
    ws = workspace(need, key="learn")
    rc = L.dlsh_learn_dictionary(_p(X), N, D_SH, K, s, float(eps), iters, _p(init),
                                 _prec(precision), _p(D), _p(idx), _p(coef), _p(nnz), _p(rmse),
                                 _p(ws), ws.numel(), _stream(), FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_learn_dictionary")
    return D, idx, coef, nnz, rmse


def csc_from_ell(idx, coef, nnz, sync: bool = False):
    """The paper's CSC storage: (col_ptr (N+1,), row_idx (nnz,), val (nnz,))."""
    N, s = coef.shape
    col_ptr = torch.empty((N + 1,), dtype=torch.int64, device=coef.device)
    row_idx = torch.empty((max(N * s, 1),), dtype=torch.int16, device=coef.device)
    val = torch.empty((max(N * s, 1),), dtype=torch.float32, device=coef.device)
    L = _lib.lib()
    need = L.dlsh_csc_workspace_size(N)
    ws = workspace(need, key="csc")
    rc = L.dlsh_csc_from_ell(_p(idx.contiguous()), _p(coef.contiguous()), _p(nnz.contiguous()), N,
                             s, _p(col_ptr), _p(row_idx), _p(val), _p(ws), ws.numel(), _stream(),
                             FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_csc_from_ell")
    total = int(col_ptr[-1].item())
    return col_ptr, row_idx[:total], val[:total]
