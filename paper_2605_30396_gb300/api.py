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

PRECISION = {"fp32": 0, "bf16": 1, "fp8": 2, "bf16_qw": 3, "fp8_qw": 4}
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


def _pd(t):
    """Pointer of a tensor the kernels read or write: it must live on the GPU
    (a host pointer reaching a kernel would fault it)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"expected a CUDA tensor, got one on {t.device}")
    return ctypes.c_void_p(t.data_ptr())


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


ENCODE_VARIANTS = {1: "encode_kernel (one tile per CTA)", 2: "encode_pair_kernel",
                   3: "encode_alt_kernel", 4: "encode_split_kernel (TF32 parts)",
                   5: "encode_split_kernel (FP16 parts)", 6: "encode_split_kernel (FP16 parts, three tiles)",
                   7: "encode_kernel (one tile per CTA, FP16 parts)"}


def encode_variant(K: int, s: int, precision="fp32") -> int:
    """The encoder kernel encode() runs for (K, s, precision) without a tuning
    record (see dlsh_encode_variant); 0 if unsupported."""
    return int(_lib.lib().dlsh_encode_variant(int(K), int(s), _prec(precision)))


def encode_profile(D, X, s: int, eps: float = 0.0, precision="fp32"):
    """encode() plus per-phase SM-cycle counters of the encoder (see dlsh.h)."""
    D = _to_device(D, torch.float32)
    X = _to_device(X, torch.float32)
    N, K = X.shape[0], D.shape[0]
    idx = torch.empty((N, s), dtype=torch.int16, device=X.device)
    coef = torch.empty((N, s), dtype=torch.float32, device=X.device)
    nnz = torch.empty((N,), dtype=torch.uint8, device=X.device)
    resid = torch.empty((N,), dtype=torch.float32, device=X.device)
    cyc = torch.zeros((12,), dtype=torch.int64, device=X.device)
    L = _lib.lib()
    need = L.dlsh_encode_workspace_size(K, D.shape[1], s, _prec(precision))
    ws = workspace(need, key="encode")
    rc = L.dlsh_encode_profile(_p(D), K, D.shape[1], _p(X), N, s, float(eps), _prec(precision),
                               _p(idx), _p(coef), _p(nnz), _p(resid), _p(ws), ws.numel(), _p(cyc),
                               _stream(), FLAG_SYNC)
    _check(rc, "dlsh_encode_profile")
    c = cyc.cpu().tolist()
    variant = c[11]
    if variant == 3:  # two tiles served in turn by all warps (see dlsh.h)
        names = ("sel_wait_mma", "selection", "solver", "solver_wait_staging", "tile_iterations",
                 "unused", "mma_wait_a", "mma_wait_chunk", "mma_wait_tmem", "mma_wait_copy")
    elif variant in (4, 5, 6):  # selection and solver warps (TF32 / FP16 products, 2 or 3 tiles)
        names = ("sel_wait_mma", "selection", "solver", "solver_wait_staging", "jobs",
                 "solver_wait_cand", "mma_wait_a", "mma_wait_chunk", "mma_wait_tmem", "mma_wait_copy",
                 "sel_wait_solver")
    else:
        names = ("wait_mma", "selection", "barrier1", "solver", "barrier2", "iterations",
                 "mma_wait_a", "mma_wait_chunk", "mma_wait_tmem", "tma_wait_stage")
    out = dict(zip(names, c))
    out["variant"] = variant
    return (idx, coef, nnz, resid), out


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


def decode(D, idx, coef, nnz, dirs=None, means=None, cam=None, sync: bool = False, out=None, dc=None):
    """RGB (N, 3) from sparse codes; either dirs, or means + cam.  View-dependent
    part only, or with dc (N, 3) the full colour max(0, Y00 dc + view + 0.5)."""
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
    dcd = _to_device(dc, torch.float32) if dc is not None else None
    rgb = out if out is not None else torch.empty((N, 3), dtype=torch.float32, device=coef.device)
    L = _lib.lib()
    rc = L.dlsh_decode(_p(D), D.shape[0], D.shape[1], _p(idx), _p(coef), _p(nnz), s, N, _p(dm),
                       cam_arr, _p(dcd), _p(rgb), _stream(), FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_decode")
    return rgb.cpu() if host else rgb


def compact_codes(idx, coef, K: int, sync: bool = False):
    """ELL codes -> compact codes: (uint8 indices if K <= 256 else int16, FP16 coefficients)."""
    N, s = coef.shape
    ib = 1 if K <= 256 else 2
    idx_c = torch.empty((N, s), dtype=torch.uint8 if ib == 1 else torch.int16, device=coef.device)
    coef_c = torch.empty((N, s), dtype=torch.float16, device=coef.device)
    rc = _lib.lib().dlsh_compact_codes(_pd(idx.contiguous()), _pd(coef.contiguous()), N, s, K, _p(idx_c), ib,
                                       _p(coef_c), _stream(), FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_compact_codes")
    return idx_c, coef_c


def decode_compact(D, idx_c, coef_c, nnz, dirs=None, means=None, cam=None, sync: bool = False, out=None,
                   dc=None):
    """decode() on compact codes (FP16 coefficients, 8/16-bit indices, FP16 dictionary in shared memory)."""
    D = _dev_f32(D)
    N, s = coef_c.shape
    ib = 1 if idx_c.dtype == torch.uint8 else 2
    if dirs is not None:
        dm = _dev_f32(dirs)
        cam_arr = None
    else:
        dm = _dev_f32(means)
        c = [float(v) for v in (cam.tolist() if hasattr(cam, "tolist") else cam)]
        cam_arr = (ctypes.c_float * 3)(*c)
    rgb = out if out is not None else torch.empty((N, 3), dtype=torch.float32, device=coef_c.device)
    dcd = _dev_f32(dc) if dc is not None else None
    rc = _lib.lib().dlsh_decode_compact(_p(D), D.shape[0], D.shape[1], _pd(idx_c.contiguous()), ib,
                                        _pd(coef_c.contiguous()), _pd(nnz.contiguous()), s, N, _p(dm), cam_arr,
                                        _p(dcd), _p(rgb), _stream(), FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_decode_compact")
    return rgb


def camera(R, t, fx: float, fy: float, width: int, height: int, z_near: float = 0.2) -> "_lib.Camera":
    """A dlsh_camera: world -> camera rotation R (3x3, row-major) and translation t."""
    Rf = [float(v) for v in torch.as_tensor(R, dtype=torch.float64).reshape(9).tolist()]
    tf = [float(v) for v in torch.as_tensor(t, dtype=torch.float64).reshape(3).tolist()]
    return _lib.Camera((ctypes.c_float * 9)(*Rf), (ctypes.c_float * 3)(*tf), fx, fy, int(width), int(height),
                       z_near)


def preprocess(cam, means, scales, quats, dc, sh=None, D=None, idx=None, coef=None, nnz=None,
               sync: bool = False, out=None):
    """Splatting preprocess (project, cull, colour) of N Gaussians on the device.

    Colour from dense SH `sh` (N, 45), or from codes (D, idx, coef, nnz): FP32
    `coef` selects the ELL path, FP16 `coef` the compact path (uint8 or int16
    `idx`).  Returns a dict of xy (N, 2), depth (N,), conic (N, 3), radius (N,)
    int32 and rgb (N, 3); `out` may supply that dict preallocated."""
    # the kernels read and write device memory only: host inputs are copied over
    keep = [_to_device(t, torch.float32) for t in (means, scales, quats, dc)]
    N = keep[0].shape[0]
    dev = keep[0].device
    if out is None:
        out = {"xy": torch.empty((N, 2), dtype=torch.float32, device=dev),
               "depth": torch.empty((N,), dtype=torch.float32, device=dev),
               "conic": torch.empty((N, 3), dtype=torch.float32, device=dev),
               "radius": torch.empty((N,), dtype=torch.int32, device=dev),
               "rgb": torch.empty((N, 3), dtype=torch.float32, device=dev)}
    for k in ("xy", "depth", "conic", "radius", "rgb"):
        if not (out[k].is_cuda and out[k].is_contiguous()):
            raise ValueError(f"preprocess: out[{k!r}] must be a contiguous CUDA tensor")
    g = _lib.Gaussians(*(t.data_ptr() for t in keep), N)
    o = _lib.SplatOut(*(out[k].data_ptr() for k in ("xy", "depth", "conic", "radius", "rgb")))
    flags = FLAG_SYNC if sync else 0
    L = _lib.lib()
    if sh is not None:
        sh = _to_device(sh, torch.float32)
        rc = L.dlsh_preprocess_sh(ctypes.byref(cam), ctypes.byref(g), _p(sh), ctypes.byref(o), _stream(), flags)
        _check(rc, "dlsh_preprocess_sh")
        return out
    D = _dev_f32(D)
    s = coef.shape[1]
    idx, nnz = _to_device(idx), _to_device(nnz)
    coef = _to_device(coef, None if coef.dtype == torch.float16 else torch.float32)
    if coef.dtype == torch.float16:
        ib = 1 if idx.dtype == torch.uint8 else 2
        rc = L.dlsh_preprocess_compact(ctypes.byref(cam), ctypes.byref(g), _p(D), D.shape[0], _p(idx), ib, _p(coef),
                                       _p(nnz), s, ctypes.byref(o), _stream(), flags)
        _check(rc, "dlsh_preprocess_compact")
    else:
        rc = L.dlsh_preprocess_codes(ctypes.byref(cam), ctypes.byref(g), _p(D), D.shape[0], _p(idx), _p(coef),
                                     _p(nnz), s, ctypes.byref(o), _stream(), flags)
        _check(rc, "dlsh_preprocess_codes")
    return out


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
    rc = L.dlsh_mod_update(_p(X), N, D_SH, K, _pd(idx.contiguous()), _pd(coef.contiguous()),
                           _pd(nnz.contiguous()), s, _p(D_old),
                           _pd(resid_sq.contiguous()) if resid_sq is not None else None, _p(D_new),
                           _p(ws), ws.numel(), _stream(), FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_mod_update")
    return D_new


def ksvd_update(X, D_old, idx, coef, nnz, resid_sq=None, sync: bool = False):
    """One approximate K-SVD sweep; returns D_new (K, 45).  `coef` (a contiguous
    FP32 device tensor) is updated in place with the refitted coefficients."""
    X = _dev_f32(X)
    D_old = _dev_f32(D_old)
    N, s = coef.shape
    K = D_old.shape[0]
    if not (coef.is_cuda and coef.dtype == torch.float32 and coef.is_contiguous()):
        raise ValueError("ksvd_update: coef must be a contiguous FP32 CUDA tensor (it is updated in place)")
    D_new = torch.empty_like(D_old)
    L = _lib.lib()
    need = L.dlsh_ksvd_workspace_size(K, D_SH, s, N)
    if need == 0:
        raise DlshError(-2, "dlsh_ksvd_workspace_size")
    ws = workspace(need, key="ksvd")
    idx, nnz = _to_device(idx), _to_device(nnz)
    rc = L.dlsh_ksvd_update(_p(X), N, D_SH, K, _p(idx), _p(coef), _p(nnz), s,
                            _p(D_old), _pd(resid_sq.contiguous()) if resid_sq is not None else None, _p(D_new),
                            _p(ws), ws.numel(), _stream(), FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_ksvd_update")
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
    rc = L.dlsh_csc_from_ell(_pd(idx.contiguous()), _pd(coef.contiguous()), _pd(nnz.contiguous()), N,
                             s, _p(col_ptr), _p(row_idx), _p(val), _p(ws), ws.numel(), _stream(),
                             FLAG_SYNC if sync else 0)
    _check(rc, "dlsh_csc_from_ell")
    total = int(col_ptr[-1].item())
    return col_ptr, row_idx[:total], val[:total]


# ---- learned support proposal --------------------------------------------------
HIDDEN = 256
X_IN = 64


def mlp_num_params(K: int) -> int:
    return int(_lib.lib().dlsh_mlp_num_params(K))


def mlp_pack(params: dict, K: int) -> torch.Tensor:
    """Flattens {W1 (256,45 or 64), b1, W2, b2, W3 (K,256), b3} into the C ABI's
    parameter vector (FP32, W1 zero-padded to 64 input columns)."""
    W1 = torch.as_tensor(params["W1"], dtype=torch.float32)
    if W1.shape[1] < X_IN:
        W1 = torch.nn.functional.pad(W1, (0, X_IN - W1.shape[1]))
    parts = [W1, params["b1"], params["W2"], params["b2"], params["W3"], params["b3"]]
    vec = torch.cat([torch.as_tensor(p, dtype=torch.float32).reshape(-1) for p in parts])
    assert vec.numel() == mlp_num_params(K)
    return vec


def mlp_unpack(vec: torch.Tensor, K: int) -> dict:
    v = vec.detach().to("cpu", torch.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (HIDDEN, X_IN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)),
                        ("b2", (HIDDEN,)), ("W3", (K, HIDDEN)), ("b3", (K,))):
        n = 1
        for d in shape:
            n *= d
        out[name] = v[o:o + n].reshape(shape).numpy()
        o += n
    return out


class MLP:
    """Device-resident support-proposal network (parameters + Adam state)."""

    def __init__(self, K: int, params: dict):
        self.K = K
        L = _lib.lib()
        self.blob = torch.empty(L.dlsh_mlp_size(K), dtype=torch.uint8, device="cuda")
        vec = mlp_pack(params, K).cuda()
        _check(L.dlsh_mlp_init(_p(self.blob), K, _p(vec), _stream(), FLAG_SYNC), "dlsh_mlp_init")
        self.step = 0

    def params(self) -> torch.Tensor:
        out = torch.empty(mlp_num_params(self.K), dtype=torch.float32, device="cuda")
        _check(_lib.lib().dlsh_mlp_params(_p(self.blob), self.K, _p(out), _stream(), FLAG_SYNC),
               "dlsh_mlp_params")
        return out

    def _ws(self, B):
        return workspace(_lib.lib().dlsh_mlp_workspace_size(self.K, B), key="mlp")

    def forward(self, X):
        X = _dev_f32(X)
        B = X.shape[0]
        out = torch.empty((B, self.K), dtype=torch.float32, device="cuda")
        ws = self._ws(B)
        _check(_lib.lib().dlsh_mlp_forward(_p(self.blob), self.K, _p(X), B, _p(out), _p(ws),
                                           ws.numel(), _stream(), FLAG_SYNC), "dlsh_mlp_forward")
        return out

    def gradients(self, X, idx, nnz):
        X = _dev_f32(X)
        B, s = idx.shape
        g = torch.empty(mlp_num_params(self.K), dtype=torch.float32, device="cuda")
        loss = torch.empty((1,), dtype=torch.float32, device="cuda")
        ws = self._ws(B)
        _check(_lib.lib().dlsh_mlp_gradients(_p(self.blob), self.K, _p(X), B, _pd(idx.contiguous()),
                                             _pd(nnz.contiguous()), s, _p(g), _p(loss), _p(ws),
                                             ws.numel(), _stream(), FLAG_SYNC), "dlsh_mlp_gradients")
        return g, float(loss.item())

    def train_step(self, X, idx, nnz, lr: float):
        X = _dev_f32(X)
        B, s = idx.shape
        self.step += 1
        loss = torch.empty((1,), dtype=torch.float32, device="cuda")
        ws = self._ws(B)
        _check(_lib.lib().dlsh_mlp_train_step(_p(self.blob), self.K, _p(X), B, _pd(idx.contiguous()),
                                              _pd(nnz.contiguous()), s, float(lr), self.step,
                                              _p(loss), _p(ws), ws.numel(), _stream(), FLAG_SYNC),
               "dlsh_mlp_train_step")
        return float(loss.item())

    def train(self, X, idx, nnz, epochs: int, batch: int, lr: float, sync: bool = True):
        X = _dev_f32(X)
        N, s = idx.shape
        steps = (N // batch) * epochs
        losses = torch.empty((max(steps, 1),), dtype=torch.float32, device="cuda")
        ws = self._ws(batch)
        _check(_lib.lib().dlsh_mlp_train(_p(self.blob), self.K, _p(X), N, _pd(idx.contiguous()),
                                         _pd(nnz.contiguous()), s, epochs, batch, float(lr),
                                         _p(losses), _p(ws), ws.numel(), _stream(),
                                         FLAG_SYNC if sync else 0), "dlsh_mlp_train")
        self.step += steps
        return losses[:steps]

    def propose(self, X, m: int):
        X = _dev_f32(X)
        N = X.shape[0]
        cand = torch.empty((N, m), dtype=torch.int16, device="cuda")
        ws = workspace(_lib.lib().dlsh_mlp_propose_workspace_size(self.K, N), key="propose")
        _check(_lib.lib().dlsh_mlp_propose(_p(self.blob), self.K, _p(X), N, m, _p(cand), _p(ws),
                                           ws.numel(), _stream(), FLAG_SYNC), "dlsh_mlp_propose")
        return cand


def encode_restricted(D, X, cand, s: int, eps: float = 0.0, sync: bool = True):
    D = _dev_f32(D)
    X = _dev_f32(X)
    N, m = cand.shape
    K = D.shape[0]
    idx = torch.empty((N, s), dtype=torch.int16, device="cuda")
    coef = torch.empty((N, s), dtype=torch.float32, device="cuda")
    nnz = torch.empty((N,), dtype=torch.uint8, device="cuda")
    resid = torch.empty((N,), dtype=torch.float32, device="cuda")
    L = _lib.lib()
    ws = workspace(L.dlsh_encode_workspace_size(K, D_SH, s, 0), key="encode")
    _check(L.dlsh_encode_restricted(_p(D), K, D_SH, _p(X), N, _pd(cand.contiguous()), m, s,
                                    float(eps), _p(idx), _p(coef), _p(nnz), _p(resid), _p(ws),
                                    ws.numel(), _stream(), FLAG_SYNC if sync else 0),
           "dlsh_encode_restricted")
    return idx, coef, nnz, resid


def encode_learned(D, X, s: int, mlp: "MLP", mode: str = "deploy", tau: float = 0.0,
                   eps: float = 0.0, fallback_precision="fp32", sync: bool = False, out=None,
                   m: int = 0):
    """Learned proposal (m candidates, 0 = 2s) + restricted OMP + plain-OMP
    fallback.  Returns (idx, coef, nnz, resid_sq, n_fallback_tensor)."""
    host = not X.is_cuda
    D = _to_device(D, torch.float32)
    X = _to_device(X, torch.float32)
    N, K = X.shape[0], D.shape[0]
    if out is None:
        idx = torch.empty((N, s), dtype=torch.int16, device="cuda")
        coef = torch.empty((N, s), dtype=torch.float32, device="cuda")
        nnz = torch.empty((N,), dtype=torch.uint8, device="cuda")
        resid = torch.empty((N,), dtype=torch.float32, device="cuda")
    else:
        idx, coef, nnz, resid = out
    nfb = torch.zeros((1,), dtype=torch.int64, device="cuda")
    L = _lib.lib()
    need = L.dlsh_encode_learned_workspace_size(K, D_SH, s, N, int(m))
    if need == 0:
        raise DlshError(-2, "dlsh_encode_learned_workspace_size")
    ws = workspace(need, key="learned")
    _check(L.dlsh_encode_learned(_p(D), K, D_SH, _p(X), N, s, float(eps), _p(mlp.blob), int(m),
                                 0 if mode == "exact" else 1, float(tau), _prec(fallback_precision),
                                 _p(idx), _p(coef), _p(nnz), _p(resid), _p(nfb), _p(ws), ws.numel(),
                                 _stream(), FLAG_SYNC if sync else 0), "dlsh_encode_learned")
    if host:
        return tuple(t.to("cpu") for t in (idx, coef, nnz, resid, nfb))
    return idx, coef, nnz, resid, nfb


def calibrate_fallback(resid_learned, resid_plain, max_ratio: float = 1.01) -> float:
    tau = ctypes.c_float(0.0)
    _check(_lib.lib().dlsh_calibrate_fallback(_pd(resid_learned.contiguous()),
                                              _pd(resid_plain.contiguous()), resid_learned.numel(),
                                              float(max_ratio), ctypes.byref(tau), _stream()),
           "dlsh_calibrate_fallback")
    return float(tau.value)


# ---- many scenes in one call, autotuner ------------------------------------------
def encode_multi(scenes, precision="fp32", bn: int = 0, sync: bool = False):
    """scenes: list of dicts {D (K,45), X (N,45), s, eps=0}.  Returns a list of
    (idx, coef, nnz, resid_sq) per scene; the scenes are encoded concurrently on
    streams forked from the current one (graph-capturable)."""
    outs, keep, arr = [], [], (_lib.Scene * len(scenes))()
    for i, sc in enumerate(scenes):
        D = _dev_f32(sc["D"])
        X = _dev_f32(sc["X"])
        s = int(sc["s"])
        N = X.shape[0]
        o = (torch.empty((N, s), dtype=torch.int16, device="cuda"),
             torch.empty((N, s), dtype=torch.float32, device="cuda"),
             torch.empty((N,), dtype=torch.uint8, device="cuda"),
             torch.empty((N,), dtype=torch.float32, device="cuda"))
        keep += [D, X]
        outs.append(o)
        arr[i] = _lib.Scene(D.data_ptr(), D.shape[0], X.data_ptr(), N, s, float(sc.get("eps", 0.0)),
                            o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr(), o[3].data_ptr())
    L = _lib.lib()
    need = L.dlsh_encode_multi_workspace_size(ctypes.byref(arr), len(scenes), _prec(precision), bn)
    if need == 0:
        raise DlshError(-2, "dlsh_encode_multi_workspace_size")
    ws = workspace(need, key="multi")
    _check(L.dlsh_encode_multi(ctypes.byref(arr), len(scenes), _prec(precision), bn, _p(ws),
                               ws.numel(), _stream(), FLAG_SYNC if sync else 0), "dlsh_encode_multi")
    if not sync:
        _KEEPALIVE.append(keep)
    return outs


_KEEPALIVE = []


def autotune_encode(D, X, s: int, precision="fp32") -> int:
    """Times every encoder kernel whose plan fits on this sample, then shallower
    dictionary rings for the fastest; returns the winner as dlsh_autotune_encode
    codes it (kernel variant + 256 x ring-stage cap).  Later encodes of the same
    K, s, precision use it."""
    D = _dev_f32(D)
    X = _dev_f32(X)
    N, K = X.shape[0], D.shape[0]
    idx = torch.empty((N, s), dtype=torch.int16, device="cuda")
    coef = torch.empty((N, s), dtype=torch.float32, device="cuda")
    nnz = torch.empty((N,), dtype=torch.uint8, device="cuda")
    resid = torch.empty((N,), dtype=torch.float32, device="cuda")
    L = _lib.lib()
    ws = workspace(L.dlsh_encode_workspace_size(K, D_SH, s, _prec(precision)), key="encode")
    best = ctypes.c_int(0)
    _check(L.dlsh_autotune_encode(_p(D), K, D_SH, _p(X), N, s, _prec(precision), _p(idx), _p(coef),
                                  _p(nnz), _p(resid), _p(ws), ws.numel(), _stream(),
                                  ctypes.byref(best)), "dlsh_autotune_encode")
    return int(best.value)


def autotune_decode(D, idx, coef, nnz, dirs=None, means=None, cam=None):
    """Times the decode of these codes at batches of 8 and 16 Gaussians per warp
    and several warp counts per CTA; records the fastest for the codes' format
    (FP32 coef: dlsh_decode; FP16 coef: compact codes), K and s, and returns it
    as (batch, warps).  Later decodes of that shape use it."""
    D = _dev_f32(D)
    N, s = coef.shape
    if coef.dtype == torch.float16:
        fmt = 1 if idx.dtype == torch.uint8 else 2
        coef = coef.contiguous()
    else:
        fmt = 0
        coef = _dev_f32(coef)
    idx = idx.contiguous()
    nnz = nnz.contiguous()
    if dirs is not None:
        dm, cam_arr = _dev_f32(dirs), None
    else:
        dm = _dev_f32(means)
        c = [float(v) for v in (cam.tolist() if hasattr(cam, "tolist") else cam)]
        cam_arr = (ctypes.c_float * 3)(*c)
    rgb = torch.empty((N, 3), dtype=torch.float32, device=coef.device)
    gb, nw = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib.lib().dlsh_autotune_decode(_p(D), D.shape[0], D.shape[1], _pd(idx), _pd(coef), fmt, _pd(nnz), s,
                                           N, _p(dm), cam_arr, _p(rgb), _stream(), ctypes.byref(gb),
                                           ctypes.byref(nw)), "dlsh_autotune_decode")
    return int(gb.value), int(nw.value)
