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


def _half(a):
    return np.asarray(a, dtype=np.float32).astype(np.float16).astype(np.float64)


@pytest.mark.parametrize("N,K,s", [(1, 16, 1), (1000, 256, 8), (4099, 1024, 16), (333, 1100, 4), (700, 200, 32)])
def test_compact_decode_matches_oracle_on_rounded_inputs(lib, N, K, s):
    """Compact storage: 8-bit indices for K <= 256 (else 16-bit) and FP16
    coefficients; the dictionary is rounded to FP16 in shared memory.  The
    result equals the oracle's decode of the FP16-rounded dictionary and
    coefficients (FP32 sums), and stays close to the FP32 decode."""
    rng = np.random.default_rng(N + 3 * K)
    D = synth.hidden_dictionary(K, 5).astype(np.float32)
    idx, coef, nnz = _codes(rng, N, K, s)
    dirs = synth.unit_directions(N, 6)
    Dt = torch.from_numpy(D).cuda()
    it = torch.from_numpy(idx.astype(np.int16)).cuda()
    ct = torch.from_numpy(coef).cuda()
    nt = torch.from_numpy(nnz).cuda()
    dt = torch.from_numpy(dirs).cuda()
    idx_c, coef_c = lib.compact_codes(it, ct, K, sync=True)
    assert idx_c.dtype == (torch.uint8 if K <= 256 else torch.int16)
    got_idx = idx_c.cpu().numpy().astype(np.int64) if K <= 256 else lib.idx_as_long(idx_c).cpu().numpy()
    np.testing.assert_array_equal(got_idx, idx.astype(np.int64))
    np.testing.assert_array_equal(coef_c.cpu().numpy(), coef.astype(np.float16))
    rgb = lib.decode_compact(Dt, idx_c, coef_c, nt, dirs=dt, sync=True).cpu().numpy()
    ref = osh.decode(_half(D), idx, _half(coef), nnz, dirs=dirs)
    ok, worst = close_rel(rgb, ref)
    assert ok, worst
    full = osh.decode(D, idx, coef, nnz, dirs=dirs)
    scale = np.abs(full).max() + 1e-6
    assert np.abs(rgb - full).max() <= 5e-3 * scale, np.abs(rgb - full).max() / scale


def test_compact_decode_rejects_bad_sizes(lib):
    from paper_2605_30396_gb300 import _lib as L
    kmax = L.lib().dlsh_decode_compact_max_k(8)
    assert 1200 < kmax < 2000
    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    # 8-bit indices with K > 256, and a dictionary beyond shared memory
    assert L.lib().dlsh_compact_codes(t.data_ptr(), t.data_ptr(), 1, 8, 300, t.data_ptr(), 1, t.data_ptr(),
                                      st, 0) != 0
    assert L.lib().dlsh_decode_compact(t.data_ptr(), kmax + 1, 45, t.data_ptr(), 2, t.data_ptr(), t.data_ptr(),
                                       8, 1, t.data_ptr(), None, None, t.data_ptr(), st, 0) != 0


@pytest.mark.parametrize("compact", [False, True])
def test_decode_full_colour_with_dc(lib, compact):
    """With the DC coefficients the decode returns max(0, Y00 dc + view + 0.5)."""
    N, K, s = 3001, 200, 6
    rng = np.random.default_rng(71)
    D = synth.hidden_dictionary(K, 72).astype(np.float32)
    idx, coef, nnz = _codes(rng, N, K, s)
    dirs = synth.unit_directions(N, 73)
    dc = (2.0 * rng.standard_normal((N, 3))).astype(np.float32)  # some colours clamp at 0
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    if compact:
        idx_c, coef_c = lib.compact_codes(c(idx.astype(np.int16)), c(coef), K, sync=True)
        rgb = lib.decode_compact(c(D), idx_c, coef_c, c(nnz), dirs=c(dirs), dc=c(dc), sync=True).cpu().numpy()
        view = osh.decode(_half(D), idx, _half(coef), nnz, dirs=dirs)
    else:
        rgb = lib.decode(c(D), c(idx.astype(np.int16)), c(coef), c(nnz), dirs=c(dirs), dc=c(dc),
                         sync=True).cpu().numpy()
        view = osh.decode(D, idx, coef, nnz, dirs=dirs)
    ref = osh.full_colour(view, dc.astype(np.float64))
    assert (ref == 0).any() and (ref > 0).any()
    ok, worst = close_rel(rgb, ref)
    assert ok, worst


@pytest.mark.parametrize("K,s,compact", [(1024, 8, False), (2048, 8, False), (1024, 8, True), (200, 4, True)])
def test_decode_autotune_keeps_colours(lib, K, s, compact):
    """The decode's batch size and warps per CTA change how Gaussians are dealt
    to warps, not the arithmetic of one Gaussian: after tuning, the colours are
    bitwise those of the default shape (K = 2048 reads the rows through the
    read-only cache; K = 200 compact uses 8-bit indices)."""
    rng = np.random.default_rng(K + s + int(compact))
    N = 20011
    D = synth.hidden_dictionary(K, 5).astype(np.float32)
    idx, coef, nnz = _codes(rng, N, K, s)
    dirs = synth.unit_directions(N, 6)
    Dt = torch.from_numpy(D).cuda()
    it = torch.from_numpy(idx.astype(np.int16)).cuda()
    ct = torch.from_numpy(coef).cuda()
    nt = torch.from_numpy(nnz).cuda()
    dt = torch.from_numpy(dirs).cuda()
    if compact:
        it, ct = lib.compact_codes(it, ct, K, sync=True)
        run = lambda: lib.decode_compact(Dt, it, ct, nt, dirs=dt, sync=True).cpu().numpy()
    else:
        run = lambda: lib.decode(Dt, it, ct, nt, dirs=dt, sync=True).cpu().numpy()
    before = run()
    gb, nw = lib.autotune_decode(Dt, it, ct, nt, dirs=dt)
    assert gb in (8, 16) and 1 <= nw <= 32
    np.testing.assert_array_equal(run(), before)
    import ctypes
    from paper_2605_30396_gb300 import _lib as L
    b, w = ctypes.c_int(0), ctypes.c_int(0)
    fmt = 0 if not compact else (1 if K <= 256 else 2)
    assert L.lib().dlsh_tuned_decode(fmt, K, s, ctypes.byref(b), ctypes.byref(w)) == 1
    assert (b.value, w.value) == (gb, nw)
