"""Splatting preprocess (project, cull, colour) vs the FP64 oracle, with the
colour read from dense SH, from FP32 codes and from compact codes."""
import numpy as np
import pytest
import torch

from gpu_common import close_rel
from oracle import splat as osp
from paper_2605_30396_gb300 import synth

pytestmark = pytest.mark.gpu

W, H, FX, FY, NEAR = 640, 480, 520.0, 500.0, 0.2
VIEWS = {
    # outside the cloud, looking at it: nearly everything visible
    "outside": ((0.4, -3.2, 1.1), (0.0, 0.0, 0.0)),
    # inside the cloud: most Gaussians behind the camera or off screen, some
    # straddling the near plane
    "inside": ((0.15, -0.1, 0.05), (1.0, 0.4, -0.3)),
}


def _camera(lib, view):
    R, t = synth.look_at(*VIEWS[view])
    R32, t32 = R.astype(np.float32), t.astype(np.float32)
    return lib.camera(R32, t32, FX, FY, W, H, NEAR), R32.astype(np.float64), t32.astype(np.float64)


def _gauss(N, seed):
    return synth.splat_gaussians(N, seed)


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _run(lib, cam, g, **colour):
    means, scales, quats, dc = _dev(*g)
    out = lib.preprocess(cam, means, scales, quats, dc, sync=True, **colour)
    return {k: v.cpu().numpy() for k, v in out.items()}


def _oracle(g, R, t, **colour):
    means, scales, quats, dc = (a.astype(np.float64) for a in g)
    return osp.preprocess(means, scales, quats, R, t, FX, FY, W, H, NEAR, dc, **colour)


def _ambiguous(ref):
    """Gaussians whose visibility or radius the FP32 and FP64 sides may decide
    differently: a deciding quantity within rounding of its threshold."""
    raw = ref["raw"]
    z, px, py, det, ext = raw["z"], raw["px"], raw["py"], raw["det"], raw["extent"]
    rc = np.ceil(ext)
    amb = np.abs(z - NEAR) < 1e-5 * (1 + np.abs(z))
    amb |= raw["front"] & (np.abs(det) < 1e-5)
    amb |= raw["front"] & (np.abs(ext - np.round(ext)) < 1e-4 * (1 + ext))
    for edge in (px + rc, W - (px - rc), py + rc, H - (py - rc)):
        amb |= raw["front"] & (np.abs(edge) < 2e-2 + 1e-5 * np.abs(px))
    return amb


def _compare(out, ref, colour_rel=1e-4):
    amb = _ambiguous(ref)
    vo = ref["radius"] > 0
    vg = out["radius"] > 0
    assert (vo == vg)[~amb].all(), np.flatnonzero((vo != vg) & ~amb)[:10]
    sel = vo & vg & ~amb
    assert (out["radius"][sel] == ref["radius"][sel]).all()
    for k in ("xy", "depth", "conic"):
        ok, worst = close_rel(out[k][sel], ref[k][sel])
        assert ok, (k, worst)
    ok, worst = close_rel(out["rgb"][sel], ref["rgb"][sel], colour_rel)
    assert ok, ("rgb", worst)
    culled = ~vg
    for k in ("xy", "depth", "conic", "rgb"):
        assert (out[k][culled] == 0).all(), k
    return int(vo.sum())


@pytest.mark.parametrize("view", sorted(VIEWS))
@pytest.mark.parametrize("N,offset", [(1, 0), (33, 0), (5003, 0), (5003, 1)])
def test_preprocess_sh(lib, view, N, offset):
    # offset 1 starts the SH rows 4 bytes past a 16-byte boundary (the copy
    # then takes 4-byte granules even for fully visible batches)
    cam, R, t = _camera(lib, view)
    g = _gauss(N, 10 + N)
    y = (0.2 * np.random.default_rng(N).standard_normal((N, 45))).astype(np.float32)
    buf = torch.zeros(N * 45 + offset, device="cuda")
    sh = buf[offset:].view(N, 45)
    sh.copy_(torch.from_numpy(y))
    out = _run(lib, cam, g, sh=sh)
    ref = _oracle(g, R, t, y=y.astype(np.float64))
    _compare(out, ref)


def test_views_cover_culling(lib):
    # the fixtures exercise both visible and culled Gaussians of every kind
    N = 5003
    g = _gauss(N, 10 + N)
    for view, lo, hi in (("outside", 0.9, 1.0), ("inside", 0.02, 0.6)):
        _, R, t = _camera(lib, view)
        ref = _oracle(g, R, t, y=np.zeros((N, 45)))
        frac = (ref["radius"] > 0).mean()
        assert lo <= frac <= hi, (view, frac)
        if view == "inside":
            assert (~ref["raw"]["front"]).sum() > 100  # behind the camera or the near plane
            assert ((ref["radius"] == 0) & ref["raw"]["front"]).sum() > 100  # off screen


@pytest.mark.parametrize("view", sorted(VIEWS))
@pytest.mark.parametrize("N,K,s", [(5003, 300, 8), (2100, 90, 12), (1000, 800, 5), (257, 16, 1),
                                   (300, 64, 32), (700, 33, 3)])
def test_preprocess_codes(lib, view, N, K, s):
    cam, R, t = _camera(lib, view)
    g = _gauss(N, 20 + N)
    D = synth.hidden_dictionary(K, 7).astype(np.float32)
    idx, coef, nnz = synth.random_codes(N, K, s, 30 + N)
    out = _run(lib, cam, g, D=torch.from_numpy(D), idx=torch.from_numpy(idx.astype(np.int16)).cuda(),
               coef=torch.from_numpy(coef).cuda(), nnz=torch.from_numpy(nnz).cuda())
    ref = _oracle(g, R, t, D=D.astype(np.float64), idx=idx.astype(np.int64), coef=coef.astype(np.float64),
                  nnz=nnz)
    _compare(out, ref)


@pytest.mark.parametrize("N,K,s", [(5003, 90, 12), (3001, 256, 8), (2000, 1024, 8), (999, 1500, 16)])
def test_preprocess_compact(lib, N, K, s):
    if K > lib_max_k(lib, s, 1):
        pytest.skip("dictionary larger than the compact shared-memory table")
    cam, R, t = _camera(lib, "outside")
    g = _gauss(N, 40 + N)
    D = synth.hidden_dictionary(K, 8).astype(np.float32)
    idx, coef, nnz = synth.random_codes(N, K, s, 50 + N)
    idx_c = idx.astype(np.uint8) if K <= 256 else idx.astype(np.int16)
    coef_c = coef.astype(np.float16)
    out = _run(lib, cam, g, D=torch.from_numpy(D), idx=torch.from_numpy(idx_c).cuda(),
               coef=torch.from_numpy(coef_c).cuda(), nnz=torch.from_numpy(nnz).cuda())
    # the oracle decodes the FP16-rounded dictionary and coefficients
    D16 = D.astype(np.float16).astype(np.float64)
    ref = _oracle(g, R, t, D=D16, idx=idx.astype(np.int64), coef=coef_c.astype(np.float64), nnz=nnz)
    _compare(out, ref)


def lib_max_k(lib, s, compact):
    from paper_2605_30396_gb300 import _lib
    return int(_lib.lib().dlsh_preprocess_max_k(s, compact))


def test_geometry_identical_across_colour_sources(lib):
    N, K, s = 4000, 200, 8
    cam, _, _ = _camera(lib, "inside")
    g = _gauss(N, 3)
    D = synth.hidden_dictionary(K, 9).astype(np.float32)
    idx, coef, nnz = synth.random_codes(N, K, s, 4)
    a = _run(lib, cam, g, sh=torch.zeros((N, 45), device="cuda"))
    b = _run(lib, cam, g, D=torch.from_numpy(D), idx=torch.from_numpy(idx.astype(np.int16)).cuda(),
             coef=torch.from_numpy(coef).cuda(), nnz=torch.from_numpy(nnz).cuda())
    c = _run(lib, cam, g, D=torch.from_numpy(D), idx=torch.from_numpy(idx.astype(np.uint8)).cuda(),
             coef=torch.from_numpy(coef.astype(np.float16)).cuda(), nnz=torch.from_numpy(nnz).cuda())
    for k in ("xy", "depth", "conic", "radius"):
        np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a[k], c[k])


def test_out_of_range_code_entries_count_as_zero(lib):
    N, K, s = 600, 50, 6
    cam, R, t = _camera(lib, "outside")
    g = _gauss(N, 5)
    D = synth.hidden_dictionary(K, 3).astype(np.float32)
    idx, coef, nnz = synth.random_codes(N, K, s, 6, nnz_min=3)
    rng = np.random.default_rng(7)
    bad_idx = idx.copy()
    hit = rng.random((N, s)) < 0.1
    bad_idx[hit] = K + rng.integers(0, 1000, hit.sum())
    bad_nnz = nnz.copy()
    bad_nnz[::7] = s + 5  # beyond s: clamped to s
    out = _run(lib, cam, g, D=torch.from_numpy(D), idx=torch.from_numpy(bad_idx.astype(np.int16)).cuda(),
               coef=torch.from_numpy(coef).cuda(), nnz=torch.from_numpy(bad_nnz).cuda())
    ref_coef = np.where(hit, 0.0, coef)
    ref_idx = np.where(hit, 0, idx)
    ref = _oracle(g, R, t, D=D.astype(np.float64), idx=ref_idx.astype(np.int64), coef=ref_coef,
                  nnz=np.minimum(bad_nnz, s))
    _compare(out, ref)


def test_empty_and_errors(lib):
    cam, _, _ = _camera(lib, "outside")
    z3 = torch.empty((0, 3), device="cuda")
    z4 = torch.empty((0, 4), device="cuda")
    out = lib.preprocess(cam, z3, z3, z4, z3, sh=torch.empty((0, 45), device="cuda"), sync=True)
    assert out["rgb"].shape == (0, 3)
    N = 64
    means, scales, quats, dc = _dev(*_gauss(N, 1))
    buf = torch.empty(N * 4 + 1, device="cuda")
    misaligned = buf[1:].view(N, 4)
    with pytest.raises(lib.DlshError):
        lib.preprocess(cam, means, scales, misaligned, dc, sh=torch.zeros((N, 45), device="cuda"))
    D = torch.from_numpy(synth.hidden_dictionary(300, 1).astype(np.float32))
    idx = torch.zeros((N, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.DlshError):  # 8-bit indices with K > 256
        lib.preprocess(cam, means, scales, quats, dc, D=D, idx=idx,
                       coef=torch.zeros((N, 4), dtype=torch.float16, device="cuda"),
                       nnz=torch.zeros(N, dtype=torch.uint8, device="cuda"))
    big = torch.zeros((int(lib_max_k(lib, 4, 0)) + 1, 45))
    with pytest.raises(lib.DlshError):  # dictionary larger than shared memory
        lib.preprocess(cam, means, scales, quats, dc, D=big, idx=idx.to(torch.int16),
                       coef=torch.zeros((N, 4), device="cuda"),
                       nnz=torch.zeros(N, dtype=torch.uint8, device="cuda"))
