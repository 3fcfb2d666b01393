"""CPU-side checks of the C ABI: the library builds, loads, exports every symbol
the header declares, and rejects bad arguments on the host before any launch."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    from paper_2605_30396_gb300 import _lib
    return _lib.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "dlsh.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dlsh_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n


def test_binding_covers_header(L):
    from paper_2605_30396_gb300 import _lib
    assert set(_declared()) <= set(_lib.SIGNATURES)


def test_workspace_queries_and_limits(L):
    assert L.dlsh_encode_workspace_size(1024, 45, 8, 0) > 0
    assert L.dlsh_encode_workspace_size(1024, 44, 8, 0) == 0
    assert L.dlsh_encode_workspace_size(70000, 45, 8, 0) == 0
    assert L.dlsh_encode_workspace_size(1024, 45, 17, 1) == 0
    assert L.dlsh_mod_workspace_size(1024, 45, 8, 1000) > 0
    assert L.dlsh_learn_workspace_size(256, 45, 8, 10000, 0) > 0
    assert L.dlsh_csc_workspace_size(10) > 0


def test_host_side_argument_errors(L):
    P = ctypes.c_void_p
    fake = P(0x1000)
    # d != 45
    rc = L.dlsh_encode(fake, 16, 44, fake, 10, 4, 0.0, 0, fake, fake, fake, None, fake, 1 << 20, None, 0)
    assert rc == -2 and b"d must be 45" in L.dlsh_last_error()
    # NULL D
    rc = L.dlsh_encode(None, 16, 45, fake, 10, 4, 0.0, 0, fake, fake, fake, None, fake, 1 << 20, None, 0)
    assert rc == -1
    # s out of range
    rc = L.dlsh_encode(fake, 16, 45, fake, 10, 40, 0.0, 0, fake, fake, fake, None, fake, 1 << 20, None, 0)
    assert rc == -2
    # workspace too small / missing / misaligned
    rc = L.dlsh_encode(fake, 16, 45, fake, 10, 4, 0.0, 0, fake, fake, fake, None, fake, 16, None, 0)
    assert rc == -5
    rc = L.dlsh_encode(fake, 16, 45, fake, 10, 4, 0.0, 0, fake, fake, fake, None, None, 1 << 20, None, 0)
    assert rc == -5
    rc = L.dlsh_encode(fake, 16, 45, fake, 10, 4, 0.0, 0, fake, fake, fake, None, P(0x1001), 1 << 20, None, 0)
    assert rc == -1
    # negative eps, unknown precision
    rc = L.dlsh_encode(fake, 16, 45, fake, 10, 4, -1.0, 0, fake, fake, fake, None, fake, 1 << 20, None, 0)
    assert rc == -1
    rc = L.dlsh_encode(fake, 16, 45, fake, 10, 4, 0.0, 7, fake, fake, fake, None, fake, 1 << 20, None, 0)
    assert rc == -1
    # decode
    rc = L.dlsh_decode(fake, 16, 45, fake, fake, fake, 33, 10, fake, None, None, fake, None, 0)
    assert rc == -2
    rc = L.dlsh_decode(fake, 16, 45, None, fake, fake, 4, 10, fake, None, None, fake, None, 0)
    assert rc == -1
    # mod
    rc = L.dlsh_mod_update(fake, 10, 45, 5000, fake, fake, fake, 4, fake, None, fake, fake, 1 << 30, None, 0)
    assert rc == -2
    # learn: N < K
    rc = L.dlsh_learn_dictionary(fake, 10, 45, 64, 4, 0.0, 2, fake, 0, fake, fake, fake, fake, fake, fake, 1 << 30, None, 0)
    assert rc == -1
    # csc
    rc = L.dlsh_csc_from_ell(fake, fake, fake, 10, 0, fake, fake, fake, fake, 1 << 20, None, 0)
    assert rc == -1


def test_host_side_errors_of_the_later_entries(L):
    """K-SVD, the splatting preprocess and compact decode reject bad arguments on
    the host, before any launch."""
    from paper_2605_30396_gb300 import _lib
    P = ctypes.c_void_p
    fake = P(0x1000)
    # K-SVD: d, K, aliasing D_new with D_old, misaligned indices, small workspace
    assert L.dlsh_ksvd_workspace_size(64, 45, 4, 1000) > 0
    assert L.dlsh_ksvd_workspace_size(64, 45, 33, 1000) == 0
    rc = L.dlsh_ksvd_update(fake, 10, 44, 8, fake, fake, fake, 4, fake, None, P(0x2000), fake, 1 << 30, None, 0)
    assert rc == -2
    rc = L.dlsh_ksvd_update(fake, 10, 45, 5000, fake, fake, fake, 4, fake, None, P(0x2000), fake, 1 << 30, None, 0)
    assert rc == -2
    rc = L.dlsh_ksvd_update(fake, 10, 45, 8, fake, fake, fake, 4, fake, None, fake, fake, 1 << 30, None, 0)
    assert rc == -1 and b"alias" in L.dlsh_last_error()
    rc = L.dlsh_ksvd_update(fake, 10, 45, 8, P(0x1002), fake, fake, 4, fake, None, P(0x2000), fake, 1 << 30,
                            None, 0)
    assert rc == -1
    rc = L.dlsh_ksvd_update(fake, 10, 45, 8, fake, fake, fake, 4, fake, None, P(0x2000), fake, 16, None, 0)
    assert rc == -5
    # preprocess: missing structs, bad camera, misaligned rotations, dictionary too large
    assert L.dlsh_preprocess_max_k(0, 0) == 0 and L.dlsh_preprocess_max_k(33, 1) == 0
    assert 600 < L.dlsh_preprocess_max_k(8, 0) < L.dlsh_preprocess_max_k(8, 1) < 2000
    cam = _lib.Camera((ctypes.c_float * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1), (ctypes.c_float * 3)(0, 0, 0),
                      100.0, 100.0, 64, 48, 0.1)
    g = _lib.Gaussians(0x1000, 0x1000, 0x1000, 0x1000, 10)
    o = _lib.SplatOut(0x1000, 0x1000, 0x1000, 0x1000, 0x1000)
    br = ctypes.byref
    assert L.dlsh_preprocess_sh(None, br(g), fake, br(o), None, 0) == -1
    assert L.dlsh_preprocess_sh(br(cam), br(g), None, br(o), None, 0) == -1
    bad_cam = _lib.Camera(cam.R, cam.t, 0.0, 100.0, 64, 48, 0.1)
    assert L.dlsh_preprocess_sh(br(bad_cam), br(g), fake, br(o), None, 0) == -1
    g_mis = _lib.Gaussians(0x1000, 0x1000, 0x1004, 0x1000, 10)
    assert L.dlsh_preprocess_sh(br(cam), br(g_mis), fake, br(o), None, 0) == -1
    big = int(L.dlsh_preprocess_max_k(8, 1)) + 1
    assert L.dlsh_preprocess_compact(br(cam), br(g), fake, big, fake, 2, fake, fake, 8, br(o), None, 0) == -2
    assert L.dlsh_preprocess_compact(br(cam), br(g), fake, 300, fake, 1, fake, fake, 8, br(o), None, 0) == -2
    assert L.dlsh_preprocess_codes(br(cam), br(g), fake, 16, fake, fake, fake, 40, br(o), None, 0) == -2
    # compact decode: 8-bit indices need K <= 256
    rc = L.dlsh_decode_compact(fake, 300, 45, fake, 1, fake, fake, 8, 10, fake, None, None, fake, None, 0)
    assert rc == -2


def test_autotuner_and_ring_cap_argument_errors(L):
    """The decode autotuner and the multi-scene call's kernel / ring-cap code
    reject bad arguments on the host, before any GPU work."""
    from paper_2605_30396_gb300 import _lib
    P = ctypes.c_void_p
    fake = P(0x1000)
    A = L.dlsh_autotune_decode
    assert A(fake, 16, 44, fake, fake, 0, fake, 8, 10, fake, None, fake, None, None, None) == -2
    assert A(fake, 16, 45, fake, fake, 3, fake, 8, 10, fake, None, fake, None, None, None) == -1
    assert A(fake, 16, 45, fake, fake, 0, fake, 8, 0, fake, None, fake, None, None, None) == -1
    assert A(fake, 16, 45, fake, fake, 0, fake, 40, 10, fake, None, fake, None, None, None) == -2
    assert A(fake, 300, 45, fake, fake, 1, fake, 8, 10, fake, None, fake, None, None, None) == -2
    assert A(fake, 16, 45, None, fake, 0, fake, 8, 10, fake, None, fake, None, None, None) == -1
    sc = (_lib.Scene * 1)()
    sc[0] = _lib.Scene(0x1000, 1024, 0x1000, 100, 8, 0.0, 0x1000, 0x1000, 0x1000, 0)
    W = L.dlsh_encode_multi_workspace_size
    assert W(ctypes.byref(sc), 1, 0, 0) > 0
    assert W(ctypes.byref(sc), 1, 0, 5 + 256 * 2) > 0
    assert W(ctypes.byref(sc), 1, 0, 2 * 256) > 0
    for bad in (1, 8, 65, 5 + 256, 5 + 256 * 33, -5):
        assert W(ctypes.byref(sc), 1, 0, bad) == 0, bad
    rc = L.dlsh_encode_multi(ctypes.byref(sc), 1, 0, 5 + 256, fake, 1 << 30, None, 0)
    assert rc == -1 and b"ring cap" in L.dlsh_last_error()


def test_tuning_table_read_from_the_cache_file(tmp_path):
    """The autotuners' table as DLSH_AUTOTUNE_CACHE keeps it: JSON lines keyed by
    configuration (and the older encoder-only lines), read back at first use.
    Runs in a child process so that the file is the table's first source."""
    import subprocess
    import sys
    cache = tmp_path / "tune.jsonl"
    cache.write_text('{"key": "encode K=1024 s=8 p=0", "values": [6, 2]}\n'
                     '{"K": 512, "s": 4, "precision": 1, "bn": 2}\n'
                     '{"key": "decode f=0 K=1024 s=8", "values": [16, 14]}\n'
                     '{"key": "decode f=3 K=700 s=4", "values": [8, 21]}\n'
                     'not a record\n')
    code = (
        "import ctypes, sys\n"
        "sys.path.insert(0, %r)\n"
        "from paper_2605_30396_gb300 import _lib\n"
        "L = _lib.lib()\n"
        "b, w = ctypes.c_int(0), ctypes.c_int(0)\n"
        "r = [L.dlsh_tuned_encode(1024, 8, 0), L.dlsh_tuned_encode(512, 4, 1), L.dlsh_tuned_encode(256, 8, 0),\n"
        "     L.dlsh_tuned_encode(1024, 8, 9)]\n"
        "d = L.dlsh_tuned_decode(0, 1024, 8, ctypes.byref(b), ctypes.byref(w))\n"
        "r += [d, b.value, w.value]\n"
        "d = L.dlsh_tuned_decode(2, 700, 4, ctypes.byref(b), ctypes.byref(w))\n"
        "r += [d, b.value, w.value, L.dlsh_tuned_decode(1, 1024, 8, None, None), L.dlsh_tuned_decode(3, 1024, 8, None, None)]\n"
        "print(r)\n" % ROOT)
    env = dict(os.environ, DLSH_AUTOTUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    got = eval(out.stdout.strip().splitlines()[-1])
    # encoder: kernel 6 with a ring cap of 2; the older line; nothing recorded; bad precision
    assert got[:4] == [6 + 256 * 2, 2, 0, 0], got
    # decode: FP32 codes at K = 1024 (the shared-memory table), compact 16-bit codes
    # (internal format 3); nothing recorded for 8-bit codes; format out of range
    assert got[4:] == [1, 16, 14, 1, 8, 21, 0, 0], got


def test_binding_refuses_host_tensors_for_device_arguments():
    import torch

    from paper_2605_30396_gb300 import api
    import pytest
    with pytest.raises(ValueError):
        api._pd(torch.zeros(4))
    assert api._pd(None) is None


def test_encode_variant_choice(L):
    """The built-in encoder choice (host logic only): FP32 with s <= 8 on the
    selection/solver warps with FP16 parts, s > 8 on one tile per CTA with FP16
    parts, BF16/FP8 on two warp groups (one tile for s > 8); unsupported
    arguments give 0."""
    assert L.dlsh_encode_variant(1024, 8, 0) == 5
    assert L.dlsh_encode_variant(256, 1, 0) == 5
    assert L.dlsh_encode_variant(1024, 16, 0) == 7
    assert L.dlsh_encode_variant(1024, 8, 1) == 2
    assert L.dlsh_encode_variant(1024, 8, 2) == 2
    assert L.dlsh_encode_variant(1024, 16, 1) == 1
    assert L.dlsh_encode_variant(1024, 17, 1) == 0
    assert L.dlsh_encode_variant(0, 8, 0) == 0
    assert L.dlsh_encode_variant(1024, 0, 0) == 0
    assert L.dlsh_encode_variant(1024, 8, 5) == 0
