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
