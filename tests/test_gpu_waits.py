"""Bounded device waits: a wait whose arrival never comes gives up after its
cycle budget with DLSH_ERR_TIMEOUT, and the CUDA context stays usable (the
pipelined kernels use the same mbarrier and grid-barrier helpers)."""
import numpy as np
import pytest
import torch

from oracle import omp as oomp
from paper_2605_30396_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu

DLSH_ERR_TIMEOUT = -4


@pytest.mark.parametrize("kind", [0, 1])
def test_lost_arrival_times_out_and_context_survives(lib, kind):
    L = _lib.lib()
    n = L.dlsh_selftest_workspace_size()
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    # about a millisecond at GB300 clocks
    rc = L.dlsh_selftest_bounded_wait(kind, 2_000_000, ws.data_ptr(), n,
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == DLSH_ERR_TIMEOUT, (rc, L.dlsh_last_error())
    assert b"ran out" in L.dlsh_last_error()
    # the context still runs kernels and gives correct results
    K, s, N = 64, 4, 500
    D = synth.hidden_dictionary(K, 3).astype(np.float32)
    X = synth.signals(N, D.astype(np.float64), s, 4)
    idx, coef, nnz, resid = api.encode(torch.from_numpy(D).cuda(), torch.from_numpy(X).cuda(), s, sync=True)
    ref = oomp.omp(D.astype(np.float64), X.astype(np.float64), s)
    rg = float(np.sqrt(resid.double().sum().item() / (N * 45)))
    ro = float(np.sqrt(ref["resid_sq"].sum() / (N * 45)))
    assert abs(rg - ro) <= 1e-4 * ro


def test_bad_arguments_rejected(lib):
    L = _lib.lib()
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert L.dlsh_selftest_bounded_wait(2, 1000, ws.data_ptr(), 256, st) != 0
    assert L.dlsh_selftest_bounded_wait(0, 0, ws.data_ptr(), 256, st) != 0
    assert L.dlsh_selftest_bounded_wait(0, 1000, ws.data_ptr(), 16, st) != 0
