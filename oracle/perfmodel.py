"""The paper's per-Gaussian cost model of the colour step (Sec. 2.2, Eqs. 2-3).

Test infrastructure only: the tests use it; the library never does.

The model charges a Gaussian's colour evaluation its arithmetic at the GPU's
FP32 rate plus its memory traffic at the DRAM bandwidth, the two added:
    T = FLOPs / peak_flops + bytes / bandwidth.
The original renderer reads the 48 SH floats of a Gaussian (192 bytes); the
compressed one reads the nonzero values and their indices, the DC colour and a
column pointer of the CSC storage; the shared dictionary is amortised away.

Pin (tests/test_oracle_perfmodel.py): the worked example the paper prints for
an RTX 4090 (tests/golden/perf_model_eq2_eq3.json).
"""
from __future__ import annotations


def time_per_gaussian(flops: float, nbytes: float, peak_flops: float, bandwidth: float):
    """(compute seconds, memory seconds, total seconds) of one Gaussian."""
    tc = flops / peak_flops
    tm = nbytes / bandwidth
    return tc, tm, tc + tm


def csc_bytes_per_gaussian(k: float, value_bytes: int = 4, index_bytes: int = 4, dc_bytes: int = 12,
                           pointer_bytes: int = 4) -> float:
    """Bytes a compressed Gaussian reads: k (value, index) pairs, its DC colour
    and one column pointer."""
    return k * (value_bytes + index_bytes) + dc_bytes + pointer_bytes


def sh_bytes_per_gaussian(n_floats: int = 48) -> float:
    """Bytes an uncompressed Gaussian reads: all of its SH coefficients."""
    return 4.0 * n_floats
