"""Pin of oracle.perfmodel: the paper's worked example of its cost model."""
import json
import os

from oracle import perfmodel as PM

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "perf_model_eq2_eq3.json")


def test_worked_example_of_eqs_2_and_3():
    g = json.load(open(GOLDEN))
    for key in ("original", "compressed"):
        c = g[key]
        tc, tm, t = PM.time_per_gaussian(c["flops"], c["bytes"], g["peak_flops"], g["bandwidth"])
        assert round(tc * 1e9, 4) == c["t_comp_ns"]
        assert round(tm * 1e9, 4) == c["t_mem_ns"]
        # the printed total is the sum of the two rounded parts
        assert round(round(tc * 1e9, 4) + round(tm * 1e9, 4), 4) == c["t_ns"]
        assert abs(t * 1e9 - c["t_ns"]) < 1e-4


def test_byte_counts_behind_the_example():
    g = json.load(open(GOLDEN))
    assert PM.sh_bytes_per_gaussian() == g["original"]["bytes"]
    # 11.7 (FP32 value, 32-bit index) pairs + 12 B of DC + a 4 B pointer = 109.6 B
    assert round(PM.csc_bytes_per_gaussian(g["mean_nonzeros"])) == g["compressed"]["bytes"]
