"""Benchmark of the sparse SH codec's hot path on one GB300 (or N replicas).

A step is one pass of the whole hot path over the scene-scale workload:
OMP encode of every Gaussian's 45 SH coefficients against the current dictionary
(correlation on tcgen05 + argmax + incremental Cholesky LS), the MOD dictionary
update with those codes, and a decode of one view-dependent colour per Gaussian
from a random camera.  Steps chain like learning iterations (step t encodes with
the dictionary step t-1 produced).

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, on a bounded sample of the same workload, on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("OMP Gaussians/s at K=1024,s=8, learned+BF16 vs plain at equal RMSE; decode GB/s")
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 : BF16 ratio
# DRAM bytes (read + write) per signal of the encoder, from one ncu capture of
# encode_kernel at N = 1,000,000, K = 1024, s = 8, FP32 (184.92 MB read +
# 37.26 MB written); the traffic grows with the number of signals, so a launch
# over N signals moves N times it.
ENCODE_TRAFFIC = {(1024, 8, "fp32"): (184.9216e6 + 37.260032e6) / 1_000_000}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=3_000_000)
    ap.add_argument("--K", type=int, default=1024)
    ap.add_argument("--s", type=int, default=8)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--workload", default="scene", choices=["scene", "multi"],
                    help="scene: the single-scene step (default); multi: 13 scenes of uneven "
                         "size, K and s encoded by one graph-captured multi-scene call")
    ap.add_argument("--multi-scale", type=float, default=1.0,
                    help="scale of the multi-scene Gaussian counts (1.0 = 0.5M..6M per scene)")
    ap.add_argument("--leg", default="step",
                    choices=["step", "encode", "mod", "decode", "decode_compact", "propose", "train",
                             "tolerance", "splat", "ksvd"],
                    help="time the whole step (default) or one leg alone, for profiling")
    return ap.parse_args()


def aggregate_ranks(ms_local: float, n_local: int, world: int, device=None):
    """Whole-job timing over replicas: the step time is the slowest rank's
    (max over ranks) and the value counts every rank's Gaussians.  Returns
    (ms, Gaussians/s).  With world > 1 the process group must be initialised."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local, float(n_local)], dtype=torch.float64, device=device)
        mx = t[:1].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        tot = t[1:].clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        ms, n = float(mx.item()), float(tot.item())
    else:
        ms, n = ms_local, float(n_local)
    return ms, n / (ms * 1e-3)


def workload(N, K, s, seed_offset=0):
    """Scene-scale inputs: hidden K-atom dictionary (rho = 0.6), s-sparse signals,
    initial dictionary from K signals, camera on a radius-4 sphere, means in [-1,1]^3."""
    from paper_2605_30396_gb300 import synth
    Dh = synth.hidden_dictionary(K, 0 + seed_offset, rho=0.6)
    X = synth.signals(N, Dh, s, 1 + seed_offset)
    init = synth.init_atom_indices(N, K, 0 + seed_offset)
    cam, mu = synth.camera_and_means(N, 2 + seed_offset, 3 + seed_offset)
    return X, init, cam, mu


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # let the sampler reach its steady 100 ms cadence before the timed
            # region starts, then keep only the samples taken inside it
            t0 = time.time()
            while not self.rows and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.rows = []
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _oracle_worker(args):
    D, X, s = args
    from oracle import omp as oomp
    return oomp.omp(D, X, s)["resid_sq"]


def cpu_oracle_rate(X, init, K, s, budget_s=15.0):
    """The FP64 oracle OMP timed on this host's cores over a bounded sample of the
    workload (processes started with spawn, one BLAS thread each)."""
    import multiprocessing as mp

    import numpy as np
    from oracle import mod as omod
    cores = os.cpu_count() or 1
    D0 = omod.init_dictionary(X, init)
    X = X[:400_000]
    # probe: size the sample for ~budget_s of work
    from oracle import omp as oomp
    n_probe = 2000
    t0 = time.perf_counter()
    oomp.omp(D0, X[:n_probe].astype(np.float64), s)
    per = (time.perf_counter() - t0) / n_probe
    n = int(min(len(X), max(cores * 200, budget_s * cores / max(per, 1e-9))))
    n = min(n, 400_000)
    chunks = np.array_split(np.arange(n), cores * 2)
    env_old = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            t0 = time.perf_counter()
            pool.map(_oracle_worker, [(D0, X[c].astype(np.float64), s) for c in chunks])
            dt = time.perf_counter() - t0
    finally:
        if env_old is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = env_old
    return {"value": n / dt, "unit": "Gaussians/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 numpy OMP (K={K}, s={s}) on the first {n} of the {len(X)} signals "
                      f"against the initial dictionary, {cores} spawn workers x 1 BLAS thread; "
                      f"{dt:.1f} s",
            "single_process": {"value": 1.0 / per, "unit": "Gaussians/s",
                               "sample": f"the first {n_probe} signals in one process"}}


def learned_leg(api, synth, D, X, s, K, cal_tau=1.01, n_train=2_000_000, n_cal=200_000,
                epochs=10, batch=8192, lr=1e-2, seed=7):
    """The learned encoder against plain FP32 OMP at (near) equal RMSE.

    The MLP is trained by the library's own kernels on (signal, OMP support)
    pairs the codec generates: n_train fresh signals from the same hidden
    dictionary, encoded with the current dictionary D.  The fallback threshold
    tau is calibrated on another fresh n_cal signals so that the deployed RMSE
    stays within cal_tau of plain OMP's; then both encoders are timed on X (the
    held-out scene, inputs resident)."""
    import numpy as np
    import torch
    Dh = synth.hidden_dictionary(K, 0, rho=0.6)
    Xtr = torch.from_numpy(synth.signals(n_train, Dh, s, seed)).cuda()
    itr, _, ntr, _ = api.encode(D, Xtr, s, sync=True)
    net = api.MLP(K, synth.mlp_params(K, seed))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.train(Xtr, itr, ntr, epochs=epochs, batch=batch, lr=lr)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del Xtr, itr, ntr
    Xc = torch.from_numpy(synth.signals(n_cal, Dh, s, seed + 1)).cuda()
    _, _, _, rp_c = api.encode(D, Xc, s, sync=True)
    cand = net.propose(Xc, 2 * s)
    _, _, _, rr_c = api.encode_restricted(D, Xc, cand, s)
    tau = api.calibrate_fallback(rr_c, rp_c, cal_tau)
    del Xc, cand

    N = X.shape[0]
    st = torch.cuda.current_stream()

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            r = fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    ms_plain, (_, _, _, rp) = timed(lambda: api.encode(D, X, s, precision="fp32"))
    ms_l, (_, _, _, rl, nfb) = timed(lambda: api.encode_learned(D, X, s, net, mode="deploy", tau=tau,
                                                               fallback_precision="bf16"))
    ms_b, (_, _, _, rb) = timed(lambda: api.encode(D, X, s, precision="bf16"))
    rm = lambda r: float(np.sqrt(r.double().sum().item() / (N * 45)))
    l = losses.float().cpu().numpy()
    return {
        "train_pairs": n_train, "train_epochs": epochs, "train_s": train_s,
        "train_loss_first_last": [float(l[:20].mean()), float(l[-20:].mean())],
        "tau": tau, "fallback_rate": int(nfb.item()) / N,
        "learned_bf16_gaussians_per_s": N / (ms_l * 1e-3),
        "plain_fp32_gaussians_per_s": N / (ms_plain * 1e-3),
        "plain_bf16_gaussians_per_s": N / (ms_b * 1e-3),
        "rmse_learned": rm(rl), "rmse_plain_fp32": rm(rp), "rmse_plain_bf16": rm(rb),
        "speedup_learned_vs_plain_fp32": ms_plain / ms_l,
    }


def multi_scenes(scale=1.0, n_scenes=13):
    """Config-5 scenes: K = (512, 1024, 2048)[i % 3], s = (4, 8, 16)[(i // 3) % 3],
    hidden dictionary of K atoms with seed 1000 + i, N log-uniform in
    [0.5M, 6M] (drawn with seed 0), times `scale`."""
    import numpy as np
    from paper_2605_30396_gb300 import synth
    rng = np.random.default_rng(0)
    ns = np.exp(rng.uniform(np.log(0.5e6), np.log(6e6), n_scenes))
    out = []
    for i in range(n_scenes):
        K = (512, 1024, 2048)[i % 3]
        s = (4, 8, 16)[(i // 3) % 3]
        N = max(1, int(round(ns[i] * scale)))
        Dh = synth.hidden_dictionary(K, 1000 + i)
        X = synth.signals(N, Dh, s, 2000 + i)
        init = synth.init_atom_indices(N, K, 3000 + i)
        cam, mu = synth.camera_and_means(N, 4000 + i, 5000 + i)
        out.append({"K": K, "s": s, "N": N, "X": X, "init": init, "cam": cam, "mu": mu})
    return out


def run_multi(a):
    """13 scenes encoded by one graph-captured dlsh_encode_multi call (each
    scene's (K, s) autotuned on a sample first), then decoded from one camera
    per scene.  A step = the graph replay plus the decodes."""
    import torch

    from paper_2605_30396_gb300 import _lib, api
    torch.cuda.set_device(0)
    L = _lib.lib()
    sc = multi_scenes(a.multi_scale)
    scenes, decs = [], []
    tuned = {}
    for x in sc:
        X = torch.from_numpy(x["X"]).cuda()
        D = api.init_dictionary(X, x["init"])
        key = (x["K"], x["s"])
        if key not in tuned:
            tuned[key] = api.autotune_encode(D, X[:65536], x["s"])
        scenes.append({"D": D, "X": X, "s": x["s"]})
        decs.append((torch.from_numpy(x["mu"]).cuda(), x["cam"]))
    total = sum(x["N"] for x in sc)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        api.encode_multi(scenes)  # warm-up: workspaces and internal streams exist
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        outs = api.encode_multi(scenes)
    rgbs = [torch.empty((x["N"], 3), dtype=torch.float32, device="cuda") for x in sc]

    def step():
        g.replay()
        for o, (mu, cam), sc_, rgb in zip(outs, decs, scenes, rgbs):
            api.decode(sc_["D"], o[0], o[1], o[2], means=mu, cam=cam, out=rgb)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = Clocks(0)
    clocks.start()
    launches0 = L.dlsh_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    cl = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    rm = []
    for o, x in zip(outs, sc):
        rm.append(float((o[3].double().sum() / (x["N"] * 45)).sqrt().item()))
    print(json.dumps({
        "metric": METRIC, "value": total / (ms * 1e-3), "unit": "Gaussians/s", "n_gpus": 1,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "multi-scene: 13 scenes, N log-uniform in [0.5M, 6M] x %g, "
                               "K in {512,1024,2048}, s in {4,8,16}; step = one graph replay of "
                               "the multi-scene encode + a decode per scene" % a.multi_scale,
                   "total_N": total, "scenes": [[x["N"], x["K"], x["s"]] for x in sc],
                   "tuned_bn": {f"{k[0]},{k[1]}": v for k, v in tuned.items()}},
        "gpu_launches_untimed_graph": L.dlsh_kernel_launches() - launches0,
        "clocks": cl, "detail": {"rmse_per_scene": rm},
    }))


def run_leg(a, api, L, X, MU, cam, D, out, rgb, stream):
    """One leg alone (encode or decode) for profiling: W untimed and K timed
    calls on resident inputs, CUDA events on the launching stream."""
    import torch
    N, K, s = a.N, a.K, a.s
    idx, coef, nnz, resid = out
    if a.leg == "decode":
        api.encode(D, X, s, precision=a.precision, out=out, sync=True)
        fn = lambda: api.decode(D, idx, coef, nnz, means=MU, cam=cam, out=rgb)
    elif a.leg == "decode_compact":
        api.encode(D, X, s, precision=a.precision, out=out, sync=True)
        idx_c, coef_c = api.compact_codes(idx, coef, K, sync=True)
        ref = api.decode(D, idx, coef, nnz, means=MU, cam=cam, sync=True).clone()
        fn = lambda: api.decode_compact(D, idx_c, coef_c, nnz, means=MU, cam=cam, out=rgb)
    elif a.leg == "mod":
        api.encode(D, X, s, precision=a.precision, out=out, sync=True)
        fn = lambda: api.mod_update(X, D, idx, coef, nnz, resid)
    elif a.leg in ("propose", "train"):
        # the proposal network at the learned encoder's sizes (2s candidates,
        # batches of 8192 training pairs), random-init weights
        from paper_2605_30396_gb300 import synth
        net = api.MLP(K, synth.mlp_params(K, 7))
        if a.leg == "propose":
            fn = lambda: net.propose(X, 2 * s)
        else:
            B = 8192
            ib, _, nb, _ = api.encode(D, X[:B], s, sync=True)
            fn = lambda: net.train_step(X[:B], ib, nb, lr=1e-3)
            N = B
    else:
        fn = lambda: api.encode(D, X, s, precision=a.precision, out=out)
    for _ in range(a.warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.steps, 1)
    line = {"leg": a.leg, "N": N, "K": K, "s": s, "precision": a.precision, "ms": ms,
            "gaussians_per_s": N / (ms * 1e-3)}
    if a.leg == "decode":
        line["GBps"] = N * (12 + 6 * s + 1 + 12) / (ms * 1e-3) / 1e9
    if a.leg == "decode_compact":
        ib = 1 if K <= 256 else 2
        line["GBps"] = N * (12 + (ib + 2) * s + 1 + 12) / (ms * 1e-3) / 1e9
        line["code_bytes_per_gaussian"] = {"fp32_ell": 6 * s + 1, "compact": (ib + 2) * s + 1}
        diff = (rgb - ref).double()
        line["rgb_rms_vs_fp32_decode"] = float(torch.sqrt((diff * diff).mean()).item())
        line["rgb_rms"] = float(torch.sqrt((ref.double() ** 2).mean()).item())
    print(json.dumps(line))


def tolerance_leg(a, api, X):
    """Tolerance-driven OMP (the residual stop of Sec. 2.1) and the CSC storage
    of Sec. 2.2 it implies.  The codes are taken against the workload's hidden
    dictionary with up to 16 atoms; each eps is relative to the RMS signal norm.
    Bytes per Gaussian: CSC with int64 column pointers, uint16 row indices and
    FP32 values, against 45 FP32 SH coefficients (180 B) without the DC term."""
    import numpy as np
    import torch
    from paper_2605_30396_gb300 import synth
    N, K = X.shape[0], a.K
    Dh = torch.from_numpy(synth.hidden_dictionary(K, 0, rho=0.6).astype(np.float32)).cuda()
    rms = float(torch.sqrt((X.double() ** 2).sum(dim=1).mean()).item())
    smax = 16
    st = torch.cuda.current_stream()
    rows = []
    for eps_rel in (0.03, 0.05, 0.1, 0.2):
        eps = eps_rel * rms
        out = (torch.empty((N, smax), dtype=torch.int16, device="cuda"),
               torch.empty((N, smax), dtype=torch.float32, device="cuda"),
               torch.empty((N,), dtype=torch.uint8, device="cuda"),
               torch.empty((N,), dtype=torch.float32, device="cuda"))
        api.encode(Dh, X, smax, eps=eps, precision=a.precision, out=out, sync=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(3):
            api.encode(Dh, X, smax, eps=eps, precision=a.precision, out=out)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        idx, coef, nnz, resid = out
        col_ptr, row_idx, val = api.csc_from_ell(idx, coef, nnz, sync=True)
        total = int(col_ptr[-1].item())
        nz = nnz.double()
        csc = 8 * (N + 1) + total * (2 + 4)
        rows.append({
            "eps_rel": eps_rel, "eps": eps, "mean_nnz": float(nz.mean().item()),
            "stopped_by_eps": float((resid.double() <= eps * eps).double().mean().item()),
            "rmse": float(np.sqrt(resid.double().sum().item() / (N * 45))),
            "csc_bytes_per_gaussian": csc / N,
            "compression_vs_45_fp32": 180.0 * N / csc,
            "dictionary_bytes": K * 45 * 4,
            "encode_ms": ms, "gaussians_per_s": N / (ms * 1e-3),
        })
    print(json.dumps({"leg": "tolerance", "N": N, "K": K, "s_max": smax, "precision": a.precision,
                      "rms_signal_norm": rms, "dictionary": "the workload's hidden dictionary",
                      "rows": rows}))


def ksvd_leg(a, api, X, init):
    """Objective against time for the two readings of the D-step: the learning
    loop {encode (FP32); D-update} from the same initial dictionary, with MOD or
    with the approximate K-SVD sweep.  Per iteration: the RMSE of the encoder's
    codes, the RMSE right after the update (K-SVD refits the coefficients; MOD
    keeps them), and the device times of both steps."""
    import numpy as np
    import torch
    N, K, s = X.shape[0], a.K, a.s
    st = torch.cuda.current_stream()
    iters = max(2, min(a.steps, 8))

    def rmse_of(D, idx, coef, nnz):
        il = idx.to(torch.int64) & 0xFFFF
        live = torch.arange(s, device="cuda")[None, :] < nnz[:, None].to(torch.int64)
        c = torch.where(live, coef, torch.zeros_like(coef)).double()
        rec = torch.zeros((N, 45), dtype=torch.float64, device="cuda")
        for t in range(s):
            rec += c[:, t, None] * D.double()[il[:, t]]
        r = X.double() - rec
        return float(torch.sqrt((r * r).sum() / (N * 45)).item())

    out = {}
    for method in ("mod", "ksvd"):
        D = api.init_dictionary(X, init)
        idx = torch.empty((N, s), dtype=torch.int16, device="cuda")
        coef = torch.empty((N, s), dtype=torch.float32, device="cuda")
        nnz = torch.empty((N,), dtype=torch.uint8, device="cuda")
        resid = torch.empty((N,), dtype=torch.float32, device="cuda")
        rows, cum = [], 0.0
        for it in range(iters):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(st)
            api.encode(D, X, s, precision="fp32", out=(idx, coef, nnz, resid))
            e[1].record(st)
            if method == "mod":
                Dn = api.mod_update(X, D, idx, coef, nnz, resid)
            else:
                Dn = api.ksvd_update(X, D, idx, coef, nnz, resid)
            e[2].record(st)
            torch.cuda.synchronize()
            enc_ms, upd_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
            cum += enc_ms + upd_ms
            rows.append({"iter": it, "rmse_codes": float(torch.sqrt(resid.double().sum() / (N * 45)).item()),
                         "rmse_after_update": rmse_of(Dn, idx, coef, nnz), "encode_ms": enc_ms,
                         "update_ms": upd_ms, "cumulative_ms": cum})
            D = Dn
        api.encode(D, X, s, precision="fp32", out=(idx, coef, nnz, resid))
        torch.cuda.synchronize()
        out[method] = {"iters": rows, "final_rmse": float(torch.sqrt(resid.double().sum() / (N * 45)).item())}
    print(json.dumps({"leg": "ksvd", "N": N, "K": K, "s": s, "precision": "fp32", **out}))


def splat_leg(a):
    """Splatting preprocess (project, cull, colour) of N synthetic Gaussians,
    with the colour read from 45 dense FP32 SH coefficients (the baseline
    renderer) or from sparse codes and the shared dictionary (Sec. 2.2), for two
    views: outside the cloud (nearly all Gaussians visible) and inside it (most
    culled).  Dictionaries: the scene's K = 1024 at s = 8, and the paper's
    rendering size K = 90 with 12 nonzeros (its mean k is 11.7).  Inputs
    (>= 300 MB) exceed L2.  Algorithmic HBM bytes per Gaussian: 52 in (mean,
    scale, rotation, DC) + 40 out (xy, depth, conic, radius, rgb), plus 180 B of
    SH per visible Gaussian, or the codes of every Gaussian.  The timed launches
    are replayed from a CUDA graph."""
    import numpy as np
    import torch
    from paper_2605_30396_gb300 import _lib, api, synth
    torch.cuda.set_device(0)
    N = a.N
    g = [torch.from_numpy(x).cuda() for x in synth.splat_gaussians(N, 11)]
    sh = (0.2 * torch.randn((N, 45), generator=torch.Generator().manual_seed(12))).cuda()
    views = {"outside": ((0.4, -3.2, 1.1), (0.0, 0.0, 0.0)), "inside": ((0.15, -0.1, 0.05), (1.0, 0.4, -0.3))}
    W, H, F = 1920, 1080, 1100.0
    codes = {}
    for K, s in ((1024, 8), (90, 12)):
        D = torch.from_numpy(synth.hidden_dictionary(K, 13).astype(np.float32)).cuda()
        idx, coef, nnz = synth.random_codes(N, K, s, 14, nnz_min=s)
        idx_t = torch.from_numpy(idx.astype(np.int16)).cuda()
        coef_t = torch.from_numpy(coef).cuda()
        nnz_t = torch.from_numpy(nnz).cuda()
        idx_c, coef_c = api.compact_codes(idx_t, coef_t, K, sync=True)
        codes[(K, s)] = (D, idx_t, coef_t, nnz_t, idx_c, coef_c)
    out = None
    st = torch.cuda.current_stream()
    rows = []
    for view, (eye, target) in views.items():
        R, t = synth.look_at(eye, target)
        cam = api.camera(R, t, F, F, W, H, 0.2)
        cases = [("sh", None, {"sh": sh})]
        for (K, s), (D, idx_t, coef_t, nnz_t, idx_c, coef_c) in codes.items():
            if K <= _lib.lib().dlsh_preprocess_max_k(s, 0):  # FP32 table in shared memory
                cases.append(("codes_fp32", (K, s), {"D": D, "idx": idx_t, "coef": coef_t, "nnz": nnz_t}))
            cases.append(("codes_compact", (K, s), {"D": D, "idx": idx_c, "coef": coef_c, "nnz": nnz_t}))
        vis = None
        for name, ks, kw in cases:
            fn = lambda: api.preprocess(cam, *g, out=out, **kw)
            out = fn()
            torch.cuda.synchronize()
            if vis is None:
                vis = float((out["radius"] > 0).double().mean().item())
            for _ in range(a.warmup):
                fn()
            # the timed launches are replayed from a CUDA graph, so that host
            # overhead between these short kernels does not enter the time
            graph = torch.cuda.CUDAGraph()
            reps = max(a.steps, 1)
            with torch.cuda.graph(graph):
                for _ in range(reps):
                    fn()
            graph.replay()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            graph.replay()
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            if name == "sh":
                colour_bytes = 180.0 * vis
            else:
                K, s = ks
                colour_bytes = (6 * s + 1) if name == "codes_fp32" else ((1 if K <= 256 else 2) + 2) * s + 1
            bpg = 92.0 + colour_bytes
            rows.append({"view": view, "colour": name, "K": ks[0] if ks else None, "s": ks[1] if ks else None,
                         "visible": vis, "ms": ms, "gaussians_per_s": N / (ms * 1e-3),
                         "bytes_per_gaussian": bpg, "GBps": N * bpg / (ms * 1e-3) / 1e9})
        base = next(r["ms"] for r in rows if r["view"] == view and r["colour"] == "sh")
        for r in rows:
            if r["view"] == view:
                r["speedup_vs_sh"] = base / r["ms"]
    print(json.dumps({"leg": "splat", "N": N, "image": [W, H], "focal": F, "rows": rows}))


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    X, init, cam, mu = workload(min(a.N, 400_000), a.K, a.s)
    cb = cpu_oracle_rate(X, init, a.K, a.s, budget_s=max(5.0, 60.0 / max(1, a.steps + a.warmup)))
    v = cb["value"]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Gaussians/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": a.N / v * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"scene N={a.N} d=45 K={a.K} s={a.s} (oracle on a sample)"},
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": "Gaussians/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "multi":
        return run_multi(a)
    if a.leg == "splat":
        return splat_leg(a)
    import numpy as np
    import torch

    from paper_2605_30396_gb300 import _lib, api, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    L = _lib.lib()
    N, K, s = a.N, a.K, a.s
    X_np, init, cam, mu = workload(N, K, s, seed_offset=100 * rank)
    X = torch.from_numpy(X_np).cuda()
    MU = torch.from_numpy(mu).cuda()
    D = api.init_dictionary(X, init)
    idx = torch.empty((N, s), dtype=torch.int16, device="cuda")
    coef = torch.empty((N, s), dtype=torch.float32, device="cuda")
    nnz = torch.empty((N,), dtype=torch.uint8, device="cuda")
    resid = torch.empty((N,), dtype=torch.float32, device="cuda")
    rgb = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    out = (idx, coef, nnz, resid)
    stream = torch.cuda.current_stream()

    ev = {k: [] for k in ("enc", "mod", "dec")}

    if a.leg == "tolerance":
        return tolerance_leg(a, api, X)
    if a.leg == "ksvd":
        return ksvd_leg(a, api, X, init)
    if a.leg != "step":
        return run_leg(a, api, L, X, MU, cam, D, out, rgb, stream)

    def step(Dcur, record=False):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        api.encode(Dcur, X, s, precision=a.precision, out=out)
        e1.record(stream)
        Dn = api.mod_update(X, Dcur, idx, coef, nnz, resid)
        e2.record(stream)
        api.decode(Dn, idx, coef, nnz, means=MU, cam=cam, out=rgb)
        e3.record(stream)
        if record:
            ev["enc"].append((e0, e1))
            ev["mod"].append((e1, e2))
            ev["dec"].append((e2, e3))
        return Dn

    Dcur = D
    for _ in range(a.warmup):
        Dcur = step(Dcur)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = L.dlsh_kernel_launches() if hasattr(L, "dlsh_kernel_launches") else None
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_start.record(stream)
    for _ in range(a.steps):
        Dcur = step(Dcur, record=True)
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = (L.dlsh_kernel_launches() - launches0) if launches0 is not None else None
    cl = clocks.stop()
    ms, value = aggregate_ranks(t_start.elapsed_time(t_end) / a.steps, N, world, device="cuda")
    enc_ms = statistics.mean(x.elapsed_time(y) for x, y in ev["enc"])
    mod_ms = statistics.mean(x.elapsed_time(y) for x, y in ev["mod"])
    dec_ms = statistics.mean(x.elapsed_time(y) for x, y in ev["dec"])
    rmse = float(np.sqrt(resid.double().sum().item() / (N * 45)))

    # roofline of the dominant kernel (encode: correlation GEMM on the tensor pipe)
    peaks, src = load_peaks()
    bf16 = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]))
    if a.precision == "fp32":
        peak = bf16 * TF32_PER_BF16 / 3.0
        peak_note = "TF32 dense (bf16 sustained x 1.1/2.25) / 3 for the 3xTF32 split"
    elif a.precision == "bf16":
        peak, peak_note = bf16, "bf16 dense sustained"
    else:
        peak, peak_note = bf16 * 2.0, "fp8 dense (bf16 sustained x 2)"
    flops = 2.0 * K * 45 * s * N  # algorithmic correlation FLOPs of one encode pass
    achieved = flops / (enc_ms * 1e-3) / 1e12
    dec_bytes = N * (12 + 6 * s + 1 + 12)  # means, idx+coef, nnz, rgb
    dec_gbs = dec_bytes / (dec_ms * 1e-3) / 1e9

    # End to end through the public API, one step per repetition.  The step's
    # inputs (signals, means, dictionary) go host -> device from pinned memory
    # and its results (codes, residuals, the new dictionary, the decoded
    # colours) come back to pinned host memory.  The copies run on a second
    # stream: the signals go in chunks, each chunk encoded as soon as it has
    # landed, and the codes go back while the MOD update and the decode run.
    e2e = None
    if not a.no_e2e:
        Xh = torch.from_numpy(X_np).pin_memory()
        MUh = MU.cpu().pin_memory()
        Dh = Dcur.cpu().pin_memory()
        oh = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (idx, coef, nnz, resid, rgb)]
        Dnh = torch.empty(Dh.shape, dtype=Dh.dtype).pin_memory()
        Xd = torch.empty_like(X)
        MUd = torch.empty_like(MU)
        Dd = torch.empty_like(Dcur)
        copy = torch.cuda.Stream()
        # chunk edges on whole waves of the encoder (one 128-signal tile per
        # SM), the first chunk small so that the encode starts early
        wave = 128 * torch.cuda.get_device_properties(0).multi_processor_count
        if N >= 40 * wave:
            first = 8 * wave
            rest = (N - first) // (3 * wave) * wave
            bnd = [0, first, first + rest, first + 2 * rest, N]
        else:
            bnd = [0, N]
        nch = len(bnd) - 1
        reps = max(1, min(3, a.steps))
        for rep in range(reps + 1):  # the first repetition is an untimed warm-up
            if rep == 1:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            landed = []
            with torch.cuda.stream(copy):
                Dd.copy_(Dh, non_blocking=True)
                for c in range(nch):
                    Xd[bnd[c]:bnd[c + 1]].copy_(Xh[bnd[c]:bnd[c + 1]], non_blocking=True)
                    landed.append(copy.record_event())
                MUd.copy_(MUh, non_blocking=True)
                mu_in = copy.record_event()
            for c in range(nch):
                stream.wait_event(landed[c])
                sl = slice(bnd[c], bnd[c + 1])
                api.encode(Dd, Xd[sl], s, precision=a.precision,
                           out=(idx[sl], coef[sl], nnz[sl], resid[sl]))
            coded = stream.record_event()
            with torch.cuda.stream(copy):
                copy.wait_event(coded)
                for h, d in zip(oh[:4], (idx, coef, nnz, resid)):
                    h.copy_(d, non_blocking=True)
            Dn = api.mod_update(Xd, Dd, idx, coef, nnz, resid)
            stream.wait_event(mu_in)
            api.decode(Dn, idx, coef, nnz, means=MUd, cam=cam, out=rgb)
            oh[4].copy_(rgb, non_blocking=True)
            Dnh.copy_(Dn, non_blocking=True)
            torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        h2d = X_np.nbytes + mu.nbytes + Dh.numel() * 4
        d2h = sum(t.numel() * t.element_size() for t in (idx, coef, nnz, resid, rgb)) + Dh.numel() * 4
        e2e = {"value": N / dt, "unit": "Gaussians/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "signal_chunks": nch}

    learned = None
    if not a.no_learned:
        learned = learned_leg(api, synth, Dcur, X, s, K)
        learned["workload"] = ("MLP 45-256-256-%d trained on 2M fresh (signal, OMP support) pairs; "
                               "learned proposal (2s candidates) + restricted OMP + BF16 plain-OMP "
                               "fallback on the %d scene signals" % (K, N))

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_oracle_rate(X_np, init, K, s)
    line = {
        "metric": METRIC, "value": value, "unit": "Gaussians/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"scene-scale: N={N} Gaussians x d=45 SH coeffs (FP32, rho=0.6), "
                               f"K={K} atoms, s={s}; step = OMP encode ({a.precision}) + MOD "
                               f"update + decode from a random camera",
                   "N": N, "K": K, "s": s, "precision": a.precision,
                   "l2": "inputs larger than L2 (X = %.0f MB)" % (X_np.nbytes / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": (ENCODE_TRAFFIC[(K, s, a.precision)] * N
                                 if (K, s, a.precision) in ENCODE_TRAFFIC else None),
                     "kernel": "encode_kernel (prep+gram included in the timing)",
                     "peak_source": f"{src}: {peak_note}"},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": cl,
        "detail": {"encode_ms": enc_ms, "encode_gaussians_per_s": N / (enc_ms * 1e-3),
                   "mod_ms": mod_ms, "decode_ms": dec_ms, "decode_GBps": dec_gbs,
                   "decode_hbm_frac": dec_gbs / float(peaks["hbm_gbs"]), "rmse": rmse,
                   "learned": learned},
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
