#!/usr/bin/env python3
"""Benchmark of the GB300 kernel-ridge-regression hot path.

One step is one pass of the whole path on the SUSY-shaped workload
(n = 65536 training points, d = 8, 16-component Gaussian mixture,
standardized; h = 1, lambda = 4, leaf 128): feature standardization,
recursive two-means ordering, randomized HSS compression (adaptive
sampling through the fused tcgen05 kernel-times-block product), ULV-type
factorization, HSS-preconditioned GMRES to the relative residual 10 eps
(eps = 1e-4) for 10 right-hand sides, and prediction of 4096 test points.

Reported (one JSON line on rank 0): seconds per step (mixed precision),
the FP64 "plain" GPU path on the same step, the fused sampling kernel's
algorithmic TFLOP/s against the measured tensor peak, an end-to-end time
through host buffers, and the CPU oracle's time on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "kernel-sampling TFLOP/s and KRR compress+solve sec at n=65536: mixed vs FP64 plain"
WL = dict(n=65536, d=8, comps=16, sigma=0.7, seed=2, h=1.0, lam=4.0, leaf=128, eps=1e-4, eps_c=0.05, r0=64,
          nrhs=10, m_test=4096)
WORKLOAD = ("SUSY-shaped synthetic Gaussian mixture (16 components, d=8, standardized), n=65536 train / 4096 test; "
            "h=1, lambda=4, leaf 128, eps=1e-4 (GMRES to relative residual 5e-4 <= 10 eps), HSS eps_c=0.05, "
            "r0=64 adaptive, 10 right-hand sides")
CPU_SAMPLE_N = 16384  # about 10-20 s of the oracle on 8-16 host cores


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_source_hash():
    """sha1 of the fused kernel's source: DRAM counters taken from an ncu
    capture are valid only for the kernel they were measured on."""
    import hashlib
    with open(os.path.join(ROOT, "paper_1803_10274_gb300", "csrc", "sample_tc.cu"), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def _traffic():
    """DRAM bytes per launch (n=65536, r=256) from profiles/sample_tc_traffic.txt,
    or None when that capture was taken on a different kernel source."""
    vals = {}
    try:
        with open(os.path.join(ROOT, "profiles", "sample_tc_traffic.txt")) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 2:
                    vals[parts[0]] = parts[1]
    except OSError:
        return None
    if vals.get("kernel_source_sha1") != kernel_source_hash():
        return None
    v = vals.get("bytes_per_launch_n65536_r256")
    return int(v) if v else None


def _dense_accuracy():
    """Test accuracy of the exact dense FP64 solve of this workload, written
    by the oracle into tests/golden/dense_n65536.txt (its inputs are
    standardized in FP64; the bench's on the GPU: the same data up to FP32
    rounding)."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "dense_n65536.txt")) as f:
            for line in f:
                if line.startswith("accuracy:"):
                    return float(line.split(":")[1])
    except OSError:
        pass
    return None


def _inputs():
    import synth
    X, y, Xt, yt, _, _ = synth.mixture(WL["n"], WL["d"], WL["comps"], WL["sigma"], WL["seed"], WL["m_test"])
    Y = np.concatenate([y[:, None], np.random.default_rng(3).standard_normal((WL["n"], WL["nrhs"] - 1))], 1)
    return X.astype(np.float32), Xt.astype(np.float32), np.ascontiguousarray(Y), yt


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, dev):
        self.dev = dev
        self.p = None
        self.f = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except Exception:
                self.p.kill()

    def summary(self):
        if not self.f:
            return None
        try:
            rows = [l.strip().split(", ") for l in open(self.f.name) if l.strip()]
        except Exception:
            return None
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) >= 9:
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _flush_l2(buf):
    buf.add_(1.0)


def max_over_ranks(value):
    """Largest value over the ranks of the initialized process group (the
    slowest replica sets the step time).  The tensor lives where the
    backend wants it: on the GPU for NCCL, on the host for gloo."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch
    import paper_1803_10274_gb300 as K
    from paper_1803_10274_gb300 import _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    peaks, peak_src = _peaks()
    ctx = K.Context()
    # The step runs the fused product's default launch variants: autotuned
    # variants change the products' summation order, and with it the IDs and
    # the GMRES iteration count (23 against 27 at this size), by more than
    # they gain.  The kernel-alone measurements below are autotuned.
    stream = ctx.stream
    X, Xt, Y, yt = _inputs()
    Xd, Xtd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Xt).cuda(), torch.from_numpy(Y).cuda()
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    tol = 0.5 * 10 * WL["eps"]

    def opts(prec):
        return K.default_options(h=WL["h"], lambda_=WL["lam"], eps_c=WL["eps_c"], leaf=WL["leaf"], precision=prec,
                                 seed=WL["seed"], r0=WL["r0"])

    def step(prec, Xs, Xts, Ys):
        K.krr_standardize(ctx, Xs, Xts)
        H = K.hss_compress(ctx, Xs, opts(prec))
        H.factor()
        a, res = H.solve(Ys, tol=tol, max_refine=200)
        dec = H.predict(Xts, a[:, :1].contiguous())
        st = H.stats()
        H.close()
        return a, dec, res, st

    def timed_step(prec):
        Xs, Xts = Xd.clone(), Xtd.clone()
        _flush_l2(l2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        a, dec, res, st = step(prec, Xs, Xts, Yd)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, a, dec, res, st

    for _ in range(args.warmup):
        timed_step(K.KRR_MIXED)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    l0 = _lib.lib().krr_launch_count()
    times, last = [], None
    with Clocks(dev) as clk:
        for _ in range(args.steps):
            t, a, dec, res, st = timed_step(K.KRR_MIXED)
            times.append(t)
            last = (a, dec, res, st)
    launches = (_lib.lib().krr_launch_count() - l0) // max(args.steps, 1)
    t_step = sum(times) / len(times)
    if world > 1:
        t_step = max_over_ranks(t_step)
    a, dec, res, st = last
    acc = float(np.mean(np.where(dec.cpu().numpy()[:, 0] >= 0, 1.0, -1.0) == yt))

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- fused sampling kernel alone: algorithmic TFLOP/s (CUDA events on the library's stream)
    ctx.set_autotune(True)  # launch variants picked by measurement (first call of each shape class)
    Xs = Xd.clone()
    K.krr_standardize(ctx, Xs)
    samp = {}
    n, d = WL["n"], WL["d"]
    for r in (64, 256):
        R = torch.from_numpy(np.random.default_rng(7).standard_normal((n, r)).astype(np.float16).astype(np.float32)).cuda()
        S = torch.empty(n, r, device="cuda")
        for _ in range(3):
            K.krr_sample(ctx, Xs, Xs, WL["h"], 0.0, R, S=S)
        ts = []
        for _ in range(5):
            _flush_l2(l2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            K.krr_sample(ctx, Xs, Xs, WL["h"], 0.0, R, S=S)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        t = statistics.median(ts)
        samp[r] = (2.0 * n * n * (d + r) / t / 1e12, t)
    ach, tk = samp[256]
    peak = float(peaks["bf16_tflops"])
    traffic = _traffic()
    # arithmetic-pipe rates measured now (krr_probe_rate) and the secondary
    # bounds: the fused kernel's exponentials (n^2 per launch) against the
    # SFU's ex2 rate, the FP64 comparator's product against the FP64 FMA rate
    rates = {"fp32_fma_tflops": ctx.probe_rate(0) / 1e12, "fp64_fma_tflops": ctx.probe_rate(1) / 1e12,
             "ex2_per_s": ctx.probe_rate(2), "f32_to_f16_per_s": ctx.probe_rate(3)}
    n64 = 16384
    Xf = torch.from_numpy(X[:n64].astype(np.float64)).cuda()
    R64 = torch.from_numpy(np.random.default_rng(7).standard_normal((n64, 64))).cuda()
    S64 = torch.empty(n64, 64, dtype=torch.float64, device="cuda")
    K.krr_sample_f64(ctx, Xf, Xf, WL["h"], 0.0, R64, S=S64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    K.krr_sample_f64(ctx, Xf, Xf, WL["h"], 0.0, R64, S=S64)
    e1.record(stream)
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) / 1e3
    f64_tflops = 2.0 * n64 * n64 * (d + 64) / t64 / 1e12
    secondary = {"ex2_frac_r256": (n * n / samp[256][1]) / rates["ex2_per_s"],
                 "ex2_frac_r64": (n * n / samp[64][1]) / rates["ex2_per_s"],
                 "tensor_frac_r64": samp[64][0] / peak,
                 "fp64_product_n16384_r64": {"seconds": t64, "tflops": f64_tflops,
                                             "frac_of_fp64_fma": f64_tflops / rates["fp64_fma_tflops"]}}

    ctx.set_autotune(False)  # the end-to-end steps and the extra workloads: default variants, as the step
    # ---- end to end through host buffers (H2D inputs, D2H weights + predictions inside the timed region)
    Xh = torch.from_numpy(X).pin_memory()
    Xth = torch.from_numpy(Xt).pin_memory()
    Yh = torch.from_numpy(Y).pin_memory()
    ah = torch.empty((n, WL["nrhs"]), dtype=torch.float64).pin_memory()
    dh = torch.empty((WL["m_test"], 1), dtype=torch.float64).pin_memory()
    e_times = []
    for it in range(max(1, min(args.steps, 2)) + 1):
        _flush_l2(l2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xs = Xh.to("cuda", non_blocking=True)
        Xts = Xth.to("cuda", non_blocking=True)
        Ys = Yh.to("cuda", non_blocking=True)
        a, dec, res, st2 = step(K.KRR_MIXED, Xs, Xts, Ys)
        ah.copy_(a, non_blocking=True)
        dh.copy_(dec, non_blocking=True)
        torch.cuda.synchronize()
        if it > 0:
            e_times.append(time.perf_counter() - t0)
    e2e = sum(e_times) / len(e_times)
    h2d = X.nbytes + Xt.nbytes + Y.nbytes
    d2h = ah.numel() * 8 + dh.numel() * 8

    # ---- held-out loss gradient (COVTYPE-shaped) and the million-point product
    extras = {} if args.no_extras else {"gradient": bench_gradient(K, ctx, l2),
                                        "million_point_product": bench_million(K, ctx),
                                        "batch": bench_batch(K, ctx, l2),
                                        "image_d784": bench_image(K, ctx, l2),
                                        "orderings": bench_orderings(K, ctx, l2)}

    # ---- FP64 plain path, same step (one run: it is slow)
    plain = None
    if not args.no_plain:
        tp, ap, decp, resp, stp = timed_step(K.KRR_FP64)
        plain = {"seconds": tp, "resid_gpu": resp, "max_rank": stp["max_rank"], "samples": stp["samples"],
                 "gmres_iters": stp["refine_steps"]}

    # ---- CPU oracle on a bounded sample
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline(X)

    t_sample_frac = st["t_sample_ms"] / 1e3 / t_step if t_step > 0 else None
    out = {
        "metric": METRIC,
        "value": t_step,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_step,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f16 tensor-core products with f32 accumulation; f32 ID/ULV/GMRES preconditioner; f64 residuals",
        "data": "synthetic (seeded Gaussian mixture, SUSY-shaped)",
        "config": {"workload": WORKLOAD, "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "quality": {"resid_gpu": res, "test_accuracy": acc, "test_accuracy_dense": _dense_accuracy(),
                    "max_rank": st["max_rank"], "samples": st["samples"],
                    "rounds": st["rounds"], "gmres_iters": st["refine_steps"],
                    "hss_memory_MB": st["memory_bytes"] / 1e6},
        "phases_ms": {k: st[k] for k in ("t_cluster_ms", "t_sample_ms", "t_compress_ms", "t_factor_ms",
                                         "t_solve_ms")},
        "fp64_plain": plain,
        **extras,
        "sampling": {"tflops_r64": samp[64][0], "ms_r64": 1e3 * samp[64][1], "tflops_r256": samp[256][0],
                     "ms_r256": 1e3 * samp[256][1], "algorithmic_flops": "2 n^2 (d + r)",
                     "share_of_step": t_sample_frac, "secondary_bounds": secondary},
        "measured_rates": rates,
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                     "traffic": traffic,
                     "note": "fused sampling kernel, n=65536, d=8, r=256, one launch timed alone (burst peak, %s)"
                             % ("of " + peak_src)},
        "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


GRAD_WL = dict(n=16384, d=54, comps=7, cls=2, seed=4, m_test=4096, h=3.0, lam=1.0, eps_c=0.1, leaf=128, tol=1e-6)


def bench_gradient(K, ctx, l2, reps=3):
    """Held-out squared loss and its gradient in h, lambda and X on the
    COVTYPE-shaped workload (n=16384, d=54 standardized, 7-component
    mixture, one-vs-rest labels for class 2, 4096 held out; h=3, lambda=1):
    one timed step = HSS compression + krr_heldout_grad (two preconditioned
    solves to 1e-6 and the augmented fused products)."""
    import torch
    import synth
    W = GRAD_WL
    X, _, Xt, _, c, ct = synth.mixture(W["n"], W["d"], W["comps"], 0.7, W["seed"], W["m_test"])
    y, yt = synth.labels_one_vs_rest(c, W["cls"]), synth.labels_one_vs_rest(ct, W["cls"])
    # standardizing the inputs (krr_standardize) is data preparation, not part of the timed step
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    Xtd = torch.from_numpy(Xt.astype(np.float32)).cuda()
    K.krr_standardize(ctx, Xd, Xtd)
    yd, ytd = torch.from_numpy(y).cuda(), torch.from_numpy(yt).cuda()
    o = K.default_options(h=W["h"], lambda_=W["lam"], eps_c=W["eps_c"], leaf=W["leaf"], precision=K.KRR_MIXED)

    def once(full):
        _flush_l2(l2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        H = K.hss_compress(ctx, Xd, o)
        r = H.heldout_grad(Xtd, yd, ytd, tol=W["tol"], max_refine=400, grad=full)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        st = H.stats()
        H.close()
        return e0.elapsed_time(e1) / 1e3, r, st

    once(True)
    tg = [once(True) for _ in range(reps)]
    tl = [once(False) for _ in range(reps)]
    t, r, st = tg[-1]
    return {"workload": "COVTYPE-shaped mixture n=16384, d=54, 4096 held out, h=3, lambda=1, HSS eps_c=0.1, "
                        "solves to 1e-6",
            "seconds_loss_and_grad": statistics.median(x[0] for x in tg),
            "seconds_loss_only": statistics.median(x[0] for x in tl),
            "loss": r["loss"], "dL_dh": r["dh"], "dL_dlambda": r["dlambda"],
            "gmres_iters_both_solves": st["refine_steps"], "max_rank": st["max_rank"]}


BATCH_WL = dict(nprob=256, n_lo=512, n_hi=8192, dims=(8, 32, 128), hs=(0.5, 1.0, 2.0, 4.0), nrhs=16, lam=1.0,
                eps_c=0.05, eps_abs=1e-2, r_max=1024, tol=1e-4, max_refine=600, seed=5)


def batch_groups(W, K, ctx):
    """The batched workload's data: one group per feature dimension, each a
    list of (X, Y, h) systems (X on the device, standardized per problem by
    krr_standardize); the 256 problems' sizes and dimensions are drawn from
    the workload seed."""
    import torch
    import synth
    rng = np.random.default_rng(W["seed"])
    sizes = rng.integers(W["n_lo"], W["n_hi"] + 1, size=W["nprob"])
    dims = rng.choice(W["dims"], size=W["nprob"])
    groups = {}
    for d in W["dims"]:
        systems = []
        for p in np.nonzero(dims == d)[0]:
            X, y, *_ = synth.mixture(int(sizes[p]), int(d), 4, 0.7, 1000 + int(p))
            Z = torch.from_numpy(X.astype(np.float32)).cuda()
            K.krr_standardize(ctx, Z)
            Y = np.concatenate([y[:, None], rng.standard_normal((len(y), W["nrhs"] - 1))], 1)
            for h in W["hs"]:
                systems.append((Z, Y, h))
        groups[int(d)] = systems
    return groups


def group_precision(d, h, eps_c, r_max):
    """Arithmetic and sample budget of one (d, h) group of the batched
    workload: (precision, eps_c, r_max).  On standardized data the typical
    squared distance is about 2 d, so the kernel's off-diagonal entries are
    about exp(-d / h^2): with d / h^2 <= 2 (d = 8 at h = 2, 4; d = 32 at
    h = 4) the blocks are large next to lambda = 1 and the FP32
    factorization of the compressed matrix does not precondition GMRES, so
    those groups factor in FP64 (KRR_MIXED_F64; the products stay on tensor
    cores), and the smoothest (d / h^2 <= 0.5) also compress to eps_c = 0.02
    instead of 0.05.  Every group keeps the workload's sample budget
    (r_max = 1024): 2048 samples for the d = 128, h = 4 group (truncated at
    1024, 210 GMRES iterations) took 2.0 s instead of 3.7 s in a single pass,
    but the second pass of the whole workload then ran out of device
    memory."""
    s = d / (h * h)
    if s <= 0.5:
        return "mixed_f64", 0.02, r_max
    if s <= 2.0:
        return "mixed_f64", eps_c, r_max
    return "mixed", eps_c, r_max


def bench_batch(K, ctx, l2, reps=2):
    """Many independent problems: 256 seeded mixture data sets with
    n ~ U[512, 8192] and d drawn from {8, 32, 128}, each at four widths
    h in {0.5, 1, 2, 4}, 16 right-hand sides, lambda = 1.  One batched
    handle per (d, h) group: all its problems in one block-diagonal HSS
    (compress + factor) and one GMRES to 1e-4 over the group.  A step is
    every group; groups whose GMRES stops above the tolerance are reported
    with the residual they reached."""
    import torch
    W = BATCH_WL
    groups = []
    for d, systems in batch_groups(W, K, ctx).items():
        for h in W["hs"]:
            sel = [(x, y) for x, y, hh in systems if hh == h]
            off = np.concatenate([[0], np.cumsum([x.shape[0] for x, _ in sel])]).astype(np.int64)
            groups.append((d, h, torch.cat([x for x, _ in sel]).contiguous(),
                           torch.from_numpy(np.ascontiguousarray(np.concatenate([y for _, y in sel]))).cuda(), off))

    def step():
        out = []
        for d, h, X, Y, off in groups:
            prec, eps_c, r_max = group_precision(d, h, W["eps_c"], W["r_max"])
            o = K.default_options(lambda_=W["lam"], eps_c=eps_c, eps_abs=W["eps_abs"], r_max=r_max,
                                  flags=K.KRR_TRUNCATE_AT_RMAX | K.KRR_LAMBDA_TOL, leaf=128, seed=W["seed"],
                                  precision=K.KRR_MIXED_F64 if prec == "mixed_f64" else K.KRR_MIXED)
            H = K.hss_compress_batched(ctx, X, off, [h] * (len(off) - 1), o)
            H.factor()
            a, res = H.solve(Y, tol=W["tol"], max_refine=W["max_refine"], raise_on_no_convergence=False)
            st = H.stats()
            H.close()
            out.append({"d": d, "h": h, "precision": prec, "eps_c": eps_c, "r_max": r_max, "problems": len(off) - 1,
                        "rows": int(off[-1]), "resid": res,
                        "converged": bool(0 <= res <= W["tol"]), "max_rank": st["max_rank"],
                        "samples": st["samples"], "truncated": st["truncated"], "gmres_iters": st["refine_steps"]})
        return out

    step()
    ts = []
    for _ in range(reps):
        _flush_l2(l2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        info = step()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.median(ts)
    nsys = sum(g["problems"] for g in info)
    return {"workload": "256 mixture problems, n ~ U[512, 8192], d in {8, 32, 128}, 4 widths each, 16 RHS, "
                        "lambda 1; one batched handle per (d, h): HSS eps_c 0.05 (0.02 where d/h^2 <= 0.5) relative to "
                        "min(block, lambda), pivot floor 1e-2, <= 1024 samples (truncated beyond), FP64 "
                        "decompositions and factorization where d/h^2 <= 2; GMRES to 1e-4 over each group, at most "
                        "600 iterations",
            "seconds": t, "systems_per_second": nsys / t,
            "systems_converged": sum(g["problems"] for g in info if g["converged"]), "systems": nsys,
            "groups": info}


# eps_c: the compression tolerance measured fastest for this workload at the
# same GMRES tolerance (compress + factor + solve + predict: 0.30 s at 0.05
# with 26 iterations, 0.19 s at 0.02, 0.17 s at 0.01 with 5, 0.67 s at
# 0.005); the comparison of the orderings keeps 0.05 (eps_c_orderings).
IMAGE_WL = dict(n=32768, m_test=2000, h=4.0, lam=10.0, leaf=256, eps=1e-3, eps_c=0.01, eps_c_orderings=0.05, seed=3)


def bench_image(K, ctx, l2, reps=2):
    """MNIST-shaped workload (d = 784 raw pixels in [0, 1], about 80 % exact
    zeros, one-vs-all class 5; the paper's MNIST uses h = 4): n = 32768,
    h = 4, lambda = 10, leaf 256, compression eps_c = 0.01, GMRES to
    eps = 1e-3.  Timed: compress + factor + solve + predict; also the fused
    product alone at r = 64 (2 n^2 (d + r) flop)."""
    import torch
    import synth
    W = IMAGE_WL
    X, y, Xt, yt = synth.image_like(W["n"], W["seed"], m_test=W["m_test"])
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    Xtd = torch.from_numpy(Xt.astype(np.float32)).cuda()
    yd = torch.from_numpy(y[:, None].copy()).cuda()
    o = K.default_options(h=W["h"], lambda_=W["lam"], eps_c=W["eps_c"], leaf=W["leaf"], seed=W["seed"])

    def once():
        _flush_l2(l2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        H = K.hss_compress(ctx, Xd, o)
        H.factor()
        a, res = H.solve(yd, tol=W["eps"], max_refine=400)
        dec = H.predict(Xtd, a)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        st = H.stats()
        H.close()
        return e0.elapsed_time(e1) / 1e3, res, dec, st

    once()
    runs = [once() for _ in range(reps)]
    t = statistics.median(x[0] for x in runs)
    _, res, dec, st = runs[-1]
    acc = float(np.mean(np.where(dec.cpu().numpy()[:, 0] >= 0, 1.0, -1.0) == yt))
    n, d, r = W["n"], X.shape[1], 64
    R = torch.from_numpy(synth.gaussian_block(n, r, 9).astype(np.float32)).cuda()
    S = torch.empty(n, r, device="cuda")
    K.krr_sample(ctx, Xd, Xd, W["h"], 0.0, R, S=S)
    ts = []
    for _ in range(3):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        K.krr_sample(ctx, Xd, Xd, W["h"], 0.0, R, S=S)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    tp = statistics.median(ts)
    return {"workload": "MNIST-shaped image-like rows, n=32768, d=784, h=4, lambda=10, leaf 256, eps_c %g, "
                        "GMRES to 1e-3, 2000 test points" % W["eps_c"],
            "seconds": t, "resid_gpu": res, "test_accuracy": acc, "max_rank": st["max_rank"],
            "samples": st["samples"], "gmres_iters": st["refine_steps"],
            "phases_ms": {k: st[k] for k in ("t_cluster_ms", "t_sample_ms", "t_compress_ms", "t_factor_ms",
                                             "t_solve_ms")},
            "product_r64": {"seconds": tp, "tflops": 2.0 * n * n * (d + r) / tp / 1e12}}


ORDER_NAMES = {0: "2MN", 1: "NP", 2: "KD", 3: "PCA"}


def bench_orderings(K, ctx, l2):
    """The comparison of the paper's Section 5.2 table on the synthetic
    stand-ins: HSS memory (D, U, B generators), largest rank, samples,
    test accuracy and compress + factor + solve time for each ordering of
    Section 4.3, on the SUSY-shaped workload (n = 65536, d = 8; all four)
    and the MNIST-shaped one (n = 32768, d = 784; the principal-direction
    ordering is limited to d <= 64).  Sample budget 2048 columns; a
    compression that would need more keeps truncated decompositions and is
    marked so.  Reported, not gated."""
    import torch
    import synth
    out = {}
    X, y, Xt, yt, _, _ = synth.mixture(WL["n"], WL["d"], WL["comps"], WL["sigma"], WL["seed"], WL["m_test"])
    Xs = torch.from_numpy(X.astype(np.float32)).cuda()
    Xts = torch.from_numpy(Xt.astype(np.float32)).cuda()
    K.krr_standardize(ctx, Xs, Xts)
    Xi, yi, Xti, yti = synth.image_like(IMAGE_WL["n"], IMAGE_WL["seed"], m_test=IMAGE_WL["m_test"])
    cases = [("susy_n65536_d8", Xs, Xts, y, yt, WL["h"], WL["lam"], WL["leaf"], WL["eps_c"], 10 * WL["eps"] / 2,
              (0, 1, 2, 3)),
             ("mnist_n32768_d784", torch.from_numpy(Xi.astype(np.float32)).cuda(),
              torch.from_numpy(Xti.astype(np.float32)).cuda(), yi, yti, IMAGE_WL["h"], IMAGE_WL["lam"],
              IMAGE_WL["leaf"], IMAGE_WL["eps_c_orderings"], IMAGE_WL["eps"], (0, 1, 2))]
    for name, Xd, Xtd, yv, ytv, h, lam, leaf, eps_c, tol, orders in cases:
        res = {}
        yd = torch.from_numpy(np.ascontiguousarray(yv[:, None])).cuda()
        for od in orders:
            o = K.default_options(h=h, lambda_=lam, eps_c=eps_c, leaf=leaf, seed=WL["seed"], ordering=od,
                                  flags=K.KRR_TRUNCATE_AT_RMAX)
            _flush_l2(l2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            H = K.hss_compress(ctx, Xd, o)
            H.factor()
            a, rr = H.solve(yd, tol=tol, max_refine=400, raise_on_no_convergence=False)
            dec = H.predict(Xtd, a)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            st = H.stats()
            H.close()
            acc = float(np.mean(np.where(dec.cpu().numpy()[:, 0] >= 0, 1.0, -1.0) == ytv))
            res[ORDER_NAMES[od]] = {"hss_memory_MB": st["memory_bytes"] / 1e6, "max_rank": st["max_rank"],
                                    "samples": st["samples"], "truncated": st["truncated"],
                                    "gmres_iters": st["refine_steps"], "resid_gpu": rr, "test_accuracy": acc,
                                    "seconds": e0.elapsed_time(e1) / 1e3}
        out[name] = res
    return out


def bench_million(K, ctx, n=1 << 20, r=256, reps=2):
    """One fused product S = K R at n = 1,048,576, d = 8, r = 256 (about
    5.8e14 algorithmic flops), inputs resident, CUDA events."""
    import torch
    import synth
    d = 8
    X = synth.mixture(n, d, 16, 0.7, 6)[0]
    X = ((X - X.mean(0)) / X.std(0)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    R = torch.from_numpy(synth.gaussian_block(n, r, 6).astype(np.float32)).cuda()
    S = torch.empty(n, r, device="cuda")
    K.krr_sample(ctx, Xd, Xd, 1.0, 0.0, R, S=S)
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        K.krr_sample(ctx, Xd, Xd, 1.0, 0.0, R, S=S)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.median(ts)
    del R, S
    torch.cuda.empty_cache()
    return {"n": n, "d": d, "r": r, "seconds": t, "tflops": 2.0 * n * n * (d + r) / t / 1e12,
            "algorithmic_flops": "2 n^2 (d + r)"}


def solve_only(reps=8, n=None):
    """Compression and factorization of the benchmark workload (or of its
    first n points), then reps single ULV solves (no refinement) of its 10
    right-hand sides, for profiling the factor and solve kernels; prints the
    mean solve time."""
    import torch
    import paper_1803_10274_gb300 as K
    torch.cuda.set_device(0)
    ctx = K.Context()
    X, Xt, Y, yt = _inputs()
    if n:
        X, Y = X[:n], np.ascontiguousarray(Y[:n])
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    K.krr_standardize(ctx, Xd)
    o = K.default_options(h=WL["h"], lambda_=WL["lam"], eps_c=WL["eps_c"], leaf=WL["leaf"], precision=K.KRR_MIXED,
                          seed=WL["seed"], r0=WL["r0"])
    H = K.hss_compress(ctx, Xd, o)
    H.factor()
    H.solve(Yd, tol=0.0)
    ctx.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(reps):
        H.solve(Yd, tol=0.0)
    e1.record(ctx.stream)
    ctx.sync()
    print(json.dumps({"n": len(X), "nrhs": WL["nrhs"], "ulv_solve_ms": e0.elapsed_time(e1) / reps}), flush=True)
    H.close()


def gemm_only(nb):
    """nb Gram products S_b S_b^T of 128 x 2032 FP32 blocks (a level of
    interpolative decompositions at 2048 samples) through
    krr_gemm_f32_batched on the tensor cores and on the CUDA cores; prints
    the mean time and TFLOP/s of each (for profilers)."""
    import torch
    import paper_1803_10274_gb300 as K
    torch.cuda.set_device(0)
    ctx = K.Context()
    m, k = 128, 2032
    S = torch.randn(nb, m, k, generator=torch.Generator().manual_seed(1)).cuda()
    out = {"batch": nb, "m": m, "k": k}
    for path, name in ((1, "tensor_cores"), (2, "cuda_cores")):
        C = torch.zeros(nb, m, m, device="cuda")
        for _ in range(3):
            K.krr_gemm_f32_batched(ctx, S, S, C, tb=True, path=path)
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        for _ in range(5):
            K.krr_gemm_f32_batched(ctx, S, S, C, tb=True, path=path)
        e1.record(ctx.stream)
        ctx.sync()
        ms = e0.elapsed_time(e1) / 5
        out[name] = {"ms": ms, "tflops": 2.0 * nb * m * m * k / ms / 1e9}
    print(json.dumps(out), flush=True)


def step_only(steps, warmup):
    """warmup + steps whole KRR steps of the benchmark workload (standardize,
    compress, factor, GMRES, predict) with nothing else around them, for
    launch lists under a profiler; prints the phase times of the last step."""
    import torch
    import paper_1803_10274_gb300 as K
    torch.cuda.set_device(0)
    ctx = K.Context()
    X, Xt, Y, yt = _inputs()
    Xd, Xtd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Xt).cuda(), torch.from_numpy(Y).cuda()
    o = K.default_options(h=WL["h"], lambda_=WL["lam"], eps_c=WL["eps_c"], leaf=WL["leaf"], precision=K.KRR_MIXED,
                          seed=WL["seed"], r0=WL["r0"])
    st = None
    for _ in range(warmup + steps):
        Xs, Xts = Xd.clone(), Xtd.clone()
        K.krr_standardize(ctx, Xs, Xts)
        H = K.hss_compress(ctx, Xs, o)
        H.factor()
        a, res = H.solve(Yd, tol=0.5 * 10 * WL["eps"], max_refine=200)
        H.predict(Xts, a[:, :1].contiguous())
        st = H.stats()
        H.close()
    ctx.sync()
    print(json.dumps({k: st[k] for k in ("t_cluster_ms", "t_compress_ms", "t_factor_ms", "t_solve_ms",
                                         "refine_steps")}), flush=True)


def sample_only(n, r, image=False):
    """Five launches of the fused sampling product on the benchmark's data
    distribution (d=8, standardized), or with image=True on MNIST-shaped
    rows (d=784, h=4: the streamed wide-row kernel), for kernel profiling."""
    import torch
    import paper_1803_10274_gb300 as K
    import synth
    torch.cuda.set_device(0)
    ctx = K.Context()
    if image:
        X = synth.image_like(n, IMAGE_WL["seed"])[0].astype(np.float32)
        h = IMAGE_WL["h"]
    else:
        X = synth.mixture(n, WL["d"], WL["comps"], WL["sigma"], WL["seed"])[0]
        X = ((X - X.mean(0)) / X.std(0)).astype(np.float32)
        h = WL["h"]
    d = X.shape[1]
    Xd = torch.from_numpy(X).cuda()
    R = torch.from_numpy(np.random.default_rng(7).standard_normal((n, r)).astype(np.float16).astype(np.float32)).cuda()
    S = torch.empty(n, r, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(5):
        K.krr_sample(ctx, Xd, Xd, h, 0.0, R, S=S)
    e1.record(ctx.stream)
    ctx.sync()
    ms = e0.elapsed_time(e1) / 5
    print(json.dumps({"n": n, "d": d, "r": r, "ms": ms, "tflops": 2.0 * n * n * (d + r) / ms / 1e9}), flush=True)


def cpu_baseline(X):
    """The FP64 oracle's dense KRR (kernel matrix + Cholesky solve) on the
    first CPU_SAMPLE_N standardized points, extrapolated to n = 65536 (the
    kernel build scales as n^2, the factorization and solve as n^3)."""
    from oracle import kernel, prep, solve
    n0 = CPU_SAMPLE_N
    Z = prep.standardize(X[:n0].astype(np.float64))[0]
    y = np.random.default_rng(1).standard_normal((n0, WL["nrhs"]))
    t0 = time.perf_counter()
    Kd = kernel.kernel_matrix(Z, Z, WL["h"])
    t1 = time.perf_counter()
    Kd[np.diag_indices(n0)] += WL["lam"]
    solve.spd_solve(Kd, y)
    t2 = time.perf_counter()
    s = WL["n"] / n0
    est = (t1 - t0) * s * s + (t2 - t1) * s ** 3
    return {"value": est, "unit": "s", "cores": int(kernel.num_threads()), "kind": "oracle",
            "timed_n": n0, "timed_seconds": t2 - t0, "extrapolated_to_n": WL["n"],
            "sample": "dense FP64 KRR (C kernel build + LAPACK Cholesky solve, 10 RHS) at n=%d, measured %.2f s, "
                      "extrapolated to n=65536 (build x%.0f, factor/solve x%.0f)" % (n0, t2 - t0, s * s, s ** 3)}


def measure_peaks():
    """Denominators besides MEASURED_PEAKS.json's copy and bf16 matmul:
    the library's pipe probes (FP32 and FP64 FMA, SFU ex2, FP32 -> FP16
    conversion) and torch matmuls measured the same way as the bf16 peak
    (best of 10, CUDA events): FP32 with TF32 tensor cores at 8192^3 and
    FP64 at 4096^3."""
    import torch
    import paper_1803_10274_gb300 as K
    torch.cuda.set_device(0)
    ctx = K.Context()
    out = {"fp32_fma_tflops": ctx.probe_rate(0) / 1e12, "fp64_fma_tflops": ctx.probe_rate(1) / 1e12,
           "ex2_per_s": ctx.probe_rate(2), "f32_to_f16_per_s": ctx.probe_rate(3)}

    def mm(dt, nn, tf32):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(nn, nn, device="cuda", dtype=dt)
        b = torch.randn(nn, nn, device="cuda", dtype=dt)
        for _ in range(3):
            a @ b
        best = 1e30
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        torch.backends.cuda.matmul.allow_tf32 = False
        return 2.0 * nn ** 3 / best / 1e12

    out["tf32_matmul_tflops"] = mm(torch.float32, 8192, True)
    out["fp64_matmul_tflops"] = mm(torch.float64, 4096, False)
    return out


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    X, Xt, Y, yt = _inputs()
    for _ in range(args.warmup):
        cpu_baseline(X)
    vals = [cpu_baseline(X) for _ in range(args.steps)]
    v = sum(c["value"] for c in vals) / len(vals)
    cb = dict(vals[-1])
    cb["value"] = v
    out = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * v, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic (seeded Gaussian mixture, SUSY-shaped)", "impl": "reference",
           "config": {"workload": WORKLOAD, "parallelism": "host cores"},
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the FP64 plain comparator")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the gradient workload and the million-point product")
    ap.add_argument("--image", action="store_true", help="with --sample-only: MNIST-shaped rows (d=784)")
    ap.add_argument("--batch-only", action="store_true", help="only run the MNIST-shaped and batched-problems workloads")
    ap.add_argument("--image-only", action="store_true", help="only run the MNIST-shaped workload (for profilers)")
    ap.add_argument("--orderings-only", action="store_true", help="only run the comparison of the orderings")
    ap.add_argument("--gemm-only", type=int, metavar="NB",
                    help="only run NB batched 128 x 128 x 2032 Gram products on both GEMM paths (for profilers)")
    ap.add_argument("--solve-only", nargs="?", type=int, const=0, default=None, metavar="N",
                    help="only compress, factor and run single ULV solves (for profilers)")
    ap.add_argument("--step-only", action="store_true",
                    help="only run --warmup + --steps KRR steps, nothing else (for launch lists)")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the arithmetic-pipe rates and the TF32 / FP64 matmul rates, then exit")
    ap.add_argument("--sample-only", nargs=2, type=int, metavar=("N", "R"),
                    help="only run the fused sampling product at n=N, r=R (5 launches; for profilers)")
    args = ap.parse_args()
    if args.sample_only:
        sample_only(*args.sample_only, image=args.image)
    elif args.image_only:
        import torch
        import paper_1803_10274_gb300 as K
        torch.cuda.set_device(0)
        ctx = K.Context()
        l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        print(json.dumps({"image_d784": bench_image(K, ctx, l2)}), flush=True)
    elif args.batch_only:
        import torch
        import paper_1803_10274_gb300 as K
        torch.cuda.set_device(0)
        ctx = K.Context()
        l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        print(json.dumps({"image_d784": bench_image(K, ctx, l2), "batch": bench_batch(K, ctx, l2)}), flush=True)
    elif args.solve_only is not None:
        solve_only(n=args.solve_only or None)
    elif args.gemm_only:
        gemm_only(args.gemm_only)
    elif args.step_only:
        step_only(args.steps, args.warmup)
    elif args.peaks:
        print(json.dumps(measure_peaks()), flush=True)
    elif args.orderings_only:
        import torch
        import paper_1803_10274_gb300 as K
        torch.cuda.set_device(0)
        ctx = K.Context()
        l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        print(json.dumps({"orderings": bench_orderings(K, ctx, l2)}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
