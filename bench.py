#!/usr/bin/env python3
"""blockBP sweep benchmark on GB300 (one process per GPU; replicas across GPUs).

One step = one synchronous blockBP sweep (Eq. 1): every directed block message of
the lattice recomputed by the zip-up bMPS fits, normalised, and the fixed-point
residual reduced.  Default workload: the 12x12 PEPS, d=2, D=3, near-product
tensors, 3x3-site blocks (16 blocks, 48 messages), chi=32, FP32-level contractions on
TF32 tensor cores (split operands) with FP64 QR/LQ, fit tol 1e-6 / 10 sweeps, residual
target 1e-8.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec tf32x3|tf32|bf16|fp64]
  python bench.py --impl reference      # the FP64 CPU oracle, same workload
  python bench.py --serve [--requests N] # served mix: Poisson arrivals of whole solves

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import ctypes as C
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

METRIC = "blockBP sweeps/s + TFLOP/s vs FP64 GPU path at stated <O> error; p50/p99 latency"
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25   # dense nominal ratio (recipe table)
# FP64 ALU peak: 2 DFMA per cycle per SM (ncu peak_sustained of the DFMA counter) x 2 flop
# x SMs x max SM clock; 152 SMs at 2070 MHz gives 1.26 TFLOP/s (recipe nominal: 1.25)
DFMA_PER_SM_CLK = 2
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# zip-up fit stop rule (App. A: std/|mean| of the sweep's losses): the paper's 1e-6; the
# library raises it to the loss noise of TF32 / BF16 contractions on those paths
FIT_TOL = {"fp64": 1e-6, "tf32": 1e-6, "bf16": 1e-6, "tf32x3": 1e-6}
WARM = 1  # each fit starts from its previous-sweep result (identical option in the oracle)


def workload(cfg_id):
    from paper_2301_05844_gb300 import inputs as I
    cfg = I.config(cfg_id)
    Lx, Ly = cfg["Lx"], cfg["Ly"]
    if cfg.get("single_layer"):
        # the magnetisation impurity on the 2x2 centre of the block
        bx = cfg["bx"]
        c0 = bx // 2 - 1
        return cfg, [[((c0 + i) * bx + c0 + j, cfg["impurity"])] for i in range(2) for j in range(2)]
    if cfg["boundary"] == "infinite":
        # 2-site terms on the 4 nearest-neighbour bonds of the 2x2 centre of the block:
        # sx sx, sy sy, sz sz each (the Heisenberg term is their sum / 4)
        bx = cfg["bx"]
        c0 = bx // 2 - 1
        ctr = [(c0 + i) * bx + c0 + j for i in range(2) for j in range(2)]
        bonds = [(ctr[0], ctr[1]), (ctr[2], ctr[3]), (ctr[0], ctr[2]), (ctr[1], ctr[3])]
        terms = [[(a, P), (b, P)] for a, b in bonds for P in (I.SIGMA_X, I.SIGMA_Y, I.SIGMA_Z)]
        return cfg, terms
    terms = [[(s, I.SIGMA_Z)] for s in range(Lx * Ly)] + [[(s, I.SIGMA_X)] for s in range(Lx * Ly)]
    return cfg, terms


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK), "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_lattice(B, cfg, prec, stream):
    dtype = {np.dtype(np.float64): B.F64, np.dtype(np.float32): B.F32, np.dtype(np.complex64): B.C64,
             np.dtype(np.complex128): B.C128}[np.asarray(cfg["tensors"][0]).dtype]
    g = B.Lattice(Lx=cfg["Lx"], Ly=cfg["Ly"], d=cfg["d"], D=cfg["D"], bx=cfg["bx"], by=cfg["by"], chi=cfg["chi"],
                  boundary=cfg["boundary"], dtype=dtype, prec=prec, tol=cfg.get("tol", 1e-8), max_sweeps=50,
                  fit_tol=FIT_TOL[prec], fit_max_sweeps=10, seed=1, warm_start=WARM, stream=stream,
                  single_layer=cfg.get("single_layer", 0))
    return g


def oracle_sample(cfg, seconds, warmup=3):
    """The FP64 oracle as it stands: warm-up sweeps, then sweeps until `seconds` pass."""
    from oracle import blockbp as ob
    o = ob.Lattice(cfg["Lx"], cfg["Ly"], cfg["d"], cfg["D"], cfg["bx"], cfg["by"],
                   [np.asarray(t) for t in cfg["tensors"]], boundary=cfg["boundary"], chi=cfg["chi"],
                   fit_tol=1e-6, fit_max_sweeps=10, seed=1, warm_start=bool(WARM),
                   single_layer=bool(cfg.get("single_layer", 0)))
    for _ in range(warmup):
        o.sweep()
    t0 = time.perf_counter()
    n = 0
    while True:
        o.sweep()
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return n, dt


def run_reference(args):
    """The oracle as it stands on the host cores, same workload, same step definition."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import blockbp as ob
    cfg, _ = workload(args.config)
    o = ob.Lattice(cfg["Lx"], cfg["Ly"], cfg["d"], cfg["D"], cfg["bx"], cfg["by"],
                   [np.asarray(t) for t in cfg["tensors"]], boundary=cfg["boundary"], chi=cfg["chi"],
                   fit_tol=1e-6, fit_max_sweeps=10, seed=1, warm_start=bool(WARM),
                   single_layer=bool(cfg.get("single_layer", 0)))
    for _ in range(args.warmup):
        o.sweep()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.sweep()
    dt = time.perf_counter() - t0
    v = args.steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "sweeps/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": cfg["name"], "lattice": f"{cfg['Lx']}x{cfg['Ly']}", "D": cfg["D"],
                      "chi": cfg["chi"], "block": f"{cfg['bx']}x{cfg['by']}"},
           "cpu_baseline": {"value": v, "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"{args.steps} sweeps after {args.warmup} warm-up sweeps"},
           "e2e": {"value": v, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args):
    import torch
    from paper_2301_05844_gb300 import binding as B
    from paper_2301_05844_gb300 import replicas as R

    rank, local, world = R.rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MB > 129 MB L2
    cfg, terms = workload(args.config)
    prec = args.prec or cfg.get("prec", "tf32")

    g = make_lattice(B, cfg, prec, stream.cuda_stream)
    g.set_tensors(cfg["tensors"])
    tune = None
    if prec != "fp64" and not args.no_autotune:
        tb, ta, tk = g.autotune(3)
        tune = {"ms_per_sweep_default_tiles": round(tb, 4), "ms_per_sweep_tuned_tiles": round(ta, 4),
                "steps_retiled": tk}
    for _ in range(args.warmup):
        g.sweep(1)
    s0 = g.stats()
    step_ms = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        w0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
            g.sweep(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    s1 = g.stats()
    tmax = R.max_over_ranks(dev_s, device=dev)
    value = R.whole_job_rate(args.steps, world, tmax)
    flops = s1["flops"] - s0["flops"]
    qr_flops = s1["qr_flops"] - s0["qr_flops"]
    kernels = s1["kernels"] - s0["kernels"]
    # fit sweeps each column's zip-up fit loop ran (device counters), over the timed sweeps
    loops = s1["fits"] - s0["fits"]
    fit_sweeps = (s1["fit_sweeps"] - s0["fit_sweeps"]) / loops if loops > 0 else None
    vals = g.expect(terms) if not args.no_readout else None

    # kernel classes of one sweep (every fit stage active), replayed with events
    classes = {}
    for cls, name in ((0, "tcgen05_gemm"), (1, "fp64_contraction"), (2, "fp64_qr")):
        ms, n, f, by = C.c_double(), C.c_longlong(), C.c_double(), C.c_double()
        rc = B.lib().bbp_time_kernels(g.h, cls, 3, C.byref(ms), C.byref(n), C.byref(f), C.byref(by))
        if rc == 0 and n.value > 0:
            classes[name] = {"ms": ms.value, "launches": n.value, "flops": f.value, "bytes": by.value}
    pk, src = peaks()
    roofline = None
    if classes:
        dom = max(classes, key=lambda k: classes[k]["ms"])
        c = classes[dom]
        per_launch_s = c["ms"] / 1e3 / c["launches"]
        ach = c["flops"] / c["launches"] / per_launch_s / 1e12
        if dom == "tcgen05_gemm":
            base = pk["bf16_tflops"]
            peak = base if prec == "bf16" else base * NOMINAL_TF32_OVER_BF16
            bound, note = "tensor", f"of {src} bf16 burst" + ("" if prec == "bf16" else " x nominal tf32/bf16")
        else:
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            mhz = pk.get("sm_max_mhz", 2070.0)
            peak = DFMA_PER_SM_CLK * 2 * sms * mhz * 1e6 / 1e12
            bound, note = "alu", f"of derived FP64 DFMA peak ({DFMA_PER_SM_CLK} DFMA/clk/SM x {sms} SMs x {mhz:.0f} MHz)"
        roofline = {"bound": bound, "kernel": dom, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None, "peak_source": note,
                    "classes_ms_per_sweep": {k: round(v["ms"], 4) for k, v in classes.items()},
                    # TFLOP/s of each class over its replayed launches (split-TF32 GEMMs counted
                    # over 3K, their MMA work)
                    "classes_tflops": {k: round(v["flops"] / (v["ms"] / 1e3) / 1e12, 4) for k, v in classes.items()
                                       if v["ms"] > 0},
                    "classes_launches_per_sweep": {k: v["launches"] for k, v in classes.items()}}

    # the plain FP64 GPU path on the same workload, same number of sweeps
    fp64 = None
    if prec != "fp64" and not args.no_fp64:
        h = make_lattice(B, cfg, "fp64", stream.cuda_stream)
        h.set_tensors(cfg["tensors"])
        for _ in range(args.warmup):
            h.sweep(1)
        torch.cuda.synchronize()
        evs = []
        for k in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                a.record(stream)
            h.sweep(1)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        t64 = sum(a.elapsed_time(b) for a, b in evs) / 1e3
        v64 = h.expect(terms) if vals is not None else None
        fp64 = {"sweeps_per_s": args.steps / t64, "speedup": (args.steps / dev_s) / (args.steps / t64),
                "max_abs_dO": float(np.max(np.abs(vals - v64))) if vals is not None else None,
                "observables": len(terms) if vals is not None else 0}
        h.close()

    # end to end through the C ABI from host memory: upload, solve to tolerance, read out
    e2e = None
    if not args.no_e2e:
        host = [np.ascontiguousarray(t) for t in cfg["tensors"]]
        nbytes = sum(t.nbytes for t in host)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e = make_lattice(B, cfg, prec, stream.cuda_stream)
        e.set_tensors(host)
        r, k, _ = e.sweep(0)
        out = e.expect(terms)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": k / te, "unit": "sweeps/s", "h2d_bytes_per_step": nbytes / max(k, 1),
               "d2h_bytes_per_step": (8 * k + 16 * len(terms)) / max(k, 1), "sweeps_to_tol": k,
               "final_residual": r, "solve_s": te, "includes": "create+plan+graph capture, upload, sweeps, read-out"}
        e.close()

    cpu = None
    if rank == 0 and not args.no_cpu:
        n, dt = oracle_sample(cfg, args.cpu_seconds, min(3, args.warmup))
        cpu = {"value": n / dt, "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} oracle sweeps of the same workload after {min(3, args.warmup)} warm-up sweeps ({dt:.1f} s)"}

    lat = sorted(step_ms)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))]
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": {"tf32": "tf32+f64qr", "bf16": "bf16+f64qr",
                                                                "tf32x3": "3xtf32+f64qr", "fp64": "f64"}[prec],
               "data": "synthetic", "config": {"workload": cfg["name"], "lattice": f"{cfg['Lx']}x{cfg['Ly']}",
                                              "d": cfg["d"], "D": cfg["D"], "chi": cfg["chi"],
                                              "block": f"{cfg['bx']}x{cfg['by']}",
                                              "messages": 2 * ((cfg["Lx"] // cfg["bx"] - 1) * (cfg["Ly"] // cfg["by"]) + (cfg["Ly"] // cfg["by"] - 1) * (cfg["Lx"] // cfg["bx"])) if cfg["boundary"] == "obc" else 4,
                                              "network": "single-layer" if cfg.get("single_layer") else "double-layer",
                                              "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
               "tflops": flops / dev_s / 1e12, "fp64_qr_gflops": qr_flops / dev_s / 1e9,
               "gpu_launches": kernels, "fit_sweeps_per_column": fit_sweeps,
               "latency_ms": {"p50": p50, "p99": p99}, "wall_s": wall,
               "fp64_path": fp64, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
               "autotune": tune}
        print(json.dumps(out), flush=True)
    g.close()
    if dist:
        dist.destroy_process_group()


def serve_mix(n, seed):
    """Seeded mix of whole solves: L in {6,...,24} (square, OBC), block b in {2,3,4}
    dividing L, D in {2,...,5}, chi in {16,32,64}, tensors U[0,1] + 0.1 N(0,1),
    BF16 (residual tol 1e-5) or TF32 (tol 1e-6) contractions with FP64 truncation,
    at most 50 sweeps; read-out <sz> on every site."""
    from paper_2301_05844_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        L = int(rng.choice(np.arange(6, 25, 2)))
        b = int(rng.choice([x for x in (2, 3, 4) if L % x == 0]))
        D = int(rng.integers(2, 6))
        chi = int(rng.choice([16, 32, 64]))
        prec = "bf16" if rng.random() < 0.5 else "tf32"
        T = I.uniform_noise_peps(L, L, 2, D, seed=1000 + i)
        kw = dict(Lx=L, Ly=L, d=2, D=D, bx=b, by=b, chi=chi, prec=prec, tol=1e-5 if prec == "bf16" else 1e-6,
                  max_sweeps=50, fit_tol=1e-6, fit_max_sweeps=10, seed=i + 1, warm_start=WARM)
        reqs.append((T, [[(s, I.SIGMA_Z)] for s in range(L * L)], kw))
    return reqs


def run_serve(args):
    """Served mix: every request first solved alone (sequential capacity and the
    reference results), then all of them submitted to the request server with
    Poisson arrivals at 0.8x the sequential capacity."""
    import threading

    import torch
    from paper_2301_05844_gb300 import binding as B
    torch.cuda.set_device(0)
    reqs = serve_mix(args.requests, args.seed)
    # warm-up: module load and the first graph capture
    w = B.Lattice(**reqs[0][2])
    w.set_tensors(reqs[0][0])
    w.sweep(1)
    w.close()
    alone = []
    for T, terms, kw in reqs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = B.Lattice(**kw)
        g.set_tensors(T)
        r, k, _ = g.sweep(0)
        v = g.expect(terms)
        g.close()
        torch.cuda.synchronize()
        alone.append(dict(t=time.perf_counter() - t0, sweeps=k, values=v))
    solo_s = sum(a["t"] for a in alone)
    lam = 0.8 * len(reqs) / solo_s
    gaps = np.random.default_rng(args.seed + 1).exponential(1.0 / lam, len(reqs))
    arrivals = np.cumsum(gaps) - gaps[0]
    feet = [B.footprint(**kw) for _, _, kw in reqs]
    budget = int(args.serve_gb * (1 << 30))
    srv = B.Server(max_bytes=max(budget, max(feet)), max_active=args.max_active)
    ids = [None] * len(reqs)
    with Clocks(0) as clk:
        t0 = time.perf_counter()

        def submitter():
            for i, (T, terms, kw) in enumerate(reqs):
                dt = t0 + arrivals[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                ids[i] = srv.submit(T, terms, **kw)

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        outs = [srv.wait(i, timeout_s=3600.0) for i in ids]
        makespan = time.perf_counter() - t0
    st = srv.stats()
    # saturation: every request submitted at once (throughput with all slots busy)
    t1 = time.perf_counter()
    bids = [srv.submit(T, terms, **kw) for T, terms, kw in reqs]
    bouts = [srv.wait(i, timeout_s=3600.0) for i in bids]
    burst_s = time.perf_counter() - t1
    srv.close()
    bdiff = max(float(np.max(np.abs(o["values"] - a["values"]))) for o, a in zip(bouts, alone))
    lat = sorted(o["latency_s"] for o in outs)
    p = lambda q: lat[min(len(lat) - 1, int(q * len(lat)))]
    sweeps = sum(o["sweeps"] for o in outs)
    diffs = [float(np.max(np.abs(o["values"] - a["values"]))) for o, a in zip(outs, alone)]
    same_sweeps = all(o["sweeps"] == a["sweeps"] for o, a in zip(outs, alone))
    out = {"metric": "served blockBP mix: aggregate sweeps/s; p50/p99 solve latency", "value": sweeps / makespan,
           "unit": "sweeps/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
           "config": {"workload": "served mix", "requests": len(reqs), "seed": args.seed,
                      "L": sorted({kw["Lx"] for _, _, kw in reqs}), "D": sorted({kw["D"] for _, _, kw in reqs}),
                      "chi": sorted({kw["chi"] for _, _, kw in reqs}),
                      "block": sorted({kw["bx"] for _, _, kw in reqs}),
                      "prec": {p_: sum(kw["prec"] == p_ for _, _, kw in reqs) for p_ in ("bf16", "tf32")},
                      "arrivals": f"Poisson, rate 0.8 x sequential capacity = {lam:.3f} req/s",
                      "budget_gb": budget / (1 << 30), "max_active": args.max_active,
                      "largest_footprint_gb": max(feet) / 1e9},
           "latency_s": {"p50": p(0.5), "p99": p(0.99), "max": lat[-1]},
           "sequential": {"solve_s_total": solo_s, "sweeps_per_s": sum(a["sweeps"] for a in alone) / solo_s},
           "makespan_s": makespan, "sweeps": sweeps, "served_vs_sequential": (sweeps / makespan) /
           (sum(a["sweeps"] for a in alone) / solo_s),
           "alone_vs_mix": {"max_abs_dO": max(diffs), "same_sweeps": same_sweeps},
           "saturated": {"makespan_s": burst_s, "sweeps_per_s": sum(o["sweeps"] for o in bouts) / burst_s,
                         "vs_sequential": (sum(o["sweeps"] for o in bouts) / burst_s) /
                         (sum(a["sweeps"] for a in alone) / solo_s), "max_abs_dO_vs_alone": bdiff},
           "server_stats": st, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--prec", default=None, choices=[None, "fp64", "tf32", "bf16", "tf32x3"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-readout", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--serve", action="store_true")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--serve-gb", type=float, default=64.0)
    ap.add_argument("--max-active", type=int, default=16)
    args = ap.parse_args()
    if args.serve and args.impl == "ours":
        run_serve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
