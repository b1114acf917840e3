#!/usr/bin/env python3
"""blockBP sweep benchmark on GB300 (one process per GPU; replicas across GPUs).

One step = one synchronous blockBP sweep (Eq. 1): every directed block message of
the lattice recomputed by the zip-up bMPS fits, normalised, and the fixed-point
residual reduced.  Default workload: the 32x32 PEPS, d=2, D=5, tensors U[0,1] + 0.1 N(0,1)
in FP32, 4x4-site blocks (64 blocks, 224 messages), chi=96, split-precision contractions on
the tensor cores with FP64 QR/LQ, fit tol 1e-6 / 10 sweeps (App. A), warm-started fits.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config C] [--prec P]
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
FIT_TOL = {"fp64": 1e-6, "tf32": 1e-6, "bf16": 1e-6, "tf32x3": 1e-6, "bf16x3": 1e-6}
DTYPE = {"tf32": "tf32+f64qr", "bf16": "bf16+f64qr", "tf32x3": "3xtf32+f64qr", "bf16x3": "3xbf16+f64qr", "fp64": "f64"}
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


KEEP_FP64 = 0  # --keep-fp64: FP64 QR/LQ and read-out closings on the tensor-core paths too


def make_lattice(B, cfg, prec, stream, launch_mode=0):
    dtype = {np.dtype(np.float64): B.F64, np.dtype(np.float32): B.F32, np.dtype(np.complex64): B.C64,
             np.dtype(np.complex128): B.C128}[np.asarray(cfg["tensors"][0]).dtype]
    g = B.Lattice(Lx=cfg["Lx"], Ly=cfg["Ly"], d=cfg["d"], D=cfg["D"], bx=cfg["bx"], by=cfg["by"], chi=cfg["chi"],
                  boundary=cfg["boundary"], dtype=dtype, prec=prec, tol=cfg.get("tol", 1e-8), max_sweeps=50,
                  fit_tol=FIT_TOL[prec], fit_max_sweeps=10, seed=1, warm_start=WARM, stream=stream,
                  single_layer=cfg.get("single_layer", 0), launch_mode=launch_mode, keep_fp64=KEEP_FP64)
    return g


def oracle_lattice(cfg):
    from oracle import blockbp as ob
    return ob.Lattice(cfg["Lx"], cfg["Ly"], cfg["d"], cfg["D"], cfg["bx"], cfg["by"],
                      [np.asarray(t) for t in cfg["tensors"]], boundary=cfg["boundary"], chi=cfg["chi"],
                      fit_tol=1e-6, fit_max_sweeps=10, seed=1, warm_start=int(WARM),
                      single_layer=bool(cfg.get("single_layer", 0)))


def oracle_units(cfg):
    """Unit of the oracle's timed samples: whole sweeps where one takes seconds, else single
    messages (a sweep of the 224-message D=5 workload takes the oracle tens of minutes)."""
    return "message" if cfg["D"] >= 5 else "sweep"


def oracle_steps(o, unit, n=None, seconds=None):
    """Run the oracle as it stands for n units, or until `seconds` pass; returns (units, s).
    A message unit is one message of the current sweep, in order (Eq. 1 for one block and
    direction, from the previous sweep's messages)."""
    keys = sorted(o.msgs)
    t0 = time.perf_counter()
    k = 0
    while (n is not None and k < n) or (seconds is not None and time.perf_counter() - t0 < seconds):
        if unit == "sweep":
            o.sweep()
        else:
            bi, dr = keys[k % len(keys)]
            o.compute_message(bi, dr, o.msgs, o.sweeps_done)
        k += 1
    return k, time.perf_counter() - t0


def oracle_rate(cfg, o, unit, k, dt):
    """Sweeps per second from k units in dt seconds (a message unit counts 1/messages of a sweep)."""
    per_sweep = 1 if unit == "sweep" else len(o.msgs)
    return k / dt / per_sweep


def run_reference(args):
    """The oracle as it stands on the host cores, same workload and metric.  One step is one
    sweep, or, on the D=5 workload, one message of a sweep (a bounded sample of the sweep;
    the rate is scaled by the messages per sweep)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg, _ = workload(args.config)
    o = oracle_lattice(cfg)
    unit = oracle_units(cfg)
    oracle_steps(o, unit, n=args.warmup)
    k, dt = oracle_steps(o, unit, n=args.steps)
    v = oracle_rate(cfg, o, unit, k, dt)
    sample = (f"{args.steps} sweeps after {args.warmup} warm-up sweeps" if unit == "sweep" else
              f"{args.steps} messages of the first sweep after {args.warmup} warm-up messages "
              f"(random fit starts), scaled by the {len(o.msgs)} messages of a sweep")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "sweeps/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": cfg["name"], "lattice": f"{cfg['Lx']}x{cfg['Ly']}", "D": cfg["D"],
                      "chi": cfg["chi"], "block": f"{cfg['bx']}x{cfg['by']}", "step": unit},
           "cpu_baseline": {"value": v, "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def timed_sweeps(torch, g, stream, flush, steps):
    """steps sweeps, each bracketed by CUDA events on the library's stream, an L2 flush
    (a 256 MB write) before each outside the events; per-sweep milliseconds."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
        g.sweep(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def fit_sweeps_per_column(s0, s1):
    """Fit sweeps the zip-up fits ran per column fit between two stats snapshots (counted
    on the device)."""
    loops = s1["fits"] - s0["fits"]
    return (s1["fit_sweeps"] - s0["fit_sweeps"]) / loops if loops > 0 else None


def loop_iters_per_sweep(s0, s1):
    """Iterations the lockstep fit loops ran per message sweep (each loop runs until every fit
    of its group has met the stop rule; the fits that have skip their work)."""
    n = s1["sweeps"] - s0["sweeps"]
    return (s1["fit_loop_iters"] - s0["fit_loop_iters"]) / n if n > 0 else None


def kernel_roofline(B, g, prec, torch, dev):
    """Kernel-class replay of one sweep (every fit stage active, CUDA events on the library's
    stream, bbp_time_kernels); the roofline object of the dominant class."""
    classes = {}
    for cls, name in ((0, "tcgen05_gemm"), (1, "fp64_contraction"), (2, "fp64_qr")):
        ms, n, f, by = C.c_double(), C.c_longlong(), C.c_double(), C.c_double()
        rc = B.lib().bbp_time_kernels(g.h, cls, 3, C.byref(ms), C.byref(n), C.byref(f), C.byref(by))
        if rc == 0 and n.value > 0:
            classes[name] = {"ms": ms.value, "launches": n.value, "flops": f.value, "bytes": by.value}
    if not classes:
        return None
    pk, src = peaks()
    dom = max(classes, key=lambda k: classes[k]["ms"])
    c = classes[dom]
    per_launch_s = c["ms"] / 1e3 / c["launches"]
    ach = c["flops"] / c["launches"] / per_launch_s / 1e12
    if dom == "tcgen05_gemm":
        base = pk["bf16_tflops"]
        bf = prec in ("bf16", "bf16x3")
        peak = base if bf else base * NOMINAL_TF32_OVER_BF16
        bound, note = "tensor", f"of {src} bf16 burst" + ("" if bf else " x nominal tf32/bf16")
    else:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = pk.get("sm_max_mhz", 2070.0)
        peak = DFMA_PER_SM_CLK * 2 * sms * mhz * 1e6 / 1e12
        bound, note = "alu", f"of derived FP64 DFMA peak ({DFMA_PER_SM_CLK} DFMA/clk/SM x {sms} SMs x {mhz:.0f} MHz)"
    traffic = measured_traffic(dom, g, c["launches"])
    return {"bound": bound, "kernel": dom, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": traffic["bytes_per_launch"] if traffic else None,
            "traffic_source": traffic["source"] if traffic else "no ncu capture of the current kernel source",
            "algorithmic_bytes_per_launch": c["bytes"] / c["launches"], "peak_source": note,
            "classes_ms_per_sweep": {k: round(v["ms"], 4) for k, v in classes.items()},
            # TFLOP/s of each class over its replayed launches (split-operand GEMMs counted over
            # 3K, their MMA work)
            "classes_tflops": {k: round(v["flops"] / (v["ms"] / 1e3) / 1e12, 4) for k, v in classes.items()
                               if v["ms"] > 0},
            "classes_launches_per_sweep": {k: v["launches"] for k, v in classes.items()}}


def measured_traffic(cls, g, launches):
    """DRAM bytes per launch of a kernel class from the committed ncu summary of this workload
    (profiles/traffic.json: dram__bytes_read.sum + dram__bytes_write.sum over the class's
    launches of one replayed sweep, with the hash of the kernel source it was taken on).  None
    once that source has changed, or for another workload."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    e = rec.get(cls)
    if not e or e.get("workload") != g.workload_name:
        return None
    h = hashlib.sha256()
    for src in e["sources"]:
        with open(os.path.join(ROOT, src), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != e["source_sha16"]:
        return None
    return {"bytes_per_launch": e["dram_bytes_per_launch"], "source": e["profile"]}


def golden_error(B, cfg, prec, stream, torch):
    """<O> error against the stored oracle values of the workload's golden case (a smaller
    lattice at the same D, chi and block, run for the golden's fixed schedule): the chosen
    precision and the FP64 GPU path, max |d<O>| over the golden's observables."""
    from paper_2301_05844_gb300 import inputs as I
    name = cfg.get("golden")
    if not name:
        return None
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        gd = json.load(f)
    p = gd["params"]
    T = I.uniform_noise_peps(p["L"], p["L"], p["d"], p["D"], seed=p["seed"], dtype=np.float32)
    n = p["L"] * p["L"]
    terms = [[(s, I.SIGMA_Z)] for s in range(n)] + [[(s, I.SIGMA_X)] for s in range(n)]
    ref = np.array(gd["sz"] + gd["sx"])
    out = {"workload": f"peps{p['L']}x{p['L']}_D{p['D']}_chi{p['chi']}", "observables": 2 * n,
           "schedule": f"{p['sweeps']} sweeps, fit tol {p['fit_tol']} / {p['fit_max_sweeps']}, warm start",
           "max_abs_dO": {}}
    for pr in (prec, "fp64"):
        g = B.Lattice(Lx=p["L"], Ly=p["L"], d=p["d"], D=p["D"], bx=p["block"], by=p["block"], chi=p["chi"],
                      dtype=B.F32, prec=pr, fit_tol=p["fit_tol"], fit_max_sweeps=p["fit_max_sweeps"], seed=p["seed"],
                      warm_start=int(p["warm_start"]), stream=stream, keep_fp64=KEEP_FP64)
        g.set_tensors(T)
        g.sweep(p["sweeps"])
        v = g.expect(terms)
        out["max_abs_dO"][pr] = float(np.max(np.abs(v.real - ref)))
        g.close()
    torch.cuda.synchronize()
    return out


def run_replay(args):
    """For ncu captures: the configured workload (or the same recipe on an L x L lattice), one
    sweep (untimed: its graph has conditional nodes, which ncu does not profile kernel by
    kernel), then one kernel-class replay of each requested class (bbp_time_kernels: the
    sweep's launches of that class, one by one, every fit stage active)."""
    import torch
    from paper_2301_05844_gb300 import binding as B
    from paper_2301_05844_gb300 import inputs as I
    cfg, _ = workload(args.config)
    if args.lattice:
        assert cfg["boundary"] == "obc" and not cfg.get("single_layer"), "--lattice: OBC PEPS workloads only"
        L = args.lattice
        cfg = dict(cfg, Lx=L, Ly=L, name=f"peps{L}x{L}_D{cfg['D']}_chi{cfg['chi']}",
                   tensors=I.uniform_noise_peps(L, L, cfg["d"], cfg["D"], seed=args.config,
                                                dtype=np.asarray(cfg["tensors"][0]).dtype))
    prec = args.prec or cfg.get("prec", "tf32")
    torch.cuda.set_device(0)
    if args.replay == "readout":
        g = make_lattice(B, cfg, prec, None, launch_mode=1)
        g.set_tensors(cfg["tensors"])
        g.sweep(2)
        n = cfg["Lx"] * cfg["Ly"]
        terms = [[(s_, I.SIGMA_Z)] for s_ in range(n)] + [[(s_, I.SIGMA_X)] for s_ in range(n)]
        torch.cuda.synchronize()
        s0 = g.stats()
        torch.cuda.profiler.start()  # for `ncu --profile-from-start off`: the read-out's launches only
        t0 = time.perf_counter()
        g.expect(terms)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        t1 = time.perf_counter()
        s1 = g.stats()
        print(json.dumps({"workload": cfg["name"], "prec": prec, "readout_s": t1 - t0,
                          "observables": len(terms), "readout_gflop": (s1["flops"] - s0["flops"]) / 1e9,
                          "readout_kernels": s1["kernels"] - s0["kernels"]}), flush=True)
        g.close()
        return
    g = make_lattice(B, cfg, prec, None)
    g.set_tensors(cfg["tensors"])
    g.sweep(1)
    if args.replay == "steps":
        # every launch of the sweep timed on its own, with its work and the tile width
        rows = g.time_steps(reps=3)
        for r in rows:
            r["tflops"] = r["flops"] / max(r["ms"], 1e-9) / 1e9
            r["gbs"] = r["bytes"] / max(r["ms"], 1e-9) / 1e6
            print(json.dumps({"workload": cfg["name"], "prec": prec, **r}), flush=True)
        g.close()
        return
    for cls in [int(c) for c in args.replay.split(",")]:
        ms, n, f, by = C.c_double(), C.c_longlong(), C.c_double(), C.c_double()
        rc = B.lib().bbp_time_kernels(g.h, cls, 1, C.byref(ms), C.byref(n), C.byref(f), C.byref(by))
        print(json.dumps({"workload": cfg["name"], "prec": prec, "class": cls, "rc": rc, "ms": ms.value,
                          "launches": n.value, "flops": f.value, "bytes": by.value}), flush=True)
    g.close()


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
    big = cfg["D"] >= 5  # the 224-message D=5 workload: FP64 arm and read-outs sized down

    g = make_lattice(B, cfg, prec, stream.cuda_stream)
    g.workload_name = cfg["name"]
    g.set_tensors(cfg["tensors"])
    tune = None
    if prec != "fp64" and not args.no_autotune and not big:  # at D=5 it retiles for ~1% in ~2 min
        t0 = time.perf_counter()
        tb, ta, tk = g.autotune(3)
        tune = {"ms_per_sweep_default_tiles": round(tb, 4), "ms_per_sweep_tuned_tiles": round(ta, 4),
                "steps_retiled": tk, "seconds": round(time.perf_counter() - t0, 1)}
    # warm-up sweeps 1..W, timed one by one (sweep 2 is the FP64 arm's reference on the D=5 workload)
    warm_ms, warm_fit = [], []
    for _ in range(args.warmup):
        a = g.stats()
        warm_ms += timed_sweeps(torch, g, stream, flush, 1)
        warm_fit.append(fit_sweeps_per_column(a, g.stats()))
    s0 = g.stats()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        w0 = time.perf_counter()
        step_ms = timed_sweeps(torch, g, stream, flush, args.steps)
        wall = time.perf_counter() - w0
    if dist:
        dist.barrier()
    dev_s = sum(step_ms) / 1e3
    s1 = g.stats()
    tmax = R.max_over_ranks(dev_s, device=dev)
    value = R.whole_job_rate(args.steps, world, tmax)
    flops = s1["flops"] - s0["flops"]
    qr_flops = s1["qr_flops"] - s0["qr_flops"]
    kernels = s1["kernels"] - s0["kernels"]
    fit_cols = fit_sweeps_per_column(s0, s1)
    loop_iters = loop_iters_per_sweep(s0, s1)
    readout = None
    vals = None
    if not args.no_readout:
        t0 = time.perf_counter()
        vals = g.expect(terms)
        readout = {"observables": len(terms), "seconds": time.perf_counter() - t0}
    roofline = kernel_roofline(B, g, prec, torch, dev)

    # the plain FP64 GPU path on the same workload and stop rules.  On the D=5 workload (an
    # FP64 sweep takes over a minute) it times sweep 2 alone, against the same sweep of the
    # chosen path (timed during its warm-up): both start from the same messages and draws.
    fp64 = None
    if prec != "fp64" and not args.no_fp64:
        h = make_lattice(B, cfg, "fp64", stream.cuda_stream)
        h.set_tensors(cfg["tensors"])
        same = big and args.warmup >= 2
        w64 = 1 if same else args.warmup
        k64 = 1 if same else args.steps
        for _ in range(w64):
            h.sweep(1)
        torch.cuda.synchronize()
        t0 = h.stats()
        ms64 = timed_sweeps(torch, h, stream, flush, k64)
        t64 = sum(ms64) / 1e3
        t1 = h.stats()
        ref_s = warm_ms[1] / 1e3 if same else dev_s / args.steps * k64
        fp64 = {"sweeps_per_s": k64 / t64, "speedup": t64 / ref_s, "timed_sweeps": k64,
                "compared_sweeps": "sweep 2 of both paths" if same else f"sweeps {args.warmup + 1}-{args.warmup + k64}",
                "fit_sweeps_per_column": fit_sweeps_per_column(t0, t1),
                "fit_loop_iters_per_sweep": loop_iters_per_sweep(t0, t1),
                "tflops": (t1["flops"] - t0["flops"]) / t64 / 1e12}
        if same:
            fp64["chosen_path_sweep2"] = {"ms": warm_ms[1], "fit_sweeps_per_column": warm_fit[1]}
        if vals is not None and not big:
            v64 = h.expect(terms)
            fp64["max_abs_dO"] = float(np.max(np.abs(vals - v64)))
            fp64["observables"] = len(terms)
        h.close()

    oracle_err = golden_error(B, cfg, prec, stream.cuda_stream, torch) if not args.no_oracle_error else None

    # end to end through the C ABI: the tensors copied from pinned host memory, the solve run
    # to tolerance, the read-out copied back; the timed region holds all of it
    e2e = None
    if not args.no_e2e:
        flat = np.concatenate([np.ascontiguousarray(t).reshape(-1) for t in cfg["tensors"]])
        pinned = torch.empty(flat.nbytes, dtype=torch.uint8, pin_memory=True)
        pinned.numpy()[:] = flat.view(np.uint8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e = make_lattice(B, cfg, prec, stream.cuda_stream)
        e.set_tensors(host_ptr=pinned.data_ptr())
        r, k, _ = e.sweep(0)
        out = e.expect(terms) if not args.no_readout else None
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": k / te, "unit": "sweeps/s", "h2d_bytes_per_step": flat.nbytes / max(k, 1),
               "d2h_bytes_per_step": (8 * k + (16 * len(terms) if out is not None else 0)) / max(k, 1),
               "sweeps_to_tol": k, "final_residual": r, "solve_s": te, "host_memory": "pinned",
               "includes": "create+plan+graph capture, upload, sweeps to tolerance, read-out"}
        e.close()

    cpu = None
    if rank == 0 and not args.no_cpu:
        o = oracle_lattice(cfg)
        unit = oracle_units(cfg)
        k, dt = oracle_steps(o, unit, seconds=args.cpu_seconds)
        cpu = {"value": oracle_rate(cfg, o, unit, k, dt), "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": (f"{k} oracle sweeps of the same workload ({dt:.1f} s)" if unit == "sweep" else
                          f"{k} of the {len(o.msgs)} messages of the first oracle sweep of the same workload "
                          f"(random fit starts, {dt:.1f} s), scaled to sweeps")}

    served = None
    if rank == 0 and world == 1 and args.serve_requests > 0:
        r = run_serve(args, requests=args.serve_requests, emit=False)
        served = {k: r[k] for k in ("value", "unit", "latency_s", "alone_vs_mix", "sweeps", "makespan_s",
                                    "served_vs_sequential", "saturated")}
        served["config"] = {k: r["config"][k] for k in ("requests", "arrivals", "prec", "L", "D", "chi")}

    lat = sorted(step_ms)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))]
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec],
               "data": "synthetic", "config": {"workload": cfg["name"], "lattice": f"{cfg['Lx']}x{cfg['Ly']}",
                                              "d": cfg["d"], "D": cfg["D"], "chi": cfg["chi"],
                                              "block": f"{cfg['bx']}x{cfg['by']}",
                                              "messages": 2 * ((cfg["Lx"] // cfg["bx"] - 1) * (cfg["Ly"] // cfg["by"]) + (cfg["Ly"] // cfg["by"] - 1) * (cfg["Lx"] // cfg["bx"])) if cfg["boundary"] == "obc" else 4,
                                              "network": "single-layer" if cfg.get("single_layer") else "double-layer",
                                              "fit_tol": FIT_TOL[prec], "fit_max_sweeps": 10,
                                              "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
               "tflops": flops / dev_s / 1e12, "fp64_qr_gflops": qr_flops / dev_s / 1e9,
               "gpu_launches": kernels, "fit_sweeps_per_column": fit_cols, "fit_loop_iters_per_sweep": loop_iters,
               "latency_ms": {"p50": p50, "p99": p99}, "wall_s": wall,
               "fp64_path": fp64, "oracle_error": oracle_err, "readout": readout, "roofline": roofline,
               "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(), "autotune": tune,
               "served_mix": served}
        print(json.dumps(out), flush=True)
    g.close()
    if dist:
        dist.destroy_process_group()


def serve_mix(n, seed):
    """Seeded mix of whole solves: L in {6,...,24} (square, OBC), block b in {2,3,4}
    dividing L, D in {2,...,5}, chi in {16,32,64}, tensors U[0,1] + 0.1 N(0,1),
    split-BF16 (residual tol 1e-5) or split-TF32 (tol 1e-6) contractions with FP64
    truncation, at most 50 sweeps; read-out <sz> on every site."""
    from paper_2301_05844_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        L = int(rng.choice(np.arange(6, 25, 2)))
        b = int(rng.choice([x for x in (2, 3, 4) if L % x == 0]))
        D = int(rng.integers(2, 6))
        chi = int(rng.choice([16, 32, 64]))
        prec = "bf16x3" if rng.random() < 0.5 else "tf32x3"
        T = I.uniform_noise_peps(L, L, 2, D, seed=1000 + i)
        kw = dict(Lx=L, Ly=L, d=2, D=D, bx=b, by=b, chi=chi, prec=prec, tol=1e-5 if prec == "bf16x3" else 1e-6,
                  max_sweeps=50, fit_tol=1e-6, fit_max_sweeps=10, seed=i + 1, warm_start=WARM)
        reqs.append((T, [[(s, I.SIGMA_Z)] for s in range(L * L)], kw))
    return reqs


def run_serve(args, requests=None, emit=True):
    """Served mix: every request first solved alone (sequential capacity and the
    reference results), then all of them submitted to the request server with
    Poisson arrivals at 0.8x the sequential capacity.  emit=False returns the record
    instead of printing it (the compact mix of the default line)."""
    import threading

    import torch
    from paper_2301_05844_gb300 import binding as B
    torch.cuda.set_device(0)
    reqs = serve_mix(requests or args.requests, args.seed)
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
                      "prec": {p_: sum(kw["prec"] == p_ for _, _, kw in reqs) for p_ in ("bf16x3", "tf32x3")},
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
    if not emit:
        return out
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--prec", default=None, choices=[None, "fp64", "tf32", "bf16", "tf32x3", "bf16x3"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-readout", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-oracle-error", action="store_true")
    ap.add_argument("--warm-start", type=int, default=None, choices=[0, 1, 2],
                    help="fit warm start of the solve (default: the workload's; 2 also warm-starts the "
                         "read-out's environment columns)")
    ap.add_argument("--keep-fp64", action="store_true",
                    help="tensor-core paths: QR/LQ truncations and read-out closings in FP64 arithmetic (default FP32)")
    ap.add_argument("--serve", action="store_true")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="compact served mix added to the default line (0: none)")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--serve-gb", type=float, default=64.0)
    ap.add_argument("--max-active", type=int, default=16)
    ap.add_argument("--replay", default=None, help="kernel classes to replay once (for ncu), e.g. 0,2; 'readout': "
                                                   "one read-out of every site's <sz>, <sx> with every kernel launched on its own; "
                                                   "'steps': every launch of a sweep timed on its own (one JSON line each)")
    ap.add_argument("--lattice", type=int, default=0, help="with --replay: the workload's recipe on an L x L lattice")
    args = ap.parse_args()
    global KEEP_FP64, WARM
    KEEP_FP64 = int(args.keep_fp64)
    if args.warm_start is not None:
        WARM = args.warm_start
    if args.replay:
        run_replay(args)
    elif args.serve and args.impl == "ours":
        run_serve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
