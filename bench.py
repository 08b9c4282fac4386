#!/usr/bin/env python3
"""Benchmark of the SRCD sweep (Algorithm 1 over Algorithm 2) on GB300.

Metric: nnz*r coordinate updates per second. One step is one pass of the
whole hot path over the synthetic corpus: the F half (sumW, every column of
F by Algorithm 2), the W half (sumF, every row of W) and the Eq. 1 objective
for the convergence test, so U = 2 * nnz * r updates per step.

Default workload: the large document-like corpus (n = 100,000 words,
m = 1,000,000 documents, Zipf(1.1) topic laws over the vocabulary,
Dirichlet(0.1) topic weights, log-normal lengths with mean 150 tokens;
~126M nnz), r = 100, inputs resident in HBM and larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). Under torchrun each rank runs an independent
replica of the workload on its own GPU (weak scaling); the reported time is
the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "large": dict(n=100_000, m=1_000_000, K=100, desc="large document-like corpus: n=100,000 words, "
                  "m=1,000,000 docs, Zipf(1.1)/Dirichlet(0.1), lognormal mean 150 tokens"),
    "docs": dict(n=30_000, m=100_000, K=50, desc="document-like corpus: n=30,000 words, m=100,000 docs, "
                 "Zipf(1.1)/Dirichlet(0.1), lognormal mean 150 tokens"),
}
METRIC = "nnz*r coordinate updates/s per sweep"
UNIT = "updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large")
    ap.add_argument("--r", type=int, default=100)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--threads", type=int, default=0, help="host threads (0 = all cores)")
    ap.add_argument("--sample-div", type=int, default=16,
                    help="CPU legs run on the first m/sample_div documents")
    return ap.parse_args()


# --------------------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def algorithmic_bytes(nnz, units, r):
    """Bytes one half must move at least once: per nonzero its index and value
    (8 B) and the fixed factor's row (4r B); per unit its r-vector read and
    written (8r B) and its offset (8 B)."""
    return nnz * 8 + nnz * r * 4 + units * (8 * r + 8)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("sweep.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1604_04026_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload, r):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when the summary is absent or the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    entry = d.get("kernels", {}).get("%s/%s/r%d" % (workload, kernel, r))
    return None if entry is None else entry.get("dram_bytes_per_launch_full")


def make_corpus(args, threads):
    from paper_1604_04026_gb300 import synth
    w = WORKLOADS[args.workload]
    return synth.docs(w["n"], w["m"], w["K"], seed=args.seed, threads=threads)


def subsample(V, div):
    """The first m/div documents of V (all words), as its own CSC/CSR."""
    from paper_1604_04026_gb300 import synth
    m2 = max(1, V.m // div)
    nnz2 = int(V.colptr[m2])
    return synth.from_csc(V.n, m2, V.colptr[:m2 + 1].copy(), V.rowidx[:nnz2].copy(), V.val[:nnz2].copy())


def oracle_sweep_time(Vs, r, seed, threads, sweeps):
    """Wall time of `sweeps` FP64 oracle sweeps (F half + W half) on Vs."""
    import oracle
    from paper_1604_04026_gb300 import synth
    W = synth.uniform_init(r, Vs.n, seed, 0)
    F = synth.uniform_init(r, Vs.m, seed, 1)
    t0 = time.perf_counter()
    for s in range(sweeps):
        F, _ = oracle.half_F(Vs, W, F, seed, s, threads=threads)
        W, _ = oracle.half_W(Vs, W, F, seed, s, threads=threads)
    return time.perf_counter() - t0


def cpu_desc():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    threads = args.threads or os.cpu_count() or 1
    V = make_corpus(args, threads)
    Vs = subsample(V, args.sample_div)
    U = 2 * Vs.nnz * args.r
    for w in range(args.warmup):
        oracle_sweep_time(Vs, args.r, args.seed, threads, 1)
    t = oracle_sweep_time(Vs, args.r, args.seed, threads, args.steps)
    value = U * args.steps / t
    sample = "first %d of %d documents (%d nnz) of the workload, %d sweeps" % (Vs.m, V.m, Vs.nnz, args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "r": args.r, "nnz": V.nnz,
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu": cpu_desc()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import paper_1604_04026_gb300 as nk

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    threads = args.threads or os.cpu_count() or 1
    V = make_corpus(args, threads)
    r = args.r
    U = 2 * V.nnz * r

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    model = nk.NMFKL(V.n, V.m, r=r, seed=args.seed, device=local)
    model.set_data(V)
    model.init()
    plan = model.plan()
    sweep = 0
    for _ in range(args.warmup):
        model.step(sweep)
        sweep += 1
    model.counters(reset=True)
    model.kernel_times(reset=True)
    model.set_timing(True)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    kl = None
    for _ in range(args.steps):
        kl = model.step(sweep)
        sweep += 1
    ev1.record()
    barrier()
    clocks.stop()
    model.set_timing(False)
    ms = ev0.elapsed_time(ev1)
    if pg is not None:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    times = model.kernel_times(reset=True)
    counters = model.counters(reset=True)
    value = ws * U * args.steps / (ms / 1e3)

    # roofline of the dominant kernel family
    peak, peak_kind = measured_peak_hbm()
    fam = {}
    for b in plan:
        units = b["count"]
        e = fam.setdefault(b["kernel"], {"bytes": 0, "nnz": 0, "units": 0})
        e["bytes"] += algorithmic_bytes(b["nnz"], units, r)
        e["nnz"] += b["nnz"]
        e["units"] += units
    sweep_kernels = {k: v for k, v in times.items() if k.startswith("sweep_")}
    dom = max(sweep_kernels, key=lambda k: sweep_kernels[k][1])
    launches, dom_ms = sweep_kernels[dom]
    per_launch_ms = dom_ms / max(launches, 1)
    bytes_per_launch = fam[dom]["bytes"] / max(1, sum(1 for b in plan if b["kernel"] == dom))
    # each launch handles one (half, bucket); a family may run on both halves
    nlaunch_per_step = sum(1 for b in plan if b["kernel"] == dom)
    bytes_per_launch = fam[dom]["bytes"] / nlaunch_per_step
    achieved = bytes_per_launch / (per_launch_ms / 1e3) / 1e9
    step_bytes = sum(algorithmic_bytes(b["nnz"], b["count"], r) for b in plan)
    ms_step = ms / args.steps
    traffic = ncu_traffic(dom, args.workload, r)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)",
                "kernel_ms_per_launch": per_launch_ms,
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "whole_step": {"algorithmic_bytes": step_bytes,
                               "achieved": step_bytes / (ms_step / 1e3) / 1e9,
                               "frac": step_bytes / (ms_step / 1e3) / 1e9 / peak}}
    n_launch = sum(v[0] for v in times.values())

    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(args, V, nk, torch, local, barrier, pg)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        Vs = subsample(V, args.sample_div)
        t = oracle_sweep_time(Vs, r, args.seed, threads, 1)
        cpu = {"value": 2 * Vs.nnz * r / t, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "one FP64 oracle sweep on the first %d of %d documents (%d nnz)" % (Vs.m, V.m, Vs.nnz),
               "seconds": t, "cpu": cpu_desc()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "n": V.n, "m": V.m, "r": r,
                       "nnz": V.nnz, "updates_per_step": U, "l2": "inputs larger than L2 (no flush)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks.summary(),
            "gpu_launches": n_launch,
            "kl_after": kl,
            "counters": counters,
            "kernel_ms": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(times.items())},
        }
        print(json.dumps(line), flush=True)
    model.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


def e2e_run(args, V, nk, torch, local, barrier, pg):
    """The same metric through the public API from host memory: upload V from
    pinned host buffers, draw the start, run the K steps (each reads its
    objective back), and download W and F -- all inside the timed region."""
    pinned = {}
    for name in ("colptr", "rowidx", "val", "rowptr", "colidx", "rval"):
        pinned[name] = torch.from_numpy(getattr(V, name)).pin_memory()
    r = args.r
    barrier()
    t0 = time.perf_counter()
    m = nk.NMFKL(V.n, V.m, r=r, seed=args.seed, device=local)
    m.set_data(nnz=V.nnz, **pinned)
    m.init()
    for s in range(args.steps):
        m.step(s)
    W = m.get_W()
    F = m.get_F()
    barrier()
    dt = time.perf_counter() - t0
    if pg is not None:
        t = torch.tensor([dt], dtype=torch.float64, device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        dt = float(t.item())
    m.close()
    ws = pg.get_world_size() if pg is not None else 1
    h2d = sum(x.numel() * x.element_size() for x in pinned.values())
    d2h = W.nbytes + F.nbytes + 8 * args.steps
    return {"value": ws * 2 * V.nnz * r * args.steps / dt, "unit": UNIT,
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
            "seconds": dt, "scope": "one fit job: upload V, random start, K steps, download W and F"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
