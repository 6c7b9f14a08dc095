#!/usr/bin/env python
"""Benchmark of the PB-SpGEMM hot path on GB300.

One step = the whole path on one product: symbolic (Alg. 3 flop + per-row
flop + bins, one host sync) then numeric (expand, sort, compress, ConvertCSR).
Default workload: ER C = A*A, n = 2^21, d = 8, FP64 values, int32 indices
(the large single product of the headline configuration).  Inputs are seeded
synthetic matrices resident in HBM; they and the tuple buffer (1.6 GB) are far
larger than L2, so no L2 flush is needed between steps.

Printed: one JSON line (rank 0).  `value` is whole-job GFLOPS counting
2 x multiplications; the `roofline` object reports the dominant kernel's
algorithmic GB/s against the measured HBM copy bandwidth.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload er21|er12|er22|batch1024|...]

With N > 1 (torchrun) every rank runs an independent replica (the path does
not shard onto several GPUs here); value = all ranks' flops / max rank time.
`--impl reference` times the CPU oracle on the host cores instead.
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

METRIC = "SpGEMM GFLOPS and HBM GB/s as % of β·AI roofline; served p50/p99 latency vs plain"
WORKLOADS = {
    "er21": dict(kind="er", n=1 << 21, d=8, seed=1, dtype="f64",
                 desc="ER C=A*A, n=2^21, d=8 per column, FP64 values U(-1,1), int32 indices"),
    "rmat20": dict(kind="rmat", scale=20, ef=16, seed=2, dtype="f64", budget=64 << 30, exact=True,
                   desc="R-MAT C=A*A, scale 20, edge factor 16, (0.57,0.19,0.19,0.05), dedup, FP64, row panels"),
    "rmat18": dict(kind="rmat", scale=18, ef=16, seed=2, dtype="f64",
                   desc="R-MAT C=A*A, scale 18, edge factor 16, (0.57,0.19,0.19,0.05), dedup, FP64"),
    "rmat16": dict(kind="rmat", scale=16, ef=16, seed=2, dtype="f64",
                   desc="R-MAT C=A*A, scale 16, edge factor 16, (0.57,0.19,0.19,0.05), dedup, FP64"),
    "rmat20f32t": dict(kind="rmat", scale=20, ef=16, seed=2, dtype="f64_f32tuple", budget=64 << 30, exact=True,
                       desc="R-MAT C=A*A, scale 20, edge factor 16, (0.57,0.19,0.19,0.05), dedup, FP64 values, "
                            "FP32 tuples merged in FP64, row panels"),
    "er22": dict(kind="er", n=1 << 22, d=8, seed=4, dtype="f64",
                 desc="ER C=A*A, n=2^22, d=8 per column, FP64 values U(-1,1), int32 indices"),
    "rmat21f32t": dict(kind="rmat", scale=21, ef=16, seed=5, dtype="f64_f32tuple", budget=64 << 30, count_only=True,
                       desc="R-MAT C=A*A, scale 21, edge factor 16, (0.57,0.19,0.19,0.05), dedup, FP64 values, "
                            "FP32 tuples merged in FP64, row panels; counting run: every tuple phase (expand, hub-row "
                            "merge, bin sort and merge) runs, only C's entries are not written (C holds about 4e10 "
                            "entries, more than the device or a flop-sized buffer can hold)"),
    "er22f32t": dict(kind="er", n=1 << 22, d=8, seed=4, dtype="f64_f32tuple",
                     desc="ER C=A*A, n=2^22, d=8, FP64 values, FP32 tuples merged in FP64, int32 indices"),
    "er19": dict(kind="er", n=1 << 19, d=8, seed=7, dtype="f64",
                 desc="ER C=A*A, n=2^19, d=8 per column, FP64 values U(-1,1), int32 indices"),
    "er12": dict(kind="er", n=4096, d=4, seed=0, dtype="f64",
                 desc="ER C=A*A, n=4096, d=4 per column, FP64 values U(-1,1), int32 indices"),
    "serve": dict(kind="serve", grids=(32, 64, 96, 128), scales=(14, 15, 16, 17, 18, 19, 20), ef=16, seed=6,
                  budget=160 << 30, slots=4,
                  desc="Poisson-arrival request stream: AMG Galerkin P^T(A P) for the 3-D 7-point Poisson "
                       "matrix on 32^3..128^3 grids with 2x2x2 aggregation (FP64) mixed 1:1 with Markov-clustering "
                       "squarings M*M of column-stochastic R-MAT matrices, scales 14..20, edge factor 16 (FP32); "
                       "160 GiB HBM budget, 4 slots, operands resident"),
    "batch1024": dict(kind="batch", count=1024, seed=3, dtype="f64",
                      desc="1024 independent ER products A_i*A_i, n_i log-uniform in [512, 65536], d_i uniform "
                           "in {2..16}, FP64, one pb_spgemm_batch call per step replayed as a CUDA graph, "
                           "parameters autotuned per (n, d) class"),
}


def make_inputs(w):
    import synth
    if w["kind"] == "batch":
        shapes = synth.batch_er_shapes(w["count"], seed=w["seed"])
        return [synth.er(n, d, seed=1000 * w["seed"] + i) for i, (n, d) in enumerate(shapes)]
    if w["kind"] == "rmat":
        return synth.rmat(w["scale"], w["ef"], seed=w["seed"])
    return synth.er(w["n"], w["d"], seed=w["seed"])


def combine_replicas(local_ms: float, local_flop: int, device):
    """Whole-job figures of independent replicas (one per rank): the slowest
    rank's time and GFLOPS = 2 x all ranks' multiplications / that time.
    Without an initialised process group this is the single-rank figure."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    f = torch.tensor([float(local_flop)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(f, op=dist.ReduceOp.SUM)
    total_ms = float(t.item())
    return total_ms, 2.0 * float(f.item()) / (total_ms / 1e3) / 1e9


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def stored_traffic(kernel: str, w, flop: int):
    """DRAM bytes per launch of `kernel` on an ER FP64 workload: the per-tuple
    traffic of the committed ncu capture (profiles/traffic.json) times this
    workload's multiplications, while the kernel source is unchanged; else None."""
    if w.get("kind") != "er" or w.get("dtype") != "f64":
        return None
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        import hashlib
        ent = json.load(open(p)).get(kernel)
        if not ent:
            return None
        src = open(os.path.join(ROOT, "paper_2002_11302_gb300", "csrc", ent["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != ent["source_sha"]:
            return None  # kernel changed since the counters were taken
        return float(ent["dram_bytes_per_tuple"]) * flop
    except Exception:  # noqa: BLE001
        return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        os.unlink(self.out.name)
        sms, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sms.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def oracle_rows_for_budget(A, B, budget_s: float):
    """Leading rows whose oracle product takes about budget_s seconds (cost model
    t(rows) = t_fixed + c * flop(rows), from a 1-row call and a 1/16 sample)."""
    import oracle
    rf = oracle.row_flop(A, B)
    t0 = time.perf_counter()
    oracle.spgemm(A, B, np.zeros(1, np.int64))
    t_fixed = time.perf_counter() - t0
    probe = max(2, A.nrows // 16)
    t0 = time.perf_counter()
    oracle.spgemm(A, B, np.arange(probe, dtype=np.int64))
    c = max(time.perf_counter() - t0 - t_fixed, 1e-9) / max(int(rf[:probe].sum()), 1)
    cum = np.cumsum(rf)
    want = max((budget_s - t_fixed) / c, 1.0)
    nrows = int(min(A.nrows, max(np.searchsorted(cum, want) + 1, A.nrows // 256, 1)))
    return np.arange(nrows, dtype=np.int64), int(rf[:nrows].sum())


def cpu_oracle_run(A, B, repeats: int, budget_s: float = 8.0):
    """Median time of the oracle on a bounded leading-row sample; returns (seconds, cores, flop, nrows)."""
    import oracle
    rows, flop = oracle_rows_for_budget(A, B, budget_s)
    ts = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        oracle.spgemm(A, B, rows if rows.shape[0] < A.nrows else None)
        ts.append(time.perf_counter() - t0)
    return statistics.median(ts), oracle.threads(), flop, rows.shape[0]


def run_reference(args, w):
    """The oracle on host cores: same workload, metric and unit (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    if w["kind"] == "batch":
        return run_reference_batch(args, w)
    if w["kind"] == "serve":
        return run_reference_serve(args, w)
    A, B = make_inputs(w)
    # Each step is a bounded sample: a contiguous block of rows sized so the
    # whole run (warm-up + timed steps) stays near two minutes of CPU time.
    rows, flop = oracle_rows_for_budget(A, B, 120.0 / (args.steps + args.warmup))
    nrows = rows.shape[0]
    for _ in range(args.warmup):
        oracle.spgemm(A, B, rows)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.spgemm(A, B, rows)
    dt = time.perf_counter() - t0
    value = 2.0 * flop * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["desc"], "flop": flop},
        "cpu_baseline": {"value": value, "unit": "GFLOPS", "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"rows 0..{nrows - 1} of {A.nrows} ({flop} of {oracle.flop(A, B)} "
                                   f"multiplications) per step, {args.steps} timed steps"},
        "e2e": {"value": value, "unit": "GFLOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_oracle_sample(probs, budget_s: float):
    """Leading products of a batch whose oracle products take about budget_s seconds."""
    import oracle
    t0 = time.perf_counter()
    n, flop = 0, 0
    while n < len(probs) and (time.perf_counter() - t0 < budget_s or n == 0):
        oracle.spgemm(*probs[n])
        flop += oracle.flop(*probs[n])
        n += 1
    return n, flop


def run_reference_batch(args, w):
    import oracle
    probs = make_inputs(w)
    n, flop = batch_oracle_sample(probs, 120.0 / (args.steps + args.warmup))
    for _ in range(args.warmup):
        for A, B in probs[:n]:
            oracle.spgemm(A, B)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for A, B in probs[:n]:
            oracle.spgemm(A, B)
    dt = time.perf_counter() - t0
    value = 2.0 * flop * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["desc"], "flop": flop},
        "cpu_baseline": {"value": value, "unit": "GFLOPS", "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"products 0..{n - 1} of {len(probs)} ({flop} multiplications) per step, "
                                   f"{args.steps} timed steps"},
        "e2e": {"value": value, "unit": "GFLOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours_batch(args, w):
    """Batched workload: one pb_spgemm_batch call (symbolic + numeric of every product) per step."""
    import torch
    import torch.distributed as dist

    from paper_2002_11302_gb300 import binding, model

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    probs = make_inputs(w)
    # inputs as views of six concatenated buffers (so the end-to-end run copies them in six transfers)
    pin = lambda parts, dt: torch.from_numpy(np.concatenate([np.asarray(x, dtype=dt) for x in parts])).pin_memory()  # noqa: E731
    fields = [("colptr", np.int32, 0), ("rowidx", np.int32, 0), ("val", np.float64, 0),
              ("rowptr", np.int32, 1), ("colidx", np.int32, 1), ("val", np.float64, 1)]
    host = [pin([getattr(pr[side], f) for pr in probs], dt) for f, dt, side in fields]
    dev = [h.to("cuda") for h in host]
    views = [[] for _ in fields]
    for j, (f, dt, side) in enumerate(fields):
        off = 0
        for pr in probs:
            n = getattr(pr[side], f).shape[0]
            views[j].append(dev[j][off:off + n])
            off += n
    As = [binding.CscMatrix(A.nrows, A.ncols, views[0][i], views[1][i], views[2][i]) for i, (A, _) in enumerate(probs)]
    Bs = [binding.CsrMatrix(B.nrows, B.ncols, views[3][i], views[4][i], views[5][i]) for i, (_, B) in enumerate(probs)]
    handle = binding.Handle()
    bt = binding.Batch(As, Bs, handle=handle)
    flop = int(bt.flop.sum())
    tune_s = None
    if not args.no_tune:
        t0 = time.perf_counter()
        bt.autotune(reps=2)
        tune_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        l0 = binding.kernel_launches()
        bt.run(stream=stream)
        launches_per_call = binding.kernel_launches() - l0
    torch.cuda.synchronize()
    if bt.status() != 0:
        raise RuntimeError(f"device status {bt.status()} in the batch warm-up")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        bt.run(stream=stream)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if bt.status() != 0:
        raise RuntimeError(f"device status {bt.status()} in the graph warm-up")
    nnz = bt.nnz.cpu().numpy()

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.2)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for _ in range(args.steps):
            graph.replay()
        t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = t_start.elapsed_time(t_end)
    if bt.status() != 0:
        raise RuntimeError(f"device status {bt.status()} in the timed region")
    total_ms, value = combine_replicas(total_ms, flop * args.steps, "cuda")
    ms_per_step = total_ms / args.steps

    # per-phase kernel times (plain launches with phase events, after the timed region)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    binding.set_phase_events(handle, ev)
    ph = {"symbolic": 0.0, "expand": 0.0, "sort_compress": 0.0}
    reps = 5
    with torch.cuda.stream(stream):
        for _ in range(reps):
            bt.run(stream=stream)
            ev[3].synchronize()
            ph["symbolic"] += ev[0].elapsed_time(ev[1]) / reps
            ph["expand"] += ev[1].elapsed_time(ev[2]) / reps
            ph["sort_compress"] += ev[2].elapsed_time(ev[3]) / reps
    binding.set_phase_events(handle, None)
    by = [model.bytes_alg(A.nrows, A.ncols, A.nnz, B.nnz, int(bt.flop[i]), int(nnz[i]), val_in=8, tuple_bytes=12,
                          val_out=8, rowptr_out=8) for i, (A, B) in enumerate(probs)]
    tot = {k: sum(getattr(b, k) for b in by) for k in ("expand", "sort", "compress", "numeric", "total")}
    hbm, peak_kind = measured_peaks()
    kern = {"expand": (tot["expand"], ph["expand"], "k_expand"),
            "sort_compress": (tot["sort"] + tot["compress"], ph["sort_compress"], "k_binsort")}
    dom = max(kern, key=lambda k: kern[k][1])
    bytes_dom, ms_dom, kname = kern[dom]
    achieved = bytes_dom / (ms_dom / 1e3) / 1e9
    numeric_ms = ph["expand"] + ph["sort_compress"]

    # the same products, one plain call each (symbolic + allocation + numeric per product)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for A, B in zip(As, Bs):
        binding.spgemm(A, B, handle=handle)
    torch.cuda.synchronize()
    plain_ms = (time.perf_counter() - t0) * 1e3

    line = {
        "metric": METRIC, "value": value, "unit": "GFLOPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "count": len(probs), "rows": int(sum(A.nrows for A, _ in probs)),
                   "nnz_a": int(sum(A.nnz for A, _ in probs)), "flop": flop, "nnz_c": int(nnz.sum()),
                   "tuple_bytes": 12, "autotune_s": tune_s, "tuning_classes": len(binding.get_tuning(handle)),
                   "l2": "no flush: the inputs and the tuple buffer each exceed the 129 MB L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": peak_kind, "traffic": None,
                     "alg_bytes_per_launch": bytes_dom, "ms_per_launch": ms_dom},
        "pct_beta_ai": {"numeric": tot["numeric"] / (numeric_ms / 1e3) / 1e9 / hbm,
                        "step": tot["total"] / (ms_per_step / 1e3) / 1e9 / hbm, "beta_gbs": hbm,
                        "beta_kind": peak_kind},
        "phases_ms": ph,
        "vs_plain_per_call": {"plain_ms": plain_ms, "plain_gflops": 2.0 * flop / (plain_ms / 1e3) / 1e9,
                              "speedup": plain_ms / ms_per_step},
        "gpu_launches": launches_per_call * args.steps,
        "clocks": clocks,
    }
    if not args.no_e2e:
        line["e2e"] = run_e2e_batch(args, probs, host, dev, bt, stream, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        n, sflop = batch_oracle_sample(probs, 8.0)
        t0 = time.perf_counter()
        for A, B in probs[:n]:
            oracle.spgemm(A, B)
        t = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 2.0 * sflop / t / 1e9, "unit": "GFLOPS", "cores": oracle.threads(),
                                "kind": "oracle", "sample": f"products 0..{n - 1} of {len(probs)} "
                                                            f"({sflop} of {flop} multiplications)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_e2e_batch(args, probs, host, dev, bt, stream, torch):
    """The batch through the public API with host buffers: H2D of all inputs and D2H of every C per step."""
    n = len(probs)
    hrow = [torch.empty(C.rowptr.numel(), dtype=torch.int64).pin_memory() for C in bt.C]
    hcol = [torch.empty(C.colidx.numel(), dtype=torch.int32).pin_memory() for C in bt.C]
    hval = [torch.empty(C.val.numel(), dtype=torch.float64).pin_memory() for C in bt.C]
    hnnz = torch.empty(n, dtype=torch.int64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host)

    def one():
        with torch.cuda.stream(stream):
            for d, h in zip(dev, host):
                d.copy_(h, non_blocking=True)
            bt.run(stream=stream)
            hnnz.copy_(bt.nnz[:n], non_blocking=True)
            for i, C in enumerate(bt.C):
                hrow[i].copy_(C.rowptr, non_blocking=True)
            stream.synchronize()
            d2h = 8 * n
            for i, C in enumerate(bt.C):
                k = int(hnnz[i])
                hcol[i][:k].copy_(C.colidx[:k], non_blocking=True)
                hval[i][:k].copy_(C.val[:k], non_blocking=True)
                d2h += 8 * C.rowptr.numel() + 12 * k
            return d2h

    for _ in range(3):
        one()
    torch.cuda.synchronize()
    steps = max(args.steps // 10, 3)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(steps):
        d2h = one()
    e.record(stream)
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / steps
    flop = int(bt.flop.sum())
    return {"value": 2.0 * flop / (ms / 1e3) / 1e9, "unit": "GFLOPS", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ms, "steps": steps}


def serve_pool(w):
    """Host operands of the serving mix: (kind, name, A CSC, B CSR, dtype name)."""
    import synth
    pool = []
    for N in w["grids"]:
        A = synth.poisson7(N)
        pool.append(("galerkin", f"amg{N}", synth.CSC(A.nrows, A.ncols, A.rowptr, A.colidx, A.val),
                     synth.aggregation_prolongator(N), "f64"))
    for sc in w["scales"]:
        Ac, _ = synth.rmat(sc, w["ef"], seed=w["seed"] + sc)
        Mc, Mr = synth.column_stochastic(Ac, dtype=np.float32)
        pool.append(("product", f"mcl{sc}", Mc, Mr, "f32"))
    return pool


def serve_schedule(n, rate, npool, seed):
    """n requests: pool index uniform, Poisson arrivals at `rate` per second (arrival offsets in s)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, npool, n), np.cumsum(rng.exponential(1.0 / rate, n))


def pct(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else None


def run_reference_serve(args, w):
    """The oracle serving the same request mix one request at a time on the host cores."""
    import oracle
    import synth
    pool = serve_pool(w)

    def run(i):
        kind, _, A, B, _ = pool[i]
        if kind == "galerkin":
            AP = oracle.spgemm(A, B)
            AP_csr = synth.CSR(A.nrows, B.ncols, AP.rowptr.astype(np.int32), AP.colidx, AP.val)
            oracle.spgemm(synth.transpose_csr_as_csc(B), AP_csr)
            return oracle.flop(A, B) + oracle.flop(synth.transpose_csr_as_csc(B), AP_csr)
        oracle.spgemm(A, B)
        return oracle.flop(A, B)

    # bounded sample: the smaller half of the pool (the largest requests take minutes on the host)
    small = [0, len(w["grids"])] if len(w["grids"]) else [0]
    for i in small:
        run(i)
    t0 = time.perf_counter()
    flop, lat = 0, []
    for _ in range(args.steps):
        for i in small:
            t1 = time.perf_counter()
            flop += run(i)
            lat.append((time.perf_counter() - t1) * 1e3)
    dt = time.perf_counter() - t0
    value = 2.0 * flop / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32", "data": "synthetic",
        "config": {"workload": w["desc"], "requests": [pool[i][1] for i in small]},
        "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99)},
        "cpu_baseline": {"value": value, "unit": "GFLOPS", "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"requests {[pool[i][1] for i in small]} back to back, {args.steps} times"},
        "e2e": {"value": value, "unit": "GFLOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours_serve(args, w):
    """Serving: Poisson arrivals at swept rates through pb_server; the same schedule through plain calls."""
    import threading

    import torch

    from paper_2002_11302_gb300 import binding

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    pool = serve_pool(w)
    dts = {"f64": binding.PB_F64, "f32": binding.PB_F32}
    tdt = {"f64": torch.float64, "f32": torch.float32}
    dev = [(kind, name, binding.csc_to_device(A, val_dtype=tdt[d]), binding.csr_to_device(B, val_dtype=tdt[d]),
            dts[d]) for kind, name, A, B, d in pool]
    handle = binding.Handle()
    # plain calls size their work like the server: row panels of at most half the budget,
    # and C sized by a counting run when a flop-sized C would not fit the budget
    cfg = binding.make_config(max_tuple_bytes=w["budget"] // 2)
    exact = []
    for kind, _, Ad, Bd, dt in dev:
        p = binding.symbolic(Ad, Bd, dtype=dt, config=cfg, handle=handle)
        vb = 8 if dt == binding.PB_F64 else 4
        exact.append(kind == "product" and p.workspace_bytes + p.flop * (4 + vb) + 8 * (Ad.nrows + 1) > w["budget"])
        del p

    def plain(i):
        kind, _, Ad, Bd, dt = dev[i]
        if kind == "galerkin":
            AP = binding.spgemm(Ad, Bd, dtype=dt, config=cfg, rowptr64=False, handle=handle)
            PT = binding.CscMatrix(Bd.ncols, Bd.nrows, Bd.rowptr, Bd.colidx, Bd.val)
            return binding.spgemm(PT, AP, dtype=dt, config=cfg, handle=handle)
        if exact[i]:
            return binding.spgemm_exact(Ad, Bd, dtype=dt, config=cfg, handle=handle)[0]
        return binding.spgemm(Ad, Bd, dtype=dt, config=cfg, handle=handle)

    # flop of every request kind (both products of a Galerkin request) and its plain service time
    flops, service = [], []
    for i, (kind, _, Ad, Bd, dt) in enumerate(dev):
        plain(i)
        torch.cuda.synchronize()
        if kind == "galerkin":
            f1 = binding.symbolic(Ad, Bd, dtype=dt, handle=handle).flop
            AP = binding.spgemm(Ad, Bd, dtype=dt, rowptr64=False, handle=handle)
            PT = binding.CscMatrix(Bd.ncols, Bd.nrows, Bd.rowptr, Bd.colidx, Bd.val)
            flops.append(f1 + binding.symbolic(PT, AP, dtype=dt, handle=handle).flop)
        else:
            flops.append(binding.symbolic(Ad, Bd, dtype=dt, handle=handle).flop)
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            plain(i)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        service.append(statistics.median(ts))
    mean_service = float(np.mean(service))
    n_req = args.steps

    def run_plain(kinds, arrivals):
        lat = []
        t0 = time.perf_counter()
        for i, a in zip(kinds, arrivals):
            now = time.perf_counter() - t0
            if a > now:
                time.sleep(a - now)
            plain(int(i))
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - t0 - a) * 1e3)
        return lat, time.perf_counter() - t0

    def run_served(kinds, arrivals, e2e=False):
        torch.cuda.synchronize()
        torch.cuda.empty_cache()  # the plain path's cached blocks must not crowd the server's budget
        srv = binding.Server(w["budget"], max_slots=w["slots"], handle=handle)
        ids = [None] * len(kinds)
        stats = {"d2h": 0, "h2d": 0}
        host = {}
        if e2e:  # pinned host copies of every operand: each request uploads its own
            for i, (kind, name, A, B, d) in enumerate(pool):
                host[i] = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
                           for x in (A.colptr, A.rowidx, A.val, B.rowptr, B.colidx, B.val)]
        up = torch.cuda.Stream()
        t0 = time.perf_counter()
        failed = threading.Event()

        def submitter():
            for j, (i, a) in enumerate(zip(kinds, arrivals)):
                if failed.is_set():
                    return
                now = time.perf_counter() - t0
                if a > now:
                    time.sleep(a - now)
                kind, _, Ad, Bd, dt = dev[int(i)]
                if e2e:
                    h = host[int(i)]
                    with torch.cuda.stream(up):
                        d = [x.to("cuda", non_blocking=True) for x in h]
                    up.synchronize()
                    stats["h2d"] += sum(x.numel() * x.element_size() for x in h)
                    Ad = binding.CscMatrix(Ad.nrows, Ad.ncols, d[0], d[1], d[2])
                    Bd = binding.CsrMatrix(Bd.nrows, Bd.ncols, d[3], d[4], d[5])
                ids[j] = srv.submit_galerkin(Ad, Bd, dt) if kind == "galerkin" else srv.submit_product(Ad, Bd, dt)

        th = threading.Thread(target=submitter, daemon=True)
        th.start()
        lat, pending, done_n = [], set(range(len(kinds))), 0
        while pending:
            for j in list(pending):
                if ids[j] is None:
                    continue
                done, st = srv.poll(ids[j])
                if not done:
                    continue
                if st != 0:
                    failed.set()
                    th.join()
                    srv.close()
                    raise RuntimeError(f"request {j} failed with status {st}")
                lat.append(srv.timing(ids[j])[1])
                if e2e:
                    C = srv.result(ids[j], copy=False)
                    for x in (C.rowptr, C.colidx, C.val):
                        x.cpu()
                        stats["d2h"] += x.numel() * x.element_size()
                srv.release(ids[j])
                pending.discard(j)
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
        th.join()
        st = srv.stats()
        srv.close()
        return lat, wall, st, stats

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    launches0 = binding.kernel_launches()
    rates = [0.5 / mean_service, 1.0 / mean_service, 2.0 / mean_service]
    sweep = []
    for r_i, rate in enumerate(rates):
        kinds, arrivals = serve_schedule(n_req, rate, len(pool), w["seed"] + r_i)
        fl = float(sum(flops[int(i)] for i in kinds))
        lat_s, wall_s, st, _ = run_served(kinds, arrivals)
        lat_p, wall_p = run_plain(kinds, arrivals)
        print(f"rate {rate:.2f}/s: served p50 {pct(lat_s, 50):.1f} p99 {pct(lat_s, 99):.1f} ms "
              f"{n_req / wall_s:.2f} rps; plain p50 {pct(lat_p, 50):.1f} p99 {pct(lat_p, 99):.1f} ms "
              f"{n_req / wall_p:.2f} rps", file=sys.stderr, flush=True)
        sweep.append({"rate_rps": rate,
                      "served": {"p50_ms": pct(lat_s, 50), "p99_ms": pct(lat_s, 99), "rps": n_req / wall_s,
                                 "gflops": 2.0 * fl / wall_s / 1e9, "peak_gb": st["peak_bytes"] / 1e9,
                                 "preempted": st["preempted"]},
                      "plain": {"p50_ms": pct(lat_p, 50), "p99_ms": pct(lat_p, 99), "rps": n_req / wall_p,
                                "gflops": 2.0 * fl / wall_p / 1e9}})
    clocks = sampler.stop()
    launches = binding.kernel_launches() - launches0
    top = sweep[-1]
    kinds, arrivals = serve_schedule(n_req, rates[1], len(pool), w["seed"] + 7)
    fl = float(sum(flops[int(i)] for i in kinds))
    lat_e, wall_e, _, io = run_served(kinds, arrivals, e2e=True)
    line = {
        "metric": METRIC, "value": top["served"]["gflops"], "unit": "GFLOPS", "n_gpus": 1, "steps": n_req,
        "warmup": args.warmup, "ms_per_step": 1e3 / top["served"]["rps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (AMG) / f32 (MCL)", "data": "synthetic",
        "config": {"workload": w["desc"], "requests_per_rate": n_req, "budget_bytes": w["budget"],
                   "slots": w["slots"], "pool": [p[1] for p in pool], "flop": flops,
                   "plain_service_ms": [s * 1e3 for s in service],
                   "rates": "0.5x, 1x, 2x the plain path's capacity (1 / mean service time)",
                   "l2": "no flush: operands and tuple buffers of the large requests exceed the 129 MB L2",
                   "step": "one request; value = served throughput at the highest rate"},
        "serving": sweep,
        "latency_ms": {"served_p50": top["served"]["p50_ms"], "served_p99": top["served"]["p99_ms"],
                       "plain_p50": top["plain"]["p50_ms"], "plain_p99": top["plain"]["p99_ms"]},
        "roofline": None,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": {"value": 2.0 * fl / wall_e / 1e9, "unit": "GFLOPS", "h2d_bytes_per_step": io["h2d"] / n_req,
                "d2h_bytes_per_step": io["d2h"] / n_req, "p50_ms": pct(lat_e, 50), "p99_ms": pct(lat_e, 99),
                "rate_rps": rates[1]},
    }
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line), flush=True)


def run_ours(args, w):
    import torch
    import torch.distributed as dist

    from paper_2002_11302_gb300 import binding, model

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    A, B = make_inputs(w)
    Ad, Bd = binding.csc_to_device(A), binding.csr_to_device(B)
    handle = binding.Handle()
    stream = torch.cuda.current_stream()
    cfg = binding.make_config(bin_capacity=args.capacity, expand_chunk=args.chunk,
                              max_tuple_bytes=w.get("budget", 0), deterministic=args.deterministic)
    dt = {"f64": binding.PB_F64, "f64_f32tuple": binding.PB_F64_F32TUPLE}[w["dtype"]]
    plan = binding.symbolic(Ad, Bd, dtype=dt, config=cfg, handle=handle)
    flop = plan.flop
    ws = plan.workspace()
    cap = None
    count_only = bool(w.get("count_only"))
    cnt_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    if w.get("exact"):  # size C by a counting run (a flop-sized C would not fit)
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        binding.numeric_count(plan, Ad, Bd, ws, cnt)
        cap = int(cnt.item())
    C = None if count_only else binding.alloc_output(plan, rowptr64=True, cap=cap)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    binding.set_phase_events(handle, ev)

    def step(record=None):
        if record is not None:
            record[0].record(stream)
        p = binding.symbolic(Ad, Bd, dtype=dt, config=cfg, handle=handle)
        if record is not None:
            record[1].record(stream)
        if count_only:
            binding.numeric_count(p, Ad, Bd, ws, cnt_dev)
        else:
            binding.numeric(p, Ad, Bd, C, ws)
        if record is not None:
            record[2].record(stream)
        return p

    # warm-up (also checks the device status once)
    for _ in range(max(args.warmup, 3)):
        p = step()
    if p.status() != 0:
        raise RuntimeError("device-side error during warm-up")
    nnz_c = int(cnt_dev.item()) if count_only else int(C.rowptr[-1].item())

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.2)
    per_step = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    phase_ms = {"symbolic": 0.0, "reset": 0.0, "expand": 0.0, "sort_compress": 0.0}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = binding.kernel_launches()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        step(per_step[i])
        # phase events are overwritten every step: read them once the step is done
        ev[3].synchronize()
        phase_ms["reset"] += ev[0].elapsed_time(ev[1])
        phase_ms["expand"] += ev[1].elapsed_time(ev[2])
        phase_ms["sort_compress"] += ev[2].elapsed_time(ev[3])
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = binding.kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = t_start.elapsed_time(t_end)
    for i in range(args.steps):
        phase_ms["symbolic"] += per_step[i][0].elapsed_time(per_step[i][1])
    step_ms = [per_step[i][0].elapsed_time(per_step[i][2]) for i in range(args.steps)]
    total_ms, value = combine_replicas(total_ms, flop * args.steps, "cuda")
    ms_per_step = total_ms / args.steps

    # roofline of the dominant kernel (algorithmic bytes per launch / event-timed duration)
    tuple_bytes = 12 if dt == binding.PB_F64 else 8
    by = model.bytes_alg(A.nrows, A.ncols, A.nnz, B.nnz, flop, nnz_c, val_in=8, tuple_bytes=tuple_bytes,
                         val_out=8, rowptr_out=8)
    hbm, peak_kind = measured_peaks()
    c_write = by.compress if count_only else 0  # a counting run writes no entry of C
    kern = {"expand": (by.expand, phase_ms["expand"] / args.steps, "k_expand", "pb_expand.cu"),
            "sort_compress": (by.sort + by.compress - c_write, phase_ms["sort_compress"] / args.steps, "k_binsort",
                              "pb_binsort.cu")}
    dom = max(kern, key=lambda k: kern[k][1])
    bytes_dom, ms_dom, kname, _ = kern[dom]
    achieved = bytes_dom / (ms_dom / 1e3) / 1e9
    numeric_ms = (phase_ms["reset"] + phase_ms["expand"] + phase_ms["sort_compress"]) / args.steps
    pct_numeric = (by.numeric - c_write) / (numeric_ms / 1e3) / 1e9 / hbm
    pct_step = (by.total - c_write) / (ms_per_step / 1e3) / 1e9 / hbm

    line = {
        "metric": METRIC, "value": value, "unit": "GFLOPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if dt == binding.PB_F64 else "f64 (f32 tuples)", "data": "synthetic",
        "config": {"workload": w["desc"], "n": A.nrows, "nnz_a": A.nnz, "flop": flop, "nnz_c": nnz_c,
                   "npanels": plan.npanels, "tuple_bytes": tuple_bytes, "deterministic": args.deterministic,
                   "cf": flop / max(nnz_c, 1), "nbins": plan.nbins, "bin_capacity": args.capacity or 4096,
                   "counting_run": count_only,
                   "l2": "no flush: the inputs and the tuple buffer each exceed the 129 MB L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": peak_kind,
                     "traffic": None if args.deterministic else stored_traffic(kname, w, flop),
                     "alg_bytes_per_launch": bytes_dom, "ms_per_launch": ms_dom},
        "pct_beta_ai": {"numeric": pct_numeric, "step": pct_step, "beta_gbs": hbm, "beta_kind": peak_kind,
                        "ai_flop_per_byte": flop / by.total, "numeric_bytes": by.numeric, "step_bytes": by.total,
                        "numeric_vs_nominal_7900_gbs": by.numeric / (numeric_ms / 1e3) / 1e9 / 7900.0,
                        # Tab. III with b = 16 bytes per element, as the paper counts
                        "paper_b16_numeric": (16 * (A.nnz + B.nnz) + 32 * flop + 16 * nnz_c) / (numeric_ms / 1e3)
                        / 1e9 / hbm},
        "step_ms_stats": {"median": statistics.median(step_ms), "p10": float(np.percentile(step_ms, 10)),
                          "p90": float(np.percentile(step_ms, 90)), "steps": len(step_ms)},
        "phases_ms": {k: v / args.steps for k, v in phase_ms.items()},
        "gflops_numeric": 2.0 * flop / (numeric_ms / 1e3) / 1e9,
        "gpu_launches": launches,
        "clocks": clocks,
    }

    if dt == binding.PB_F64_F32TUPLE and rank == 0 and not count_only:
        line["accuracy"] = f32_tuple_accuracy(A, B, C, nnz_c)
    if args.compare_f32_tuples and rank == 0 and world == 1 and args.workload == "er21":
        del C, ws, plan
        torch.cuda.empty_cache()
        line["fp32_tuples_vs_fp64"] = compare_tuple_forms(args, torch, binding)
    if not args.no_e2e and not w.get("exact") and not count_only:
        line["e2e"] = run_e2e(args, A, B, handle, torch, binding, flop)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t, cores, sflop, srows = cpu_oracle_run(A, B, repeats=3)
        oracle.set_threads(1)
        t1, _, sflop1, srows1 = cpu_oracle_run(A, B, repeats=1, budget_s=4.0)
        oracle.set_threads(cores)
        line["cpu_baseline"] = {"value": 2.0 * sflop / t / 1e9, "unit": "GFLOPS", "cores": cores, "kind": "oracle",
                                "sample": f"rows 0..{srows - 1} of {A.nrows} ({sflop} of {flop} multiplications), "
                                          f"median of 3 runs",
                                "one_thread": {"value": 2.0 * sflop1 / t1 / 1e9, "unit": "GFLOPS",
                                               "sample": f"rows 0..{srows1 - 1} of {A.nrows}, one run"}}
    binding.set_phase_events(handle, None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def compare_tuple_forms(args, torch, binding):
    """The mixed-precision configuration (ER n=2^22, d=8): numeric phase with FP64
    tuples and with FP32 tuples merged in FP64, same inputs, same launch sequence
    (CUDA events; median of the steps)."""
    import synth
    A, B = synth.er(1 << 22, 8, seed=4)
    Ad, Bd = binding.csc_to_device(A), binding.csr_to_device(B)
    handle = binding.Handle()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    binding.set_phase_events(handle, ev)
    out = {"workload": "ER C=A*A, n=2^22, d=8, FP64 values", "steps": 5}
    for name, dt in (("fp64", binding.PB_F64), ("fp32_tuples", binding.PB_F64_F32TUPLE)):
        plan = binding.symbolic(Ad, Bd, dtype=dt, handle=handle)
        ws = plan.workspace()
        C = binding.alloc_output(plan, rowptr64=True)
        for _ in range(3):
            binding.numeric(plan, Ad, Bd, C, ws)
        torch.cuda.synchronize()
        ms = []
        for _ in range(5):
            binding.numeric(plan, Ad, Bd, C, ws)
            ev[3].synchronize()
            ms.append(ev[0].elapsed_time(ev[3]))
        if plan.status() != 0:
            raise RuntimeError(f"device status {plan.status()} in the {name} comparison")
        t = statistics.median(ms)
        out[name] = {"numeric_ms": t, "gflops_numeric": 2.0 * plan.flop / (t / 1e3) / 1e9}
        del C, ws, plan
        torch.cuda.empty_cache()
    out["fp32_tuples_speedup"] = out["fp64"]["numeric_ms"] / out["fp32_tuples"]["numeric_ms"]
    binding.set_phase_events(handle, None)
    return out


def f32_tuple_accuracy(A, B, C, nnz_c, budget_s: float = 3.0):
    """Error of the FP32-tuple result against the FP64 oracle on a leading-row sample:
    structure must be identical; values are reported as the largest relative error and
    the largest error as a fraction of the bound 64 * 2^-24 * sum |a b|."""
    import oracle
    rows, _ = oracle_rows_for_budget(A, B, budget_s)
    ref = oracle.spgemm(A, B, rows)
    rp = C.rowptr.cpu().numpy()
    last = int(rows[-1]) + 1
    ci = C.colidx[: int(rp[last])].cpu().numpy()
    va = C.val[: int(rp[last])].double().cpu().numpy()
    same = np.array_equal(rp[: last + 1] - rp[0], ref.rowptr) and np.array_equal(ci, ref.colidx)
    err = np.abs(va - ref.val)
    rel = err / np.maximum(np.abs(ref.val), 1e-300)
    bound = 64 * 2.0 ** -24 * ref.absval
    return {"rows_sampled": int(last), "structure_identical": bool(same), "max_rel_err": float(rel.max(initial=0)),
            "median_rel_err": float(np.median(rel)) if rel.size else 0.0,
            "max_err_over_bound": float((err / np.maximum(bound, 1e-300)).max(initial=0)),
            "reference": "FP64 oracle (Gustavson, ascending k)"}


def run_e2e(args, A, B, handle, torch, binding, flop: int):
    """Same metric through pb_spgemm_host: A and B from pinned host memory, C back to
    pinned host memory; every copy is inside the timed call."""
    hA, hB = binding.host_tensors(A), binding.host_tensors(B)
    C = binding.CsrMatrix(A.nrows, B.ncols, torch.empty(A.nrows + 1, dtype=torch.int64).pin_memory(),
                          torch.empty(max(flop, 1), dtype=torch.int32).pin_memory(),
                          torch.empty(max(flop, 1), dtype=torch.float64).pin_memory())
    h2d = sum(t.numel() * t.element_size() for M in (hA, hB) for t in (M.colidx if hasattr(M, "colidx") else M.rowidx,
                                                                      M.val, M.rowptr if hasattr(M, "rowptr") else M.colptr))
    stream = torch.cuda.current_stream()

    def one():
        nnz, st = binding.spgemm_host(hA, hB, C, handle=handle)
        if st != 0:
            raise RuntimeError(f"device status {st} in the end-to-end run")
        return nnz

    for _ in range(max(args.warmup, 3)):
        one()
    torch.cuda.synchronize()
    steps = max(args.steps // 10, 5)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(steps):
        nnz = one()
    e.record(stream)
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / steps
    d2h = 8 * (A.nrows + 1) + 12 * nnz
    return {"value": 2.0 * flop / (ms / 1e3) / 1e9, "unit": "GFLOPS", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ms, "steps": steps,
            "api": "pb_spgemm_host (copies overlapped with the kernels: values during symbolic, C by row panel)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="er21")
    ap.add_argument("--capacity", type=int, default=0, help="tuples per on-chip bin (2048/4096/8192; 0 = default)")
    ap.add_argument("--chunk", type=int, default=0, help="tuples per expand work item (0 = default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="batch workload: skip the autotuner")
    ap.add_argument("--no-compare", dest="compare_f32_tuples", action="store_false",
                    help="default workload: skip the FP32-tuple vs FP64 comparison at ER n=2^22")
    ap.add_argument("--deterministic", action="store_true",
                    help="single products: fixed tuple positions, bitwise-reproducible values")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
    elif w["kind"] == "batch":
        run_ours_batch(args, w)
    elif w["kind"] == "serve":
        run_ours_serve(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
