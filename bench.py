"""Benchmark: SGD matrix entries/s of the block-wise adaptive SGD for NB GMF.

Workload (default): 20000 cells x 2000 genes of int32 NB counts (~85% zeros,
library-size offsets, per-gene NB sizes), d = 10, p = 3, q = 1, 500 x 500
blocks. One step = one epoch of Algorithm 1 = all 160 blocks (40 sweeps of
4 disjoint blocks), launched through the C ABI (gmf_sgd_epoch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32|mixed] [--workload nb_medium]

Prints one JSON line (rank 0). ``value`` = whole-job entries/s with Y resident
in HBM; ``e2e`` = the same metric through the public API with the counts
uploaded from pinned host memory each step and the deviance read back.
``--impl reference`` times the FP64 oracle on the host cores (a bounded
sample of the same workload per step).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "SGD matrix entries/s (NB GMF) and time-to-deviance within 1e-3 vs plain FP32"
UNIT = "entries/s"


def describe(w, precision):
    return {"workload": f"{w.name}: NB GMF {w.n}x{w.m} {w.y_dtype} counts (~{int(100 * (w.zero_frac or 0))}% zeros), "
                        f"d={w.d}, p={w.p}, q={w.q}, blocks {w.nb_row}x{w.nb_col}; step = one epoch "
                        f"({synth.n_sweeps(w.n, w.m, w.nb_row, w.nb_col)} sweeps, all blocks)",
            "n": w.n, "m": w.m, "d": w.d, "nb_row": w.nb_row, "nb_col": w.nb_col, "precision": precision,
            "l2": f"inputs larger than L2: Y is {w.n * w.m * (4 if w.y_dtype == 'int32' else 2) / 1e6:.0f} MB "
                  f"(L2 129 MB), every entry read once per step", "parallelism": "replicas"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_simt_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def sweep_algorithmic(w, K, fr, fc):
    """Algorithmic flops and HBM bytes of one sweep launch (all blocks of a sweep)."""
    per = min(-(-w.n // w.nb_row), -(-w.m // w.nb_col))
    entries = per * w.nb_row * w.nb_col
    flops_entry = 2 * K + 4 * fr + 4 * fc
    ybytes = 4 if w.y_dtype == "int32" else 2
    # counts once; parameters: L, R rows read; free columns + EMA (G, H) read and written
    pbytes = per * (w.nb_row * (4 * K + 24 * fr) + w.nb_col * (4 * K + 24 * fc))
    return entries, entries * flops_entry, entries * ybytes + pbytes


def cpu_baseline(w, prob, start, rp, cp, sigmas, budget_s=12.0):
    import oracle
    settings = synth.fit_settings()
    f = oracle.OracleFit(prob.Y, prob.X, prob.Z, prob.offset, start, family=w.family, nb_row=w.nb_row,
                         nb_col=w.nb_col, row_perm=rp, col_perm=cp, settings=settings)
    nsw = synth.n_sweeps(w.n, w.m, w.nb_row, w.nb_col)
    per = min(-(-w.n // w.nb_row), -(-w.m // w.nb_col))
    done = 0
    t0 = time.perf_counter()
    e = 0
    while time.perf_counter() - t0 < budget_s:
        chunk = 5
        w0 = done % nsw
        w1 = min(nsw, w0 + chunk)
        f.sweeps(sigmas[e % len(sigmas)], w0, w1)
        done += w1 - w0
        if w1 == nsw:
            e += 1
    el = time.perf_counter() - t0
    entries = done * per * w.nb_row * w.nb_col
    return {"value": entries / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} sweeps ({done * per} blocks of {w.nb_row}x{w.nb_col}) of the same workload, "
                      f"FP64 single-threaded C, {el:.1f} s"}


def run_reference(args, w):
    """--impl reference: the FP64 oracle on the host cores, bounded sample per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    prob = synth.workload_problem(w.name, seed=args.seed)
    start = synth.crude_start(prob, w.d, seed=args.seed)
    rp, cp = synth.partitions(w.n, w.m, args.seed)
    sig = synth.sweep_orders(w.n, w.m, w.nb_row, w.nb_col, 4, args.seed)
    import oracle
    f = oracle.OracleFit(prob.Y, prob.X, prob.Z, prob.offset, start, family=w.family, nb_row=w.nb_row,
                         nb_col=w.nb_col, row_perm=rp, col_perm=cp, settings=synth.fit_settings())
    nsw = synth.n_sweeps(w.n, w.m, w.nb_row, w.nb_col)
    per = min(-(-w.n // w.nb_row), -(-w.m // w.nb_col))
    sweeps_per_step = 4
    cursor = [0]

    def step():
        w0 = cursor[0] % nsw
        w1 = min(nsw, w0 + sweeps_per_step)
        f.sweeps(sig[(cursor[0] // nsw) % len(sig)], w0, w1)
        cursor[0] += w1 - w0
        return (w1 - w0) * per * w.nb_row * w.nb_col

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    entries = sum(step() for _ in range(args.steps))
    el = time.perf_counter() - t0
    v = entries / el
    sample = (f"{sweeps_per_step} sweeps ({sweeps_per_step * per} blocks of {w.nb_row}x{w.nb_col}) per step, "
              f"FP64 single-threaded C oracle")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": describe(w, "fp64"),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nb_medium")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "mixed"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    w = synth.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    if args.warmup < 3:
        raise SystemExit("warm-up must be >= 3 steps")

    import torch
    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build() if rank == 0 else None
    if dist is not None:
        dist.barrier()
    import paper_2412_20509_gb300 as gmf

    # Each rank fits its own replica of the workload (weak scaling, no data-path collective).
    prob = synth.workload_problem(w.name, seed=args.seed)
    start = synth.crude_start(prob, w.d, seed=args.seed)
    rp, cp = synth.partitions(w.n, w.m, args.seed)
    nsteps = args.warmup + args.steps
    sig = synth.sweep_orders(w.n, w.m, w.nb_row, w.nb_col, max(nsteps, 8), args.seed)
    settings = synth.fit_settings()
    Yd = torch.from_numpy(prob.Y).cuda()
    model = gmf.Model(Yd, prob.X, prob.Z, prob.offset, start, family=w.family, nb_row=w.nb_row, nb_col=w.nb_col,
                      row_perm=rp, col_perm=cp, settings=settings, precision=args.precision)
    stream = torch.cuda.current_stream()
    nsw = model.num_sweeps
    n, m, p, q, d = model.dims
    K, fr, fc = 1 + p + q + d, q + d, p + d

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- device-resident throughput
    for s in range(args.warmup):
        model.epoch(sig[s])
    dev0 = model.deviance()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for s in range(args.steps):
        model.epoch(sig[args.warmup + s])
    ev1.record(stream)
    barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    # Kernel-level timing of the dominant kernel: the same steps again, each
    # block-step launch bracketed by CUDA events on its stream.
    model.trace(True)
    model.trace_read()
    for s in range(args.steps):
        model.epoch(sig[args.warmup + s])
    kern_ms, launches = model.trace_read()
    model.trace(False)
    if dist is not None:
        t = torch.tensor([elapsed_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    entries_step = n * m
    value = ws * entries_step * args.steps / (elapsed_ms / 1e3)
    dev1 = model.deviance()

    # ---------------- end to end through the public API from pinned host memory
    Yh = torch.from_numpy(prob.Y).pin_memory()
    for s in range(3):
        model.update_y(Yh)
        model.epoch(sig[s])
        model.deviance()
    barrier()
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        model.update_y(Yh)            # H2D of the step's counts (pinned), on-device permutation
        model.epoch(sig[s])           # sigma: 4 bytes per sweep
        model.deviance()              # D2H: the FP64 deviance (+ status word)
    barrier()
    e2e_s = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = ws * entries_step * e2e_steps / e2e_s

    # ---------------- roofline of the dominant kernel (the block-step launch)
    peaks, peak_src = measured_peaks()
    ent_sweep, flops_sweep, bytes_sweep = sweep_algorithmic(w, K, fr, fc)
    avg_kernel_s = (kern_ms / max(launches, 1)) / 1e3
    if args.precision == "fp32":
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        peak = fp32_simt_peak_tflops(sm_mhz)
        achieved = flops_sweep / avg_kernel_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "sweep_kernel (FP32 CUDA cores)",
                "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz",
                "hbm_gbs": bytes_sweep / avg_kernel_s / 1e9, "hbm_peak_gbs": peaks["hbm_gbs"],
                "hbm_frac": bytes_sweep / avg_kernel_s / 1e9 / peaks["hbm_gbs"],
                "avg_launch_us": avg_kernel_s * 1e6, "launches": launches,
                "algorithmic_per_launch": {"entries": ent_sweep, "flops": flops_sweep, "bytes": bytes_sweep}}
    else:
        achieved = flops_sweep / avg_kernel_s / 1e12
        peak = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]))
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "tcgen05 block step", "peak_source": f"{peak_src} bf16 (sustained)",
                "hbm_gbs": bytes_sweep / avg_kernel_s / 1e9, "hbm_peak_gbs": peaks["hbm_gbs"],
                "hbm_frac": bytes_sweep / avg_kernel_s / 1e9 / peaks["hbm_gbs"],
                "avg_launch_us": avg_kernel_s * 1e6, "launches": launches,
                "algorithmic_per_launch": {"entries": ent_sweep, "flops": flops_sweep, "bytes": bytes_sweep}}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16x3+bf16/f32",
           "data": "synthetic (seeded NB GMF law; stands in for scRNA-seq counts)",
           "config": describe(w, args.precision), "roofline": roof,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(prob.Y.nbytes + 4 * nsw),
                   "d2h_bytes_per_step": 8 + 4},
           "gpu_launches": int(nsw * args.steps), "clocks": clk,
           "deviance": {"after_warmup": dev0, "after_timed_steps": dev1}}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, prob, start, rp, cp, sig)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
