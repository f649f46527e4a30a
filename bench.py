"""Benchmark: SGD matrix entries/s of the block-wise adaptive SGD for NB GMF.

Workload (default, nb_atlas): 200000 cells x 5000 genes of uint16 NB counts
(~90% zeros, library-size offsets, per-gene NB sizes; drawn on the GPU),
d = 20, p = 3, q = 1, 2048 x 1024 blocks, mixed precision (split-BF16 eta and
BF16 contractions on the tcgen05 tensor cores). One step = one 10-epoch fit
pass (98 sweeps of 5 disjoint blocks per epoch), launched through the C ABI
(gmf_sgd_epoch, one captured graph per epoch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload nb_atlas|nb_medium|nb_sweep|nb_project] [--precision fp32|mixed]

Prints one JSON line (rank 0). ``value`` = whole-job entries/s with Y resident
in HBM; ``e2e`` = the same metric through the public API with the counts
uploaded from pinned host memory each step and the deviance read back.
``--impl reference`` times the FP64 oracle on the host cores (a bounded
sample of the same workload per step). ``--workload nb_medium`` is the
20000 x 2000 int32 workload with a step of one epoch.
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


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the job ends when its slowest rank does)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, seconds):
    """Units of all ranks per second of the slowest rank (replicas: every rank runs the same workload)."""
    return ws * units_per_rank / seconds


class NvmlClocks:
    """SM clock and clock-event reasons read through NVML (read-only queries) every
    ~2 ms on a background thread, so that even a timed region of a few ms has
    samples; mark(True/False) brackets the timed region."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index):
        import ctypes as C
        self.C = C
        self.nvml = C.CDLL("libnvidia-ml.so.1")
        if self.nvml.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = C.c_void_p()
        if self.nvml.nvmlDeviceGetHandleByIndex_v2(C.c_uint(gpu_index), C.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        fn = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn if fn is not None else self.nvml.nvmlDeviceGetCurrentClocksThrottleReasons
        self.samples = []
        self.inside = False
        self.run = True
        self.t = threading.Thread(target=self._poll, daemon=True)

    def _poll(self):
        C = self.C
        mhz, mx, mask = C.c_uint(), C.c_uint(), C.c_ulonglong()
        while self.run:
            ok = self.nvml.nvmlDeviceGetClockInfo(self.h, 1, C.byref(mhz)) == 0   # NVML_CLOCK_SM
            ok = ok and self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, C.byref(mx)) == 0
            ok = ok and self.reasons_fn(self.h, C.byref(mask)) == 0
            if ok and self.inside:
                self.samples.append((mhz.value, mx.value, mask.value))
            time.sleep(0.002)

    def start(self):
        self.t.start()

    def mark(self, inside):
        self.inside = inside

    def stop(self):
        self.run = False
        self.t.join(timeout=2)
        try:
            self.nvml.nvmlShutdown()
        except Exception:
            pass
        sm = [a for a, _, _ in self.samples]
        reasons = sorted({nm for _, _, m in self.samples for bit, nm in self.REASONS.items() if m & bit})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(b for _, b, _ in self.samples) if self.samples else None,
                "reasons": reasons, "samples": len(sm), "source": "NVML, every ~2 ms inside the timed region"}


class ClockSampler:
    """Clock and throttle samples while the timed region runs: NVML when the
    driver's library loads, else nvidia-smi."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        try:
            self.nv = NvmlClocks(gpu_index)
        except (OSError, AttributeError):
            self.nv = None

    def start(self):
        if self.nv is not None:
            self.nv.start()
            return
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def mark(self, inside):
        if self.nv is not None:
            self.nv.mark(inside)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nv is not None:
            return self.nv.stop()
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
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, every 100 ms"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_simt_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def sfu_peak_ops(sm_mhz):
    # special-function unit (exp2, rcp, lg2): 152 SMs x 16 results per clock (4 per SM sub-partition) x clock
    return 152 * 16 * sm_mhz * 1e6


def host_cpu():
    """Core count and model of the host that runs the oracle (lscpu's model name,
    which names Arm cores by their part, else /proc/cpuinfo)."""
    model = "unknown"
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and v.strip():
                model = v.strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model == "unknown":
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    k, _, v = line.partition(":")
                    if k.strip() in ("model name", "Model name", "CPU part") and v.strip():
                        model = v.strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def sweep_entries(n, m, nb_row, nb_col, sg):
    """Matrix entries of the blocks of one sweep with offset sg (Algorithm 1's schedule)."""
    r, s = -(-n // nb_row), -(-m // nb_col)
    tot = 0
    for k in range(min(r, s)):
        rc, cc = ((sg + k) % r, k) if r >= s else (k, (sg + k) % s)
        tot += min(nb_row, n - rc * nb_row) * min(nb_col, m - cc * nb_col)
    return tot


def oracle_sweep_rate(Y, X, Z, offset, start, w, rp, cp, sigma, settings, budget_s):
    """The FP64 oracle as it stands (single-threaded C, one host core) on the same
    fit: the sweeps of one epoch in order until budget_s of host time has passed
    (at least one). Returns (entries/s, sweeps run, entries, seconds)."""
    import oracle
    oracle.build()
    f = oracle.OracleFit(Y, X, Z, offset, start, family=w.family, nb_row=w.nb_row, nb_col=w.nb_col,
                         row_perm=rp, col_perm=cp, settings=settings)
    n, m = Y.shape
    done, entries, t0 = 0, 0, time.perf_counter()
    while done < len(sigma) and (done == 0 or time.perf_counter() - t0 < budget_s):
        f.sweeps(sigma, done, done + 1)
        entries += sweep_entries(n, m, w.nb_row, w.nb_col, int(sigma[done]))
        done += 1
    dt = time.perf_counter() - t0
    return entries / dt, done, entries, dt


def sweep_algorithmic(w, K, fr, fc):
    """Algorithmic flops and HBM bytes of one sweep launch (all blocks of a sweep)."""
    per = min(-(-w.n // w.nb_row), -(-w.m // w.nb_col))
    entries = per * w.nb_row * w.nb_col
    flops_entry = 2 * K + 4 * fr + 4 * fc
    ybytes = 4 if w.y_dtype == "int32" else 2
    # counts once; parameters: L, R rows read; free columns + EMA (G, H) read and written
    pbytes = per * (w.nb_row * (4 * K + 24 * fr) + w.nb_col * (4 * K + 24 * fc))
    return entries, entries * flops_entry, entries * ybytes + pbytes


def host_problem(w, seed):
    """The workload's data on the host. The atlas-scale workload is drawn on the
    GPU when there is one (the same draw as the GPU arm's), else with numpy."""
    if w.name == "nb_atlas":
        try:
            import torch
            if torch.cuda.is_available():
                pd = synth.make_problem_device(w.n, w.m, w.p, w.q, w.d, w.family, seed=seed, zero_frac=w.zero_frac,
                                               offset=w.offset)
                return synth.Problem(Y=pd.Y.cpu().numpy().view(np.uint16), X=pd.X, Z=pd.Z, offset=pd.offset, B=pd.B,
                                     Gamma=pd.Gamma, U=pd.U, V=pd.V, nb_size=pd.nb_size, family=w.family,
                                     saturated=pd.saturated)
        except ImportError:
            pass
    return synth.workload_problem(w.name, seed=seed)


def headline_config(w, prob, precision):
    """config of the atlas-scale line (both arms)."""
    zero_frac = (float(np.count_nonzero(prob.Y == 0)) / prob.Y.size if isinstance(prob.Y, np.ndarray)
                 else float((prob.Y == 0).sum()) / prob.Y.numel())
    nsw = synth.n_sweeps(w.n, w.m, w.nb_row, w.nb_col)
    return {"workload": f"{w.name}: NB GMF {w.n}x{w.m} uint16 counts ({100 * zero_frac:.1f}% zeros, "
                        f"{prob.saturated} saturated at 65535), d={w.d}, p={w.p}, q={w.q}, blocks "
                        f"{w.nb_row}x{w.nb_col}; step = one {w.epochs}-epoch fit pass ({w.epochs * nsw} sweeps)",
            "n": w.n, "m": w.m, "d": w.d, "nb_row": w.nb_row, "nb_col": w.nb_col, "epochs_per_step": w.epochs,
            "precision": precision, "parallelism": "replicas",
            "l2": f"inputs larger than L2: Y is {w.n * w.m * 2 / 1e9:.1f} GB (L2 129 MB), every entry read once "
                  f"per epoch"}


def run_reference(args, w):
    """--impl reference: the FP64 oracle on the host cores, bounded sample per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    prob = host_problem(w, args.seed)
    start = synth.crude_start(prob, w.d, seed=args.seed)
    rp, cp = synth.partitions(w.n, w.m, args.seed)
    sig = synth.sweep_orders(w.n, w.m, w.nb_row, w.nb_col, 4, args.seed)
    import oracle
    f = oracle.OracleFit(prob.Y, prob.X, prob.Z, prob.offset, start, family=w.family, nb_row=w.nb_row,
                         nb_col=w.nb_col, row_perm=rp, col_perm=cp, settings=synth.fit_settings())
    nsw = synth.n_sweeps(w.n, w.m, w.nb_row, w.nb_col)
    per = min(-(-w.n // w.nb_row), -(-w.m // w.nb_col))
    sweeps_per_step = 1 if w.name == "nb_atlas" else 4   # about 1 s of oracle work per step
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
    cfg = headline_config(w, prob, "fp64") if w.name == "nb_atlas" else describe(w, "fp64")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": cfg,
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample, **host_cpu()},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def oracle_trajectory(wname, seed):
    """The FP64 oracle on the same fit (same start, partitions, sweep orders):
    per-epoch times and the final deviance."""
    import oracle
    w = synth.WORKLOADS[wname]
    prob = synth.workload_problem(w.name, seed=seed)
    start = synth.crude_start(prob, w.d, seed=seed)
    rp, cp = synth.partitions(w.n, w.m, seed)
    sig = synth.sweep_orders(w.n, w.m, w.nb_row, w.nb_col, w.epochs, seed)
    f = oracle.OracleFit(prob.Y, prob.X, prob.Z, prob.offset, start, family=w.family, nb_row=w.nb_row,
                         nb_col=w.nb_col, row_perm=rp, col_perm=cp, settings=synth.fit_settings())
    times = []
    t0 = time.perf_counter()
    for e in range(w.epochs):
        f.epoch(sig[e])
        times.append(time.perf_counter() - t0)
    return {"final_deviance": f.deviance(), "epoch_times": times, "entries_per_epoch": w.n * w.m,
            "epochs": w.epochs}


def source_hash(paths):
    import hashlib
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {
    "sweep_tc_kernel": ["gmf_step_tc.cu", "gmf_tc_tile.cuh", "gmf_update.cuh", "gmf_sm100.cuh", "gmf_internal.cuh"],
    "sweep_tc_cluster": ["gmf_step_tc.cu", "gmf_tc_tile.cuh", "gmf_update.cuh", "gmf_sm100.cuh", "gmf_internal.cuh"],
    "sweep_tc_epoch": ["gmf_step_tc.cu", "gmf_tc_tile.cuh", "gmf_update.cuh", "gmf_sm100.cuh", "gmf_internal.cuh"],
    "sweep_tc_flow": ["gmf_step_tc.cu", "gmf_tc_tile.cuh", "gmf_update.cuh", "gmf_sm100.cuh", "gmf_internal.cuh"],
    "deviance_tc": ["gmf_deviance_tc.cu", "gmf_tc_tile.cuh", "gmf_update.cuh", "gmf_sm100.cuh", "gmf_internal.cuh"],
    "sweep_kernel": ["gmf_step_simt.cu", "gmf_update.cuh", "gmf_internal.cuh"],
    "update_kernel": ["gmf_update.cu", "gmf_update.cuh", "gmf_internal.cuh"],
    "update_tc_kernel": ["gmf_update.cu", "gmf_update.cuh", "gmf_internal.cuh"],
    "deviance_kernel": ["gmf_step_simt.cu", "gmf_update.cuh", "gmf_internal.cuh"],
}


def kernel_hash(kernel):
    return source_hash([os.path.join(ROOT, "paper_2412_20509_gb300", "csrc", f) for f in KERNEL_SOURCES[kernel]])


def committed_traffic(kernel, workload):
    """dram read+write bytes per launch from the committed ncu summary of this
    kernel and workload, if it was captured on the current kernel sources."""
    prof = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(prof):
        return None
    got, traffic = None, None
    for line in open(prof):
        if line.startswith("source_sha256_16:"):
            got = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            traffic = float(line.split(":", 1)[1].strip())
    return traffic if got == kernel_hash(kernel) else None


RANKS = [2, 5, 10, 15, 20, 30, 40, 50]


def run_projection(args, w):
    """--workload nb_project: fit d = 20 on 100000 cells x 3000 genes, orthogonalise,
    train the warm-start encoder on the training cells' projected scores, then
    project 100000 held-out cells by 1, 2 and 3 safeguarded Fisher steps from
    the encoder's scores and from zero. Gaps (mean, median, 99th percentile) are
    to a 60-step cold fit on the penalised per-cell objective; cells/s of each."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_20509_gb300 as gmf
    n_fit = n_new = w.n // 2
    prob = synth.make_problem_device(w.n, w.m, w.p, w.q, w.d, w.family, seed=args.seed, zero_frac=w.zero_frac,
                                     offset=w.offset)
    Yfit, Ynew = prob.Y[:n_fit].contiguous(), prob.Y[n_fit:].contiguous()
    fitp = synth.Problem(Y=Yfit.cpu().numpy().view(np.uint16), X=prob.X[:n_fit], Z=prob.Z, offset=prob.offset[:n_fit],
                         B=prob.B, Gamma=prob.Gamma[:n_fit], U=prob.U[:n_fit], V=prob.V, nb_size=prob.nb_size,
                         family=w.family)
    start = synth.crude_start(fitp, w.d, seed=args.seed)
    rp, cp = synth.partitions(n_fit, w.m, args.seed)
    settings = synth.fit_settings(alpha_mode=1)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()

    def timed(fn):
        a, b = ev(), ev()
        torch.cuda.synchronize()
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, r

    model = gmf.Model(Yfit.view(torch.int16), fitp.X, fitp.Z, fitp.offset, start, family=w.family, nb_row=w.nb_row,
                      nb_col=w.nb_col, row_perm=rp, col_perm=cp, settings=settings, precision="mixed")
    sig = synth.sweep_orders(n_fit, w.m, w.nb_row, w.nb_col, w.epochs, args.seed)
    t_fit, _ = timed(lambda: [model.epoch(s) for s in sig])
    model.orthogonalize("B1")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Xf, of = dev(fitp.X), dev(fitp.offset)
    Xn, on = dev(prob.X[n_fit:]), dev(prob.offset[n_fit:])
    Utr, _, _ = model.project_cells(Yfit, Xf, of, None, n_steps=10, with_dev=False)
    epochs = 10
    net = gmf.MLP(w.m, 256, 256, w.d, max_batch=16384)   # forward in chunks of 16384 cells, training batches of 1024
    net.set_precision(args.encoder_precision)
    net.set_params({k: np.asarray(v, dtype=np.float32) for k, v in synth.mlp_init(w.m, 256, 256, w.d, 2).items()})
    t_train, losses = timed(lambda: net.train(Yfit, Utr, epochs=epochs, batch=1024, lr=1e-3, seed=5))
    lam_u, lam_g = settings["lambda_"][2], settings["lambda_"][1]

    def objective(U, G, D):
        return 0.5 * D.double() + 0.5 * lam_u * (U.double() ** 2).sum(1) + 0.5 * lam_g * (G.double() ** 2).sum(1)

    for _ in range(2):   # warm-up of the projection and forward kernels
        model.project_cells(Ynew, Xn, on, net.forward(Ynew), n_steps=3)
    t_ref, ref = timed(lambda: model.project_cells(Ynew, Xn, on, None, n_steps=60))
    oref = objective(*ref)
    conv = objective(*model.project_cells(Ynew, Xn, on, None, n_steps=30)) - oref

    def gap_stats(res):
        g = objective(*res) - oref
        return {"mean": float(g.mean()), "median": float(g.median()), "p99": float(g.quantile(0.99)),
                "max": float(g.max())}

    t_fwd, Uw = timed(lambda: net.forward(Ynew))
    heldout_mse = float(((Uw.double() - ref[0].double()) ** 2).mean())
    starts = {"warm_start": lambda k: model.project_cells(Ynew, Xn, on, net.forward(Ynew), n_steps=k),
              "cold_start": lambda k: model.project_cells(Ynew, Xn, on, None, n_steps=k)}
    res = {}
    for name, run in starts.items():
        res[name] = {}
        for k in (1, 2, 3):
            t, r = timed(lambda: run(k))
            res[name][f"steps_{k}"] = {"cells_per_s": n_new / t, "objective_gap": gap_stats(r)}
    out = {"metric": "per-cell projection of new cells: cells/s and gap to a converged cold fit",
           "value": res["warm_start"]["steps_3"]["cells_per_s"], "unit": "cells/s", "n_gpus": 1,
           "higher_is_better": True,
           "config": {"workload": f"{w.name}: fit {n_fit} + project {n_new} cells x {w.m} genes, NB, d={w.d}, "
                                  f"GMF fit {w.epochs} epochs (tensor cores), encoder {w.m}-256-256-{w.d} trained "
                                  f"{epochs} epochs on the training cells' projected scores; value = warm start, "
                                  f"3 Fisher steps, encoder forward included",
                      "encoder_precision": args.encoder_precision, "data": "synthetic (GPU-drawn)"},
           **res,
           "reference_cold_fit": {"steps": 60, "cells_per_s": n_new / t_ref, "mean_objective": float(oref.mean()),
                                  "max_gap_30_steps": float(conv.max()), "mean_gap_30_steps": float(conv.mean())},
           "encoder": {"train_samples_per_s": epochs * n_fit / t_train, "loss_first_epoch": float(losses[0]),
                       "loss_last_epoch": float(losses[-1]), "forward_cells_per_s": n_new / t_fwd,
                       "heldout_mse_to_converged_scores": heldout_mse,
                       "converged_score_second_moment": float((ref[0].double() ** 2).mean())},
           "gmf_fit_entries_per_s": n_fit * w.m * w.epochs / t_fit}
    if not args.no_cpu_baseline:
        # the FP64 oracle on the first 1000 held-out cells: the encoder's forward pass
        # and 3 safeguarded Fisher steps, and the cold 3-step projection
        import oracle.mlp as omlp
        import oracle.project as oproj
        nc = 1000
        prm = model.get_params()
        P = {k: np.asarray(v, dtype=np.float64) for k, v in net.get_params().items()}
        Yc = Ynew[:nc].cpu().numpy().view(np.uint16)
        Xc, oc = np.asarray(prob.X[n_fit:n_fit + nc]), np.asarray(prob.offset[n_fit:n_fit + nc])
        kw = dict(family=w.family, alpha=prm["alpha"], n_steps=3, lam_gamma=lam_g, lam_u=lam_u)
        t0 = time.perf_counter()
        Uo = omlp.forward(P, Yc)[0]
        oproj.project_cells(Yc, Xc, oc, prm["B"], prob.Z, prm["V"], U_start=Uo, **kw)
        t_warm = time.perf_counter() - t0
        t0 = time.perf_counter()
        oproj.project_cells(Yc, Xc, oc, prm["B"], prob.Z, prm["V"], U_start=None, **kw)
        t_cold = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": nc / t_warm, "unit": "cells/s", "cores": 1, "kind": "oracle", **host_cpu(),
                               "cold_start_3_steps_cells_per_s": nc / t_cold,
                               "sample": f"first {nc} held-out cells, encoder forward + 3 safeguarded Fisher steps "
                                         f"(FP64 numpy; {t_warm:.1f} s; the cold 3-step projection {t_cold:.1f} s)"}
    print(json.dumps(out), flush=True)
    return 0


def epoch_algorithmic(n, m, nb_row, nb_col, K, fr, fc, ybytes):
    """Algorithmic work of one epoch (every block once, ragged chunks counted
    exactly): entries, flops (2K for eta and 4 per free column and side for
    the gradient and curvature contractions, per entry) and HBM bytes (every
    count once; per block visit, each row and column of the block reads its K
    factors and reads and writes theta, Gbar and Hbar of its free columns).
    Each row chunk is visited s times per epoch and each column chunk r times."""
    r, s = -(-n // nb_row), -(-m // nb_col)
    entries = n * m
    flops = entries * (2 * K + 4 * fr + 4 * fc)
    byts = entries * ybytes + s * n * (4 * K + 24 * fr) + r * m * (4 * K + 24 * fc)
    return entries, flops, byts


def committed_sweep_traffic(workload, kernels):
    """Sum of the committed per-launch DRAM bytes of the given kernels (one
    sweep's launches), or None if any summary is missing or stale."""
    tot = 0.0
    for k in kernels:
        t = committed_traffic(k, workload)
        if t is None:
            return None
        tot += t
    return tot


def run_headline(args, w):
    """The headline line: config 3 of the benchmark suite, NB GMF at atlas scale.

    200000 x 5000 uint16 counts (~90 % zeros; drawn on the GPU), d = 20, p = 3,
    q = 1, blocks 2048 x 1024. One step = one full fit pass of the workload's
    10 epochs (980 sweeps, every entry 10 times), graph-replayed through
    gmf_sgd_epoch on the tensor-core path. value = entries/s of the timed steps
    (device-resident counts); the roofline's unit is one sweep (its tile and
    update launches), whose duration is the graph-timed step time divided by
    the sweeps of a step. Beside it: the FP32 path on the same fit, time to
    the FP32 fit's final deviance (within 1e-3) for both paths, end to end
    through the C ABI from pinned host counts, and the FP64 oracle on the
    host cores after all GPU work."""
    if args.warmup < 3:
        raise SystemExit("warm-up must be >= 3 steps")
    ws, rank, local = dist_env()
    extras = rank == 0 and ws == 1
    import torch
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

    # Every rank fits its own replica (weak scaling; the blocks of a sweep are
    # disjoint, but one sweep of this workload already fills one GPU).
    prob = synth.make_problem_device(w.n, w.m, w.p, w.q, w.d, w.family, seed=args.seed, zero_frac=w.zero_frac,
                                     offset=w.offset)
    Yhost = prob.Y.cpu()
    hp = synth.Problem(Y=Yhost.numpy().view(np.uint16), X=prob.X, Z=prob.Z, offset=prob.offset, B=prob.B,
                       Gamma=prob.Gamma, U=prob.U, V=prob.V, nb_size=prob.nb_size, family=w.family,
                       saturated=prob.saturated)
    start = synth.crude_start(hp, w.d, seed=args.seed)
    rp, cp = synth.partitions(w.n, w.m, args.seed)
    sig = synth.sweep_orders(w.n, w.m, w.nb_row, w.nb_col, w.epochs, args.seed)
    settings = synth.fit_settings()
    stream = torch.cuda.current_stream()
    eps = w.epochs                      # epochs per step: one full fit pass

    def make(precision, Y=None, flags=0):
        if precision == "mixed" and args.epoch_launch == "persistent":
            flags |= gmf.GMF_FLAG_PERSIST
        mdl = gmf.Model(prob.Y if Y is None else Y, prob.X, prob.Z, prob.offset, start, family=w.family,
                        nb_row=w.nb_row, nb_col=w.nb_col, row_perm=rp, col_perm=cp, settings=settings,
                        precision=precision, flags=flags)
        if args.flow_lag is not None:
            mdl.set_flow_lag(args.flow_lag)
        return mdl

    def step(mdl):
        for e in range(eps):
            mdl.epoch(sig[e])

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(mdl, count, clk=None):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        if clk is not None:
            clk.mark(True)
        e0.record(stream)
        for _ in range(count):
            step(mdl)
        e1.record(stream)
        barrier()
        if clk is not None:
            clk.mark(False)
        return e0.elapsed_time(e1)

    # uploads by the copy engines into a staging buffer: the gather kernel's CTAs would take SM room from the
    # epochs running beside it (the end-to-end leg below measures both routes)
    model = make("mixed", flags=gmf.GMF_FLAG_STAGED_UPLOAD)
    nsw = model.num_sweeps
    n, m, p, q, d = model.dims
    K, fr, fc = 1 + p + q + d, q + d, p + d
    # ---------------- device-resident throughput (the headline value)
    for _ in range(args.warmup):
        step(model)
    dev0 = model.deviance()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.05)
    elapsed_ms = timed_steps(model, args.steps, clocks)
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(elapsed_ms, dist, "cuda")
    ms_step = elapsed_ms / args.steps
    entries_step = n * m * eps
    value = whole_job_rate(entries_step * args.steps, ws, elapsed_ms / 1e3)
    dev1 = model.deviance()
    devk = deviance_timing(gmf, model, make, stream, n * m, K)
    launches_per_sweep = model.launches_per_sweep
    epoch_mode = model.epoch_mode
    # context only: the tile launches of one step bracketed one by one with events (outside the graph)
    model.trace(True)
    model.trace_read()
    step(model)
    kern_ms, kern_launches = model.trace_read()
    model.trace(False)

    # ---------------- end to end through the C ABI from pinned host memory
    Yh = Yhost.pin_memory()
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    res_h = torch.zeros(1, dtype=torch.float64).pin_memory()

    def e2e_run(mdl, count):
        # every step: the upload of its counts (issued during the previous step, so it overlaps that
        # step's epochs; the first one here), the fit pass, and the D2H read of its FP64 deviance
        mdl.update_y_async(Yh)
        for s in range(count):
            step(mdl)
            mdl.deviance_async(res)
            res_h.copy_(res, non_blocking=True)
            if s + 1 < count:
                mdl.update_y_async(Yh)
            stream.synchronize()
            float(res_h.item())

    def e2e_timed(mdl):
        e2e_run(mdl, 2)
        barrier()
        t0 = time.perf_counter()
        e2e_run(mdl, e2e_steps)
        barrier()
        return max_over_ranks(time.perf_counter() - t0, dist, "cuda")

    e2e_steps = max(3, min(args.steps, 8))
    e2e_s = e2e_timed(model)
    e2e_value = whole_job_rate(entries_step * e2e_steps, ws, e2e_s)
    del model
    torch.cuda.empty_cache()
    # context: the same leg with the direct gather from host memory into a second count buffer
    mg = make("mixed")
    e2e_gather = whole_job_rate(entries_step * e2e_steps, ws, e2e_timed(mg)) if extras else None
    del mg, Yh
    torch.cuda.empty_cache()

    # ---------------- roofline: one sweep (tile launch + update launch) is the unit
    peaks, peak_src = measured_peaks()
    ent_ep, flops_ep, bytes_ep = epoch_algorithmic(n, m, w.nb_row, w.nb_col, K, fr, fc, 2)
    sweep_s = ms_step / 1e3 / (eps * nsw)
    per_sweep = {"entries": ent_ep / nsw, "flops": flops_ep / nsw, "bytes": bytes_ep / nsw}
    hbm_gbs = per_sweep["bytes"] / sweep_s / 1e9
    peak = float(peaks["hbm_gbs"])
    tc_peak = float(peaks.get("bf16_tflops", 1900.0))
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    tflops = per_sweep["flops"] / sweep_s / 1e12
    tflops_exec = per_sweep["entries"] * (6 * K + 4 * fr + 4 * fc) / sweep_s / 1e12
    sfu = per_sweep["entries"] * 2 / sweep_s
    flow = epoch_mode == "persistent" and -(-w.nb_row // 128) * -(-w.nb_col // 128) > 16
    tile_k = {"cluster": "sweep_tc_cluster", "persistent": "sweep_tc_flow" if flow else "sweep_tc_epoch"}.get(
        epoch_mode, "sweep_tc_kernel")
    sweep_kernels = [tile_k] if epoch_mode != "separate" else [tile_k, "update_tc_kernel"]
    roof = {"bound": "hbm", "achieved": hbm_gbs, "peak": peak, "unit": "GB/s", "frac": hbm_gbs / peak,
            "traffic": committed_sweep_traffic(w.name, sweep_kernels),
            "kernel": " + ".join(sweep_kernels) + f" (one sweep: {launches_per_sweep} launch(es), graph-replayed)",
            "unit_of_work": "one sweep = the 5 disjoint 2048 x 1024 blocks of Algorithm 1's schedule (the epoch's "
                            "average: n*m/98 entries)",
            "sweep_us": sweep_s * 1e6, "sweeps_per_step": eps * nsw,
            "algorithmic_per_sweep": per_sweep,
            "peak_source": f"{peak_src} STREAM-style copy (MEASURED_PEAKS.json hbm_gbs)",
            "tensor_tflops": tflops, "tensor_tflops_as_executed": tflops_exec, "tensor_peak_tflops": tc_peak,
            "tensor_frac_of_measured": tflops / tc_peak,
            "tensor_frac_as_executed": tflops_exec / tc_peak,
            "sfu_ops_per_s": sfu, "sfu_peak_ops_per_s": sfu_peak_ops(sm_mhz), "sfu_frac": sfu / sfu_peak_ops(sm_mhz),
            "sfu_peak_source": f"derived: 152 SMs x 16 SFU results per clock x {sm_mhz:.0f} MHz (exp and the NB "
                               "reciprocal: 2 per entry)",
            "binding_roof": "HBM at 2.92 B per entry (2.4e12 entries/s) and the SFU at 2 results per entry "
                            "(2.5e12 entries/s) bound alike; the tensor pipe would allow ~5.8e12",
            "traced_tile_launch_us": 1e3 * kern_ms / max(kern_launches, 1),
            "traced_tile_launch_note": "context only: each tile launch of one step bracketed by events outside the "
                                       "graph (no overlap with the neighbouring launches)"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16x3 eta + bf16 contractions, f32 accumulate/epilogue",
           "data": "synthetic (seeded NB GMF law drawn on the GPU; stands in for an scRNA-seq atlas)",
           "config": headline_config(w, prob, "mixed"),
           "roofline": roof,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(n * m * 2 + 4 * nsw * eps),
                   "d2h_bytes_per_step": 8,
                   "api": "per step: gmf_update_y_async of the counts (2 GB by the copy engines into a staging "
                          "buffer, GMF_FLAG_STAGED_UPLOAD, issued one step ahead so the copy overlaps the previous "
                          "step; the permutation into the count matrix runs on the stream), 10 x gmf_sgd_epoch, "
                          "gmf_deviance_async + D2H",
                   "value_with_direct_gather": e2e_gather},
           "gpu_launches": int(launches_per_sweep * nsw * eps * args.steps), "epoch_mode": epoch_mode,
           "clocks": clk, "deviance": {"after_warmup": dev0, "after_timed_steps": dev1, **devk}}

    if extras:
        # ---------------- the FP32 path on the same fit
        mo = make("fp32")
        step(mo)
        oms = timed_steps(mo, 2)
        out["fp32_path"] = {"value": entries_step * 2 / (oms / 1e3), "ms_per_step": oms / 2}
        out["mixed_over_fp32_throughput"] = value / out["fp32_path"]["value"]
        del mo
        torch.cuda.empty_cache()
        # ---------------- time to the FP32 fit's final deviance (within 1e-3): fresh fits, deviance every epoch
        traj, orth = {}, {}
        for prec in ("mixed", "fp32"):
            mdl = make(prec)
            devbuf = torch.zeros(eps, dtype=torch.float64, device="cuda")
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(eps + 1)]
            barrier()
            evs[0].record(stream)
            for e in range(eps):
                mdl.epoch(sig[e])
                mdl.deviance_async(devbuf[e:e + 1])
                evs[e + 1].record(stream)
            barrier()
            traj[prec] = (devbuf.cpu().numpy().tolist(), [evs[0].elapsed_time(evs[e + 1]) / 1e3 for e in range(eps)])
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mdl.orthogonalize("B1")
            b.record(stream)
            torch.cuda.synchronize()
            orth[prec] = {"ms": a.elapsed_time(b), "deviance_after": mdl.deviance()}
            del mdl
            torch.cuda.empty_cache()
        target = traj["fp32"][0][-1] * (1 + 1e-3)
        ttd = {"target": target, "rule": f"within 1e-3 of the FP32 path's deviance after {eps} epochs (FP32 is held "
                                         "to the FP64 oracle within 1e-4 by the parity tests)",
               "includes_per_epoch_deviance": True, "epochs": eps}
        for prec, (devs, cum) in traj.items():
            hit = next((e for e, dv in enumerate(devs) if dv <= target), None)
            ttd[prec] = {"seconds": None if hit is None else cum[hit], "epochs": None if hit is None else hit + 1,
                         "final_deviance": devs[-1], "deviance_per_epoch": devs,
                         "orthogonalize_b1_fp64": orth[prec]}
        ttd["final_rel_gap_mixed_vs_fp32"] = traj["mixed"][0][-1] / traj["fp32"][0][-1] - 1.0
        if ttd["mixed"]["seconds"] and ttd["fp32"]["seconds"]:
            ttd["fp32_over_mixed"] = ttd["fp32"]["seconds"] / ttd["mixed"]["seconds"]
        out["time_to_deviance"] = ttd
        if not args.no_cpu_baseline:
            # the FP64 oracle on the host cores, after every GPU leg: the first sweeps of epoch 1 of the same fit
            rate, done, ent, dt = oracle_sweep_rate(hp.Y, hp.X, hp.Z, hp.offset, start, w, rp, cp, sig[0], settings,
                                                    budget_s=15.0)
            out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", **host_cpu(),
                                   "sample": f"first {done} sweeps of epoch 1 ({ent:.3g} entries) of the same fit, "
                                             f"FP64 single-threaded C on one host core, {dt:.1f} s, run after the GPU "
                                             f"legs; entries/s does not depend on the epoch count"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def deviance_timing(gmf, model, make, stream, entries, K, reps=5):
    """The full deviance (gmf_deviance_async) of the fitted model: the tensor-core kernel of mixed handles and
    the CUDA-core kernel (GMF_FLAG_SIMT_DEVIANCE) on the same parameters, each the mean of `reps` calls timed
    with events on the stream; bytes = the counts (2 B per entry) + the factor rows read once."""
    import torch
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    twin = make("mixed", flags=gmf.GMF_FLAG_SIMT_DEVIANCE)
    twin.set_params(model.get_params())
    res = {}
    for name, mdl in (("tensor_core", model), ("cuda_core", twin)):
        mdl.deviance_async(out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            mdl.deviance_async(out)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        res[name] = {"ms": ms, "entries_per_s": entries / (ms / 1e3), "total": float(out.item())}
    n, m = model.dims[:2]
    byts = 2 * entries + 4 * (n + m) * K
    res["tensor_core"]["hbm_gbs"] = byts / (res["tensor_core"]["ms"] / 1e3) / 1e9
    res["bytes_per_call"] = byts
    res["rel_gap"] = res["tensor_core"]["total"] / res["cuda_core"]["total"] - 1.0
    del twin
    torch.cuda.empty_cache()
    return {"full_deviance": res}


def run_case(args):
    """--case: one-kernel measurement cases of a size an ncu capture handles.
    atlas_sweep: 4 sweeps of the atlas workload's launch shape (5 blocks of 2048 x 1024, d = 20, uint16) on
      50000 x 5000 counts, one tile launch and one update launch each.
    deviance_50000: one full deviance of a d = 20 NB model on 50000 x 5000 uint16 counts (after one epoch).
    project_20000: a d = 20 NB model (2 fit epochs, mixed precision) on 20000 cells x 3000 genes,
      then the tensor-core projection of 20000 held-out cells with 3 Fisher passes.
    encoder_16384: the forward pass of a 3000-256-256-20 encoder (first layer on the tensor cores) on 16384
      cells."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_20509_gb300 as gmf
    ev = lambda: torch.cuda.Event(enable_timing=True)
    if args.case == "atlas_sweep":
        # the atlas workload's sweep on fewer rows (every sweep is 5 blocks of 2048 x 1024 whatever n is):
        # 50000 x 5000 uint16 (500 MB, larger than L2), d = 20, one epoch as a graph, then sweeps one launch
        # pair at a time
        w = synth.WORKLOADS["nb_atlas"]
        n = 50000
        prob = synth.make_problem_device(n, w.m, w.p, w.q, w.d, w.family, seed=1, zero_frac=w.zero_frac,
                                         offset=True)
        hp = synth.Problem(Y=prob.Y.cpu().numpy().view(np.uint16), X=prob.X, Z=prob.Z, offset=prob.offset,
                           B=prob.B, Gamma=prob.Gamma, U=prob.U, V=prob.V, nb_size=prob.nb_size, family=w.family)
        start = synth.crude_start(hp, w.d, seed=1)
        rp, cp = synth.partitions(n, w.m, 1)
        model = gmf.Model(prob.Y, prob.X, prob.Z, prob.offset, start, family=w.family, nb_row=w.nb_row,
                          nb_col=w.nb_col, row_perm=rp, col_perm=cp, settings=synth.fit_settings(),
                          precision=args.precision)
        sg = synth.sweep_orders(n, w.m, w.nb_row, w.nb_col, 2, 1)
        model.epoch(sg[0])
        r = -(-n // w.nb_row)
        # sweeps whose 5 row chunks are all full (no ragged last chunk): the per-launch work of the full workload
        full = [i for i in range(r) if all((int(sg[1][i]) + k) % r != r - 1 for k in range(5))][:4]
        run = lambda: [model.sweeps(sg[1], i, i + 1) for i in full]
        units, unit = sum(sweep_entries(n, w.m, w.nb_row, w.nb_col, int(sg[1][i])) for i in full), "entries/s"
    elif args.case == "deviance_50000":
        # the full deviance (tensor-core kernel) of a d = 20 NB model on 50000 x 5000 uint16 counts (500 MB,
        # larger than L2) after one fit epoch
        w = synth.WORKLOADS["nb_atlas"]
        n = 50000
        prob = synth.make_problem_device(n, w.m, w.p, w.q, w.d, w.family, seed=1, zero_frac=w.zero_frac,
                                         offset=True)
        hp = synth.Problem(Y=prob.Y.cpu().numpy().view(np.uint16), X=prob.X, Z=prob.Z, offset=prob.offset,
                           B=prob.B, Gamma=prob.Gamma, U=prob.U, V=prob.V, nb_size=prob.nb_size, family=w.family)
        start = synth.crude_start(hp, w.d, seed=1)
        rp, cp = synth.partitions(n, w.m, 1)
        model = gmf.Model(prob.Y, prob.X, prob.Z, prob.offset, start, family=w.family, nb_row=w.nb_row,
                          nb_col=w.nb_col, row_perm=rp, col_perm=cp, settings=synth.fit_settings(),
                          precision=args.precision)
        model.epoch(synth.sweep_orders(n, w.m, w.nb_row, w.nb_col, 1, 1)[0])
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        run = lambda: model.deviance_async(out)
        units, unit = n * w.m, "entries/s"
    elif args.case == "project_20000":
        n_fit = n_new = 20000
        m, d = 3000, 20
        prob = synth.make_problem_device(n_fit + n_new, m, 3, 1, d, "negbin", seed=1, zero_frac=0.9, offset=True)
        Yfit, Ynew = prob.Y[:n_fit].contiguous(), prob.Y[n_fit:].contiguous()
        fitp = synth.Problem(Y=Yfit.cpu().numpy().view(np.uint16), X=prob.X[:n_fit], Z=prob.Z,
                             offset=prob.offset[:n_fit], B=prob.B, Gamma=prob.Gamma[:n_fit], U=prob.U[:n_fit], V=prob.V,
                             nb_size=prob.nb_size, family="negbin")
        start = synth.crude_start(fitp, d, seed=1)
        rp, cp = synth.partitions(n_fit, m, 1)
        model = gmf.Model(Yfit, fitp.X, fitp.Z, fitp.offset, start, family="negbin", nb_row=2048, nb_col=1024,
                          row_perm=rp, col_perm=cp, settings=synth.fit_settings(alpha_mode=1), precision="mixed")
        for sg in synth.sweep_orders(n_fit, m, 2048, 1024, 2, 1):
            model.epoch(sg)
        Xn = torch.from_numpy(np.ascontiguousarray(prob.X[n_fit:])).cuda()
        on = torch.from_numpy(np.ascontiguousarray(prob.offset[n_fit:])).cuda()
        run = lambda: model.project_cells(Ynew, Xn, on, None, n_steps=3)
        units, unit = n_new, "cells/s"
    else:
        n, m = 16384, 3000
        g = torch.Generator(device="cuda")
        g.manual_seed(3)
        lam = torch.empty((n, m), device="cuda").exponential_(1.0, generator=g).mul_(0.6)
        Y = torch.poisson(lam, generator=g).clamp_(max=65535).to(torch.int32)
        Y16 = torch.where(Y > 32767, Y - 65536, Y).to(torch.int16)
        net = gmf.MLP(m, 256, 256, 20, max_batch=n)
        net.set_precision("mixed")
        net.set_params({k: np.asarray(v, dtype=np.float32) for k, v in synth.mlp_init(m, 256, 256, 20, 2).items()})
        run = lambda: net.forward(Y16)
        units, unit = n, "cells/s"
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record()
    run()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    print(json.dumps({"case": args.case, "ms": ms, "value": units / (ms / 1e3), "unit": unit}), flush=True)
    return 0


def setting_name(group):
    """The rank sweep's launch setting in words."""
    if group == -1:
        return "sequential (each model's own epoch)"
    if group == -3:
        return "one persistent launch per sweep (all models)"
    return str(group)


def run_rank_sweep(args, w):
    """--workload nb_sweep: 8 ranks on one 50000 x 3000 NB matrix, batched (one
    launch per sweep for all models) vs the same 8 fits one after another."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_20509_gb300 as gmf
    prob = synth.workload_problem(w.name, seed=args.seed)
    rp, cp = synth.partitions(w.n, w.m, args.seed)
    starts = [synth.crude_start(prob, d, seed=args.seed) for d in RANKS]
    sig = synth.sweep_orders(w.n, w.m, w.nb_row, w.nb_col, args.warmup + args.steps, args.seed)
    kw = dict(family=w.family, nb_row=w.nb_row, nb_col=w.nb_col, row_perm=rp, col_perm=cp,
              settings=synth.fit_settings(), precision=args.precision)
    Yd = torch.from_numpy(prob.Y.view(np.int16)).cuda()
    stream = torch.cuda.current_stream()

    def timed(run):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    sw = gmf.Sweep(prob.Y, prob.X, prob.Z, prob.offset, starts, RANKS, **kw)
    t0 = time.perf_counter()
    group, tune_ms = sw.autotune(sig[0])   # launch grouping timed on one epoch's sweeps, state restored
    tune_s = time.perf_counter() - t0
    for s in range(args.warmup):
        sw.epoch(sig[s])
    ms_b = timed(lambda: [sw.epoch(sig[args.warmup + s]) for s in range(args.steps)])
    devs_b = [mdl.deviance() for mdl in sw.models]
    del sw
    solo = [gmf.Model(prob.Y, prob.X, prob.Z, prob.offset, st, **kw) for st in starts]
    for mdl in solo:
        for s in range(args.warmup):
            mdl.epoch(sig[s])
    ms_s = timed(lambda: [mdl.epoch(sig[args.warmup + s]) for mdl in solo for s in range(args.steps)])
    devs_s = [mdl.deviance() for mdl in solo]
    work = len(RANKS) * w.n * w.m * args.steps
    out = {"metric": "rank sweep: model x matrix entries/s, 8 ranks d in {2,5,10,15,20,30,40,50}",
           "value": work / (ms_b / 1e3), "unit": "model-entries/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_b / args.steps, "higher_is_better": True,
           "config": {"workload": f"{w.name}: NB {w.n}x{w.m} uint16, blocks {w.nb_row}x{w.nb_col}, step = one epoch "
                                  f"of all 8 models", "precision": args.precision},
           "sequential": {"value": work / (ms_s / 1e3), "ms_per_step": ms_s / args.steps},
           "batched_over_sequential": ms_s / ms_b,
           "deviance_batched_equals_sequential": devs_b == devs_s,
           "autotune": {"models_per_launch": setting_name(group),
                        "epoch_ms_by_models_per_launch": {setting_name(k): v for k, v in tune_ms.items()},
                        "seconds": tune_s}}
    if not args.no_cpu_baseline:
        ent_all, t_all, per_rank = 0, 0.0, {}
        for d, st in zip(RANKS, starts):
            rate, done, ent, dt = oracle_sweep_rate(prob.Y, prob.X, prob.Z, prob.offset, st, w, rp, cp, sig[0],
                                                    synth.fit_settings(), budget_s=2.0)
            ent_all, t_all = ent_all + ent, t_all + dt
            per_rank[str(d)] = rate
        out["cpu_baseline"] = {"value": ent_all / t_all, "unit": "model-entries/s", "cores": 1, "kind": "oracle",
                               **host_cpu(), "per_rank_entries_per_s": per_rank,
                               "sample": f"each of the 8 models run alone for the first sweeps of epoch 1 (about "
                                         f"2 s each, {ent_all:.3g} model-entries), FP64 single-threaded C on one "
                                         f"host core, {t_all:.1f} s"}
    print(json.dumps(out), flush=True)
    return 0


def run_select(args, w):
    """--workload nb_select: rank selection (Sec. 4.2) on the rank-sweep workload's law (50000 x 3000 uint16
    NB, true d = 10) with 30 % of the entries held out uniformly (Sec. 5.2): the 8 ranks fitted together in
    the batched sweep (15 epochs, entries marked missing and imputed), then AIC / BIC, the held-out error and
    relative Poisson deviance of every rank, and the eigenvalue-ratio rank of the d = 50 fit after (B1)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_20509_gb300 as gmf
    from paper_2412_20509_gb300 import select
    prob = synth.workload_problem(w.name, seed=args.seed)
    obs = synth.holdout_mask(w.n, w.m, 0.3, args.seed)
    Ym = synth.with_missing(prob.Y, obs)
    rp, cp = synth.partitions(w.n, w.m, args.seed)
    starts = [synth.crude_start(prob, d, seed=args.seed) for d in RANKS]
    sig = synth.sweep_orders(w.n, w.m, w.nb_row, w.nb_col, w.epochs, args.seed)
    kw = dict(family=w.family, nb_row=w.nb_row, nb_col=w.nb_col, row_perm=rp, col_perm=cp,
              settings=synth.fit_settings(missing=1), precision=args.precision)
    to_dev = lambda a: torch.from_numpy(a.view(np.int16)).cuda()
    sw = gmf.Sweep(to_dev(Ym), prob.X, prob.Z, prob.offset, starts, RANKS, **kw)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for s in sig:
        sw.epoch(s)
    e1.record(stream)
    torch.cuda.synchronize()
    fit_ms = e0.elapsed_time(e1)
    Ytrue = to_dev(prob.Y)
    t0 = time.perf_counter()
    sums = [select.fit_summary(mdl, w.family, Ytrue) for mdl in sw.models]
    sw.models[-1].orthogonalize("B1")
    spec = select.singular_values(sw.models[-1])
    pick = select.select_rank(sums, spec)
    eval_s = time.perf_counter() - t0
    work = len(RANKS) * w.n * w.m * w.epochs
    out = {"metric": "rank selection: model x matrix entries/s of the batched fit with 30% held out, and the "
                     "rank each criterion selects (true d = 10)",
           "value": work / (fit_ms / 1e3), "unit": "model-entries/s", "n_gpus": 1, "higher_is_better": True,
           "config": {"workload": f"{w.name}: NB {w.n}x{w.m} uint16 (true d = {w.d}), 30% of the entries held "
                                  f"out uniformly and marked missing, ranks {RANKS}, {w.epochs} epochs, blocks "
                                  f"{w.nb_row}x{w.nb_col}", "precision": args.precision,
                      "data": "synthetic (seeded NB GMF law)"},
           "fit_ms": fit_ms, "evaluation_s": eval_s, "selected": pick, "per_rank": sums,
           "spectrum_d50": [float(x) for x in spec]}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nb_atlas", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["fp32", "mixed"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttd", action="store_true", help="skip the time-to-deviance comparison")
    ap.add_argument("--epoch-launch", default="per-sweep", choices=["per-sweep", "persistent"],
                    help="mixed precision on nb_atlas: per-sweep tile and update launches, or one persistent "
                         "launch per epoch (GMF_FLAG_PERSIST)")
    ap.add_argument("--flow-lag", type=int, default=None, help="item order of the persistent epoch (gmf_set_flow_lag)")
    ap.add_argument("--encoder-precision", default="mixed", choices=["fp32", "mixed"],
                    help="nb_project: the encoder's first layer on the tensor cores (mixed) or FP32")
    ap.add_argument("--case", default=None, choices=["atlas_sweep", "deviance_50000", "project_20000",
                                                     "encoder_16384"],
                    help="a one-kernel measurement case (the profiles' captures)")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    w = synth.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    if args.workload == "nb_atlas":
        return run_headline(args, w)
    if args.workload == "nb_sweep":
        return run_rank_sweep(args, w)
    if args.workload == "nb_project":
        return run_projection(args, w)
    if args.workload == "nb_select":
        return run_select(args, w)
    if args.warmup < 3:
        raise SystemExit("warm-up must be >= 3 steps")
    ws, rank, local = dist_env()
    extras = rank == 0 and ws == 1

    import torch
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
    stream = torch.cuda.current_stream()

    def make(precision, flags=0):
        return gmf.Model(Yd, prob.X, prob.Z, prob.offset, start, family=w.family, nb_row=w.nb_row,
                         nb_col=w.nb_col, row_perm=rp, col_perm=cp, settings=settings, precision=precision,
                         flags=flags)

    model = make(args.precision)
    nsw = model.num_sweeps
    n, m, p, q, d = model.dims
    K, fr, fc = 1 + p + q + d, q + d, p + d

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_epochs(mdl, first, count, clk=None):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        if clk is not None:
            clk.mark(True)
        e0.record(stream)
        for s in range(count):
            mdl.epoch(sig[first + s])
        e1.record(stream)
        barrier()
        if clk is not None:
            clk.mark(False)
        return e0.elapsed_time(e1)

    # ---------------- device-resident throughput (the headline value)
    for s in range(args.warmup):
        model.epoch(sig[s])
    dev0 = model.deviance()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.05)  # the sampler is polling before the timed region starts
    elapsed_ms = timed_epochs(model, args.warmup, args.steps, clocks)
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(elapsed_ms, dist, "cuda")
    entries_step = n * m
    value = whole_job_rate(entries_step * args.steps, ws, elapsed_ms / 1e3)
    dev1 = model.deviance()
    # Kernel-level timing of the dominant kernel: the same steps again, each
    # block-step launch bracketed by CUDA events on its stream.
    model.trace(True)
    model.trace_read()
    for s in range(args.steps):
        model.epoch(sig[args.warmup + s])
    kern_ms, launches = model.trace_read()
    model.trace(False)

    # ---------------- end to end through the public API from pinned host memory
    Yh = torch.from_numpy(prob.Y).pin_memory()
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    res_h = torch.zeros(1, dtype=torch.float64).pin_memory()

    def e2e_streamed(count):
        # every step: the H2D copy of its counts (issued during the previous step, so it overlaps that step's
        # epoch and deviance; the first one here), the epoch, and the D2H read of its FP64 deviance
        model.update_y_async(Yh)
        for s in range(count):
            model.epoch(sig[s])                     # sigma: 4 bytes per sweep
            model.deviance_async(res)
            res_h.copy_(res, non_blocking=True)     # D2H: 8 bytes
            if s + 1 < count:
                model.update_y_async(Yh)            # the next step's counts
            stream.synchronize()
            float(res_h.item())

    def e2e_serial(count):
        for s in range(count):
            model.update_y(Yh)                      # H2D (waits for the copy), on-device permutation
            model.epoch(sig[s])
            model.deviance()                        # D2H: the FP64 deviance (+ status word)

    e2e_steps = max(3, min(args.steps, 10))
    e2e = {}
    for name, fn in (("streamed", e2e_streamed), ("serial", e2e_serial)):
        fn(3)
        barrier()
        t0 = time.perf_counter()
        fn(e2e_steps)
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e[name] = whole_job_rate(entries_step * e2e_steps, ws, e2e_s)
    e2e_value = e2e["streamed"]
    launches_per_sweep = model.launches_per_sweep
    epoch_mode = model.epoch_mode
    del model
    # sweeps per traced launch, launches of this library per timed epoch
    sweeps_per_launch = nsw if epoch_mode == "persistent" else 1
    launches_per_epoch = 1 if epoch_mode == "persistent" else launches_per_sweep * nsw

    # ---------------- roofline of the dominant kernel (the tile launch of a sweep)
    peaks, peak_src = measured_peaks()
    ent_sweep, flops_sweep, bytes_sweep = sweep_algorithmic(w, K, fr, fc)
    ent_sweep, flops_sweep, bytes_sweep = (sweeps_per_launch * ent_sweep, sweeps_per_launch * flops_sweep,
                                           sweeps_per_launch * bytes_sweep)
    avg_kernel_s = (kern_ms / max(launches, 1)) / 1e3
    algo = {"entries": ent_sweep, "flops": flops_sweep, "bytes": bytes_sweep}
    if args.precision == "fp32":
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        peak = fp32_simt_peak_tflops(sm_mhz)
        achieved = flops_sweep / avg_kernel_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": committed_traffic("sweep_kernel", w.name), "kernel": "sweep_kernel (FP32 CUDA cores)",
                "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 flops x {sm_mhz:.0f} MHz",
                "hbm_gbs": bytes_sweep / avg_kernel_s / 1e9, "hbm_frac_of_measured": bytes_sweep / avg_kernel_s / 1e9 / peaks["hbm_gbs"]}
    else:
        achieved = bytes_sweep / avg_kernel_s / 1e9
        peak = float(peaks["hbm_gbs"])
        tc_peak = float(peaks.get("bf16_tflops", 1900.0))
        tc_kernel = {"persistent": "sweep_tc_epoch", "cluster": "sweep_tc_cluster"}.get(epoch_mode, "sweep_tc_kernel")
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": committed_traffic(tc_kernel, w.name),
                "kernel": tc_kernel + {"sweep_tc_epoch": f" (tcgen05, persistent: one launch = {nsw} sweeps)",
                                       "sweep_tc_cluster": " (tcgen05, strip updates in the same launch)"}.get(
                                           tc_kernel, " (tcgen05; the strip updates follow in update_kernel)"),
                "peak_source": f"{peak_src} STREAM-style copy (MEASURED_PEAKS.json hbm_gbs)",
                "tensor_tflops": flops_sweep / avg_kernel_s / 1e12, "tensor_peak_tflops": tc_peak,
                "tensor_frac_of_measured": flops_sweep / avg_kernel_s / 1e12 / tc_peak}
        # special-function work of the epilogue: exp per entry, and a reciprocal for the NB weight
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        sfu_ops = ent_sweep * (2 if w.family == "negbin" else 1) / avg_kernel_s
        roof.update({"sfu_ops_per_s": sfu_ops, "sfu_peak_ops_per_s": sfu_peak_ops(sm_mhz),
                     "sfu_frac": sfu_ops / sfu_peak_ops(sm_mhz),
                     "sfu_peak_source": f"derived: 152 SMs x 16 SFU results per clock x {sm_mhz:.0f} MHz"})
    roof.update({"avg_launch_us": avg_kernel_s * 1e6, "launches_timed": launches, "sweeps_per_launch": sweeps_per_launch,
                 "algorithmic_per_launch": algo})

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if args.precision == "fp32" else "bf16x3 eta + bf16 contractions, f32 accumulate/epilogue",
           "data": "synthetic (seeded NB GMF law; stands in for scRNA-seq counts)",
           "config": describe(w, args.precision), "roofline": roof,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(prob.Y.nbytes + 4 * nsw),
                   "api": "gmf_update_y_async (next step's counts copied during this step) + gmf_sgd_epoch + "
                          "gmf_deviance_async; with the synchronous gmf_update_y / gmf_deviance: "
                          f"{e2e['serial']:.4g} {UNIT}",
                   "d2h_bytes_per_step": 8},
           "gpu_launches": int(launches_per_epoch * args.steps), "epoch_mode": epoch_mode, "clocks": clk,
           "deviance": {"after_warmup": dev0, "after_timed_steps": dev1}}

    if extras:
        # ---------------- the other precision on the same workload
        other = "fp32" if args.precision == "mixed" else "mixed"
        mo = make(other)
        for s in range(args.warmup):
            mo.epoch(sig[s])
        oms = timed_epochs(mo, args.warmup, args.steps)
        out[f"{other}_path"] = {"value": entries_step * args.steps / (oms / 1e3), "ms_per_step": oms / args.steps}
        del mo
        if epoch_mode == "cluster":
            # ---------------- the same path as one persistent launch per epoch (GMF_FLAG_PERSIST)
            mo = make(args.precision, gmf.GMF_FLAG_PERSIST)
            if mo.epoch_mode == "persistent":
                for s in range(args.warmup):
                    mo.epoch(sig[s])
                oms = timed_epochs(mo, args.warmup, args.steps)
                out["persistent_epoch"] = {"value": entries_step * args.steps / (oms / 1e3),
                                           "ms_per_step": oms / args.steps}
            del mo
        # ---------------- time to the oracle's deviance (within 1e-3), both paths, fresh starts
        traj = {}
        if not args.no_ttd:
            tsig = synth.sweep_orders(w.n, w.m, w.nb_row, w.nb_col, w.epochs, args.seed)
            for prec in ("mixed", "fp32"):
                mdl = make(prec)
                devbuf = torch.zeros(w.epochs, dtype=torch.float64, device="cuda")
                evs = [torch.cuda.Event(enable_timing=True) for _ in range(w.epochs + 1)]
                barrier()
                evs[0].record(stream)
                for e in range(w.epochs):
                    mdl.epoch(tsig[e])
                    mdl.deviance_async(devbuf[e:e + 1])
                    evs[e + 1].record(stream)
                barrier()
                cum = [evs[0].elapsed_time(evs[e + 1]) / 1e3 for e in range(w.epochs)]
                traj[prec] = (devbuf.cpu().numpy().tolist(), cum)
                del mdl
        # the FP64 oracle's trajectory on a host core, after every GPU leg (it does not share the host with them)
        ores = None
        if not (args.no_cpu_baseline and args.no_ttd):
            ores = oracle_trajectory(w.name, args.seed)
        if ores is not None and not args.no_ttd:
            target = ores["final_deviance"] * (1 + 1e-3)
            ttd = {"oracle_final_deviance": ores["final_deviance"], "target": target, "epochs": w.epochs,
                   "includes_per_epoch_deviance": True, "start": "crude start (synth.crude_start), same sweep orders"}
            for prec, (devs, cum) in traj.items():
                hit = next((e for e, dv in enumerate(devs) if dv <= target), None)
                ttd[prec] = {"seconds": None if hit is None else cum[hit], "epochs": None if hit is None else hit + 1,
                             "final_deviance": devs[-1],
                             "final_rel_gap_to_oracle": devs[-1] / ores["final_deviance"] - 1.0}
            if ttd["mixed"]["seconds"] and ttd["fp32"]["seconds"]:
                ttd["fp32_over_mixed"] = ttd["fp32"]["seconds"] / ttd["mixed"]["seconds"]
            out["time_to_deviance"] = ttd
        if ores is not None and not args.no_cpu_baseline:
            times = ores["epoch_times"]
            k = next((i + 1 for i, t in enumerate(times) if t >= 12.0), len(times))
            out["cpu_baseline"] = {"value": k * ores["entries_per_epoch"] / times[k - 1], "unit": UNIT, "cores": 1,
                                   "kind": "oracle", **host_cpu(),
                                   "sample": f"first {k} epochs ({k * ores['entries_per_epoch']:.3g} entries) of the "
                                             f"same fit, FP64 single-threaded C on one host core, {times[k - 1]:.1f} s"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
