#!/usr/bin/env python3
"""Throughput of the fused B-TriRT sweep on the 2048 x 1024 production cavity.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one fused collide-and-stream sweep (pull streaming with the wall
rules, H -> (T, f_l) inversion, g and f block collisions, buoyancy, the
per-step heated-wall inflow reduction) over the whole 2048 x 1024 lattice in
FP32; the FP64 diagnostics reductions (melt fraction, sum H, max |u|, NaN
flag) are fused into every 100th sweep, the cadence of the melt-fraction and
Nusselt history.  Metric: MLUPS (million lattice-cell updates per second; one
update advances both f and g of one cell).  The working set (2 x 151 MB of
populations) is larger than L2, so no flush is needed between steps.

For N > 1 (torchrun) every rank advances its own cavity (replicas: the method
needs no exchange between independent solves); value = all cells updated by
all ranks / the slowest rank's time.

--impl reference times the FP64 CPU oracle on this host's cores and prints
the same JSON line: each step advances a band of the cavity's rows (same
width, parameters and per-cell work) sized so that the whole run takes about
two minutes; the full 1024 rows when K is small.

The default run also serves a seeded Poisson stream of cavity requests
(mixed grids, Rayleigh numbers and strip positions) with continuous batching
in BF16 storage with stochastic rounding and, for comparison, one request at a
time in plain FP32, and reports under "serving" the p50 / p99 time to result,
the aggregate MLUPS and the 16-bit results' largest melt-fraction and Nusselt
differences from an FP64 run of the same requests.

--batch N times the batched path instead: N cavities of 256 x 128 (the
serving size; Ra and strip centre varied, seeded) advanced together, one fused
launch per step over all of them (graph-replayed); the last step carries the
diagnostics.  Same JSON line, device-resident timing only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 2048, 1024
BYTES_PER_LUP = {"fp32": 144, "fp64": 288, "fp16": 72, "bf16": 72, "fp16sr": 72, "bf16sr": 72}  # 18 read + 18 written
DIAG_EVERY = 100
METRIC = "MLUPS"
FALLBACK_HBM_GBS = 6800.0
L2_MB = 129.0  # GB300 L2 capacity
REFERENCE_BUDGET_S = 120.0  # timed oracle work of one --impl reference run
# FP64 operations (adds, subtracts, multiplies, one divide; an FMA counts as
# two) in one interior-cell update as the sweep writes it out: macroscopic
# fields with the raw moments of f 41, g collision 90, f collision 96.
FP64_FLOPS_PER_LUP = 227
# GB300 FP64 pipe: 2 FMA per clock per SM, 2 flops each, 152 SMs, 2070 MHz.
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1909_13086_gb300", "csrc", f)
                  for f in ("sweep.cuh", "lbm_internal.h")]


def sweep_launches(warmup: int, steps: int) -> int:
    """Kernels launched by lbm_step(steps) after `warmup` steps: one sweep per
    step, plus the one-block diagnostics fold after every diagnostic sweep
    (every DIAG_EVERY-th step and the last one)."""
    diag = {n for n in range(warmup + 1, warmup + steps + 1) if n % DIAG_EVERY == 0}
    diag.add(warmup + steps)
    return steps + len(diag)


def workload_config(precision: str) -> dict:
    one = precision != "fp64"   # the library's default streaming (lbm_set_streaming)
    mb = BYTES_PER_LUP[precision] * NX * NY / 2 / 1e6      # one buffer of populations
    return {"workload": f"cavity {NX}x{NY}, Ra 1e8, Pr 1, Ste 1, Ma 0.1, strip W/4 centred, "
                        f"{precision.upper()} populations",
            "nx": NX, "ny": NY, "precision": precision,
            "diagnostics": f"fused every {DIAG_EVERY} steps; heated-wall flux every step",
            "streaming": ("one buffer (push / local sweeps), the call's last 1-2 sweeps over two buffers"
                          if one else "two buffers"),
            "l2": (f"inputs larger than L2 ({mb:.0f} MB of populations in the buffer a step reads and "
                   "writes), no flush" if one and mb > L2_MB else
                   f"the populations ({mb:.0f} MB in the one buffer a step reads and writes) fit in the "
                   f"{L2_MB:.0f} MB L2: a step reads what the previous one wrote, no flush" if one else
                   f"inputs larger than L2 (2 x {mb:.0f} MB populations), no flush")}


# ------------------------------------------------------------ distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_group(ws: int, backend: str):
    if ws <= 1:
        return None
    import torch.distributed as dist

    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def aggregate(elapsed_s: float, units: float, dist, device=None) -> tuple[float, float]:
    """Max of the per-rank times and sum of the per-rank units."""
    if dist is None:
        return elapsed_s, units
    import torch

    t = torch.tensor([elapsed_s, units], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


# ------------------------------------------------------------ measurement aids
def measured_peak_gbs() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for key in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
            if key in d:
                return float(d[key]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_path(precision: str, batch: int = 0) -> str:
    name = f"batch_{precision}_{batch}x256x128.md" if batch else f"sweep_{precision}_cavity_2048x1024.md"
    return os.path.join(ROOT, "profiles", name)


def profiled_traffic(precision: str = "fp32", batch: int = 0) -> float | None:
    """DRAM bytes per launch of the sweep in `precision` (of the batch kernel
    over `batch` lattices) from the committed ncu summary, if it was taken on
    the current kernel source."""
    try:
        text = open(profile_path(precision, batch)).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    m_traf = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_traf or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_traf.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle sampling around the timed region: a sample
    just before, one every 100 ms while the block runs (the warm-up and the
    timed steps), and one just after."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.bracket = []
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def once(self) -> list:
        """One sample, taken now (the timed region may be too short for the
        100 ms loop to record any)."""
        try:
            out = subprocess.run(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                 timeout=10).stdout
        except (OSError, subprocess.SubprocessError):
            return []
        return [[p.strip() for p in line.split(",")] for line in out.splitlines()
                if len(line.split(",")) >= 9]

    def __enter__(self):
        self.bracket = self.once()
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()
        self.bracket += self.once()

    def summary(self) -> dict:
        rows = []
        if self.proc is not None:
            try:
                for line in open(self.path):
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            except OSError:
                pass
        inside = len(rows)
        # the median is over the samples inside the timed region when there are
        # any, else over the two taken just before and just after it
        use = rows if rows else self.bracket
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = sorted(float(r[1]) for r in use if r[1].replace(".", "").isdigit())
        smax = max(float(r[2]) for r in rows + self.bracket if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows + self.bracket for n, v in zip(names, r[5:9])
                          if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": inside, "bracket_samples": len(self.bracket),
                "median_of": "warm-up and timed region" if rows else
                "samples just before and after the warm-up and timed region"}


# ------------------------------------------------------------ CPU oracle arm
def oracle_mlups(steps: int, warmup: int, threads: int, rows: int = NY) -> tuple[float, float, int]:
    """Time the FP64 oracle on the same workload, or on a band of `rows` of its
    rows: the same width, the same derived parameters (nu, alpha, g beta, the
    rates and the strip, all those of the full 2048 x 1024 cavity) and the same
    per-cell work.  Returns (MLUPS, seconds, steps)."""
    from oracle import oracle as O
    from paper_1909_13086_gb300 import workloads

    nx, ny, p = workloads.cavity_2048x1024()
    if rows < ny:
        # The cavity mapping takes its reference length from the height; give
        # the band the full cavity's alpha directly and the Rayleigh number that
        # reproduces its g beta over the band's height.
        d = O.derive(nx, ny, **p)
        rows = max(2, rows)
        p = dict(p, alpha_override=d.alpha, Ra=d.gbeta * rows ** 3 / (d.nu * d.alpha))
        ny = rows
    o = O.Oracle(nx, ny, threads=threads, **p)
    if warmup:
        o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return nx * ny * steps / dt / 1e6, dt, steps


def cpu_baseline_sample(threads: int) -> dict:
    """A bounded sample (about 10-20 s) of the oracle on this host."""
    from oracle import oracle as O

    O.build()
    # one step first, to size the sample
    rate1, dt1, _ = oracle_mlups(1, 0, threads)
    steps = max(2, min(200, int(12.0 / max(dt1, 1e-3))))
    rate, dt, n = oracle_mlups(steps, 0, threads)
    return {"value": round(rate, 3), "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"{n} FP64 oracle steps of the {NX}x{NY} cavity ({dt:.1f} s, "
                      f"{threads} OpenMP threads)"}


def run_reference(args) -> None:
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O

    O.build()
    threads = os.cpu_count() or 1
    # Each bench step is a bounded sample of the workload: the oracle advances
    # a band of the cavity's rows (same width, parameters and per-cell work),
    # as many as let the W + K steps finish in about REFERENCE_BUDGET_S.
    _, t1, _ = oracle_mlups(1, 0, threads)
    per_row = t1 / NY
    rows = int(REFERENCE_BUDGET_S / max(args.steps + args.warmup, 1) / per_row)
    rows = max(8, min(NY, rows))
    rate, dt, n = oracle_mlups(args.steps, args.warmup, threads, rows)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(rate, 3), "unit": METRIC,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / n * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # the same workload and config as this arm's GPU line; the oracle
        # computes it in FP64 (dtype)
        "config": workload_config(args.precision),
        "cpu_baseline": {"value": round(rate, 3), "unit": METRIC, "cores": threads,
                         "kind": "oracle",
                         "sample": f"{n} FP64 oracle steps of rows 0..{rows - 1} of the {NX}x{NY} "
                                   f"cavity ({NX}x{rows} cells per step, {dt:.1f} s)"},
        "e2e": {"value": round(rate, 3), "unit": METRIC, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def measure_e2e(args, lat, p, prec, stream, dist, local) -> dict:
    """End to end through the C ABI with host buffers: upload the state from
    pinned host memory, run the steps, read every step's result (its
    heated-wall inflow / Nusselt number, and the melt fraction on diagnostic
    steps) from the device history ring, read the final fields back."""
    import torch

    from paper_1909_13086_gb300 import lbm

    nx, ny = lat.nx, lat.ny
    cells = nx * ny
    f0, g0, _ = lat.populations()
    e2e_lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream.cuda_stream)
    lbm.lbm_set_diag_every(e2e_lat.h, DIAG_EVERY)
    e2e_steps = max(1, args.steps)
    lbm.lbm_set_history(e2e_lat.h, e2e_steps + 1)
    f_host = torch.from_numpy(f0).pin_memory().numpy()
    g_host = torch.from_numpy(g0).pin_memory().numpy()
    out = {k: torch.empty((ny, nx), dtype=torch.float64).pin_memory().numpy()
           for k in ("H", "T", "fl", "ux", "uy", "rho")}
    e2e_lat.set_populations(f_host, g_host, 0)  # first upload: staging allocated outside the timing
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_lat.set_populations(f_host, g_host, 0)
    e2e_lat.step(e2e_steps)
    hist = lbm.lbm_read_history(e2e_lat.h, e2e_steps + 1)
    lbm.lbm_read_fields(e2e_lat.h, 63, *[out[k] for k in ("H", "T", "fl", "ux", "uy", "rho")])
    t_e2e = time.perf_counter() - t0
    assert len(hist["step"]) == e2e_steps
    t_e2e_max, e2e_units = aggregate(t_e2e, float(cells * e2e_steps), dist,
                                     device=torch.device("cuda", local))
    h2d = f_host.nbytes + g_host.nbytes
    d2h = (e2e_steps + 1) * 32 + sum(a.nbytes for a in out.values())  # the whole ring
    e2e_lat.close()
    return {"value": round(e2e_units / t_e2e_max / 1e6, 1), "unit": METRIC,
            "h2d_bytes_per_step": int(h2d / e2e_steps), "d2h_bytes_per_step": int(d2h / e2e_steps),
            "steps": e2e_steps,
            "path": "lbm_write_populations (pinned host FP64 state) + lbm_step(K) + lbm_read_history "
                    "(every step's Q/Nu, melt every 100) + lbm_read_fields(all six)"}


# ------------------------------------------------------------ GPU arm
def run_ours(args) -> None:
    import numpy as np
    import torch

    from paper_1909_13086_gb300 import lbm, workloads

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_group(ws, "nccl")
    # A dedicated (non-default) stream: the library enqueues on it and the
    # CUDA events below are recorded on it.
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    nx, ny, p = workloads.cavity_2048x1024()
    prec = args.precision
    cells = nx * ny

    lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream.cuda_stream)
    lbm.lbm_set_diag_every(lat.h, DIAG_EVERY)

    # ---- device-resident timing: K sweeps, inputs already in HBM.  The clock
    # sampler starts before the warm-up, so that starting nvidia-smi does not
    # leave the GPU idle just before the timed region.
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        lat.step(args.warmup)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        start.record(stream)
        lat.step(args.steps)
        stop.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = start.elapsed_time(stop) / 1e3
    t_max, units = aggregate(elapsed, float(cells * args.steps), dist,
                             device=torch.device("cuda", local))
    value = units / t_max / 1e6
    d = lat.diagnostics()
    assert d["nan_flag"] == 0

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, lat, p, prec, stream, dist, local)

    # ---- roofline of the sweep (the only kernel in the timed region)
    peak, peak_kind = measured_peak_gbs()
    kernel_s = elapsed / args.steps
    alg_bytes = BYTES_PER_LUP[prec] * cells
    achieved = alg_bytes / kernel_s / 1e9
    traffic = profiled_traffic(prec)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": f"{peak_kind} HBM copy bandwidth",
                "algorithmic_bytes_per_launch": alg_bytes}
    if traffic:
        # The DRAM side: the profiled bytes per launch (warm L2, as in this
        # loop) over the measured time.  A step that starts on rows the
        # previous one left in L2 moves fewer bytes than it reads and writes,
        # so `frac` (algorithmic bytes) can exceed 1 while this stays below.
        roofline["dram_achieved"] = round(traffic / kernel_s / 1e9, 1)
        roofline["dram_frac"] = round(traffic / kernel_s / 1e9 / peak, 4)
    if prec == "fp64":
        # the FP64 sweep is bound by GB300's FP64 pipe, not by HBM
        flops = FP64_FLOPS_PER_LUP * cells
        tflops = flops / kernel_s / 1e12
        roofline = {"bound": "alu", "achieved": round(tflops, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                    "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                    "traffic": profiled_traffic(prec),
                    "peak_source": "derived: 152 SMs x 2 FP64 FMA/clock x 2 flops x 2070 MHz",
                    "algorithmic_flops_per_launch": flops, "hbm_achieved_gbs": round(achieved, 1)}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": METRIC, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_max / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f32 (f16 storage)",
                  "bf16": "f32 (bf16 storage)", "fp16sr": "f32 (f16 storage, stochastic rounding)",
                  "bf16sr": "f32 (bf16 storage, stochastic rounding)"}[prec], "data": "synthetic",
        "config": workload_config(prec),
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": sweep_launches(args.warmup, args.steps),
        "clocks": clocks.summary(),
        "melt_fraction": d["melt_fraction"],
    }
    if ws == 1 and not args.no_serving:
        line["serving"] = serving_leg()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(os.cpu_count() or 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    lat.close()
    if dist:
        dist.destroy_process_group()


# Serving leg of the default run: a seeded Poisson stream of cavity requests
# (grids 256 x 128 to 2048 x 1024, Ra 1e6 / 1e7 / 1e8, strip centre at five
# positions) served with continuous batching in 16-bit storage with stochastic
# rounding, against the same stream served one request at a time in plain FP32.
SERVING = dict(requests=32, rate_hz=40.0, steps=2000, precision="bf16sr", seed=7, budget_gb=64.0,
               quantum=100)


def serving_leg() -> dict:
    """p50 / p99 time to result and aggregate MLUPS of both servers, and the
    accuracy of the batched 16-bit results: every request is also advanced in
    FP64 on the GPU (batched by grid size), and the largest differences in the
    final melt fraction and in the mean Nusselt number over the run (from the
    cumulative heated-wall inflow; the one-step inflow carries the rounding
    noise of a few hundred wall populations) are reported."""
    import torch

    from paper_1909_13086_gb300 import lbm, serving

    cfg = SERVING
    reqs = serving.poisson_stream(cfg["requests"], cfg["rate_hz"], cfg["seed"], cfg["steps"],
                                  precisions=(cfg["precision"],))
    res_b, mk_b = serving.serve(reqs, int(cfg["budget_gb"] * 2 ** 30), cfg["quantum"])
    s = torch.cuda.Stream()
    res_s, mk_s = serving.sequential_fp32(reqs, s.cuda_stream)
    batched = serving.summarize(res_b, reqs, mk_b)
    sequential = serving.summarize(res_s, reqs, mk_s)
    # FP64 reference of every request, one batch per grid size
    by_id = {x.rid: x for x in res_b}
    melt_err, nu_err = 0.0, 0.0
    for nx, ny in sorted({(r.nx, r.ny) for r in reqs}):
        group = [r for r in reqs if (r.nx, r.ny) == (nx, ny)]
        lats = [lbm.Lattice(nx, ny, r.params(), precision="fp64", stream=s.cuda_stream) for r in group]
        b = lbm.Batch(len(lats), s.cuda_stream)
        for lat in lats:
            b.add(lat)
        b.step(cfg["steps"])
        for r, lat in zip(group, lats):
            d64, d16 = lat.diagnostics(), by_id[r.rid].diag
            melt_err = max(melt_err, abs(d16["melt_fraction"] - d64["melt_fraction"]))
            # mean Nu over the run is Q_cum times a constant of the request
            nu_err = max(nu_err, abs(d16["Q_cum"] - d64["Q_cum"]) / abs(d64["Q_cum"]))
        b.close()
        for lat in lats:
            lat.close()
    return {
        "stream": f"{cfg['requests']} Poisson requests at {cfg['rate_hz']:g}/s, {cfg['steps']} steps "
                  "each, grids 256x128 / 512x256 / 1024x512 / 2048x1024, Ra 1e6 / 1e7 / 1e8, strip "
                  "centre 0.2-0.8 W (seeded)",
        "batched": {"precision": cfg["precision"], "mode": "continuous batching", **batched},
        "sequential": {"precision": "fp32", "mode": "one request at a time, FIFO", **sequential},
        "p99_ratio": sequential["p99_s"] / batched["p99_s"],
        "mlups_ratio": batched["mlups"] / sequential["mlups"],
        "melt_err_max_vs_fp64": melt_err,
        "mean_nu_rel_err_max_vs_fp64": nu_err,
    }


BATCH_NX, BATCH_NY = 256, 128


def run_batch(args) -> None:
    import numpy as np
    import torch

    from paper_1909_13086_gb300 import lbm, workloads

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec, n = args.precision, args.batch
    rng = np.random.default_rng(7)
    lats = [lbm.Lattice(BATCH_NX, BATCH_NY,
                        workloads.params(Ra=float(rng.choice([1e6, 1e7, 1e8])),
                                         strip_center=float(rng.choice([0.2, 0.35, 0.5, 0.65, 0.8])),
                                         strip_width=0.25, seed=int(k)),
                        precision=prec, stream=stream.cuda_stream) for k in range(n)]
    b = lbm.Batch(n, stream.cuda_stream)
    for lat in lats:
        b.add(lat)
    # launch shape picked by the batch autotuner (scratch lattices, untimed)
    tuned = lbm.lbm_batch_autotune(b.b, 50) if not args.no_autotune else None
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        b.step(args.warmup)
        torch.cuda.synchronize()
        start.record(stream)
        b.step(args.steps)
        stop.record(stream)
        torch.cuda.synchronize()
    elapsed = start.elapsed_time(stop) / 1e3
    cells = n * BATCH_NX * BATCH_NY
    kernel_s = elapsed / args.steps
    alg_bytes = BYTES_PER_LUP[prec] * cells
    peak, peak_kind = measured_peak_gbs()
    achieved = alg_bytes / kernel_s / 1e9
    nan = sum(lat.diagnostics(raise_on_diverged=False)["nan_flag"] for lat in lats)
    assert nan == 0
    line = {
        "metric": METRIC, "value": round(cells * args.steps / elapsed / 1e6, 1), "unit": METRIC,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(kernel_s * 1e3, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": f"batch of {n} cavities {BATCH_NX}x{BATCH_NY} (Ra 1e6-1e8, strip "
                               f"W/4 at 0.2-0.8 W, seeded), {prec.upper()} populations, one fused "
                               "launch per step", "lattices": n, "precision": prec,
                   "streaming": ("one buffer (push / local sweeps), the call's last 1-2 steps over two buffers"
                                 if prec != "fp64" else "two buffers"),
                   # a step reads and writes every population once: half the algorithmic bytes
                   # is the state; with two buffers the step touches twice that
                   "l2": (f"inputs larger than L2 ({alg_bytes / 1e6:.0f} MB of populations in the two "
                          "buffers), no flush" if prec == "fp64" else
                          f"inputs larger than L2 ({alg_bytes / 2e6:.0f} MB of populations in the buffer "
                          "a step reads and writes), no flush" if alg_bytes / 2 > L2_MB * 1e6 else
                          f"the populations ({alg_bytes / 2e6:.0f} MB in the one buffer a step reads and "
                          f"writes) fit in the {L2_MB:.0f} MB L2: a step reads what the previous one "
                          "wrote, no flush"),
                   "launch": ({"rows": tuned["rows"], "prefetch": tuned["prefetch"],
                               "interleave": tuned["interleave"], "by": "lbm_batch_autotune"}
                              if tuned else "default")},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": profiled_traffic(prec, n),
                     "peak_source": f"{peak_kind} HBM copy bandwidth",
                     "algorithmic_bytes_per_launch": alg_bytes},
        "e2e": None,
        "gpu_launches": args.steps + 1,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    b.close()
    for lat in lats:
        lat.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("fp32", "fp64", "fp16", "bf16", "fp16sr", "bf16sr"), default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-autotune", action="store_true", help="--batch: keep the default launch shape")
    ap.add_argument("--batch", type=int, default=0,
                    help=f"time a batch of this many {BATCH_NX}x{BATCH_NY} cavities instead")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.batch > 0:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
