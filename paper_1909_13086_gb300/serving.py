"""Continuous-batching serving loop for cavity solves.

Requests (grid size, Rayleigh number, heated-strip position, storage precision,
step budget) arrive as a Poisson stream.  The server keeps every admitted
request's populations resident on the GPU.  Requests of one storage precision
and size class form a group: one ``Batch`` (one fused launch per step for all
members, graph-replayed) on the group's own CUDA stream, advanced in quanta of
``quantum`` steps.  Groups run concurrently, so small lattices never wait for
a large one's step, and the host polls each group's quantum by event: when it
completes, finished requests are retired (diagnostics read, memory freed), a
request whose lattice produced a non-finite value is reported as failed
without disturbing the others, and waiting requests are admitted while their
HBM footprint fits the budget -- requests that arrive while others are on the
GPU join as memory frees up, and their work overlaps on the device.

The baseline serves the same stream one request at a time, FIFO, in plain
FP32 (``sequential_fp32``).  Both report p50 / p99 time to result (completion
minus arrival) and aggregate MLUPS (cells x steps of all completed requests
over the makespan).

This module drives the C ABI only; the arithmetic is the CUDA library's.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import sys
import time

import numpy as np

from . import lbm, workloads

GRIDS = ((256, 128), (512, 256), (1024, 512), (2048, 1024))
RAS = (1e6, 1e7, 1e8)
CENTERS = (0.2, 0.35, 0.5, 0.65, 0.8)   # strip of width W/4 stays inside the wall


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the stream starts
    nx: int
    ny: int
    Ra: float
    center: float
    precision: str          # "fp32", "bf16sr", "fp16sr", ...
    steps: int

    def params(self) -> dict:
        return workloads.params(Ra=self.Ra, strip_center=self.center, seed=1000 + self.rid)

    @property
    def cells(self) -> int:
        return self.nx * self.ny


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    start: float
    finish: float
    ok: bool
    diag: dict
    fields: dict | None = None   # the final H, T, f_l, u fields (keep_fields=True)

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


def poisson_stream(n: int, rate_hz: float, seed: int = 7, steps: int = 2000,
                   precisions=("fp32", "bf16sr"), grids=GRIDS, ras=RAS, centers=CENTERS):
    """n requests with exponential inter-arrival times (rate_hz per second),
    grid, Ra, strip centre and precision drawn uniformly (seeded)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_hz)
        nx, ny = grids[rng.integers(len(grids))]
        out.append(Request(i, t, int(nx), int(ny), float(ras[rng.integers(len(ras))]),
                           float(centers[rng.integers(len(centers))]),
                           str(precisions[rng.integers(len(precisions))]), int(steps)))
    return out


ESIZE = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2, "fp16sr": 2, "bf16sr": 2}


def footprint_bytes(nx: int, ny: int, precision: str) -> int:
    """Device memory of one lattice: two buffers of 18 planes in 128-cell tiles,
    plus the per-block reduction scratch."""
    ntx = -(-nx // 128)
    pops = 2 * ntx * 128 * ny * 18 * ESIZE[precision]
    scratch = ntx * ny * 32 + max(ntx, ny) * 8 + 4096
    return pops + scratch


def size_class(nx: int, ny: int) -> int:
    """Requests are grouped by size so that small lattices never wait for a
    large lattice's step: 0 up to 256 x 128 cells, 1 up to 512 x 256, 2 up to
    1024 x 512, 3 above."""
    c = nx * ny
    return 0 if c <= 256 * 128 else (1 if c <= 512 * 256 else (2 if c <= 1024 * 512 else 3))


class Group:
    """One batch of same-precision, same-size-class requests on its own CUDA
    stream, with at most one quantum in flight.  The stream's priority rises as
    the size class falls: when SMs free up, the block scheduler serves the
    small lattices first (shortest work first), and the large ones take the
    rest of the GPU."""

    def __init__(self, max_batch: int, size_cls: int = 0, policy: str = "equal"):
        import torch

        prio = {"small_first": -(3 - size_cls), "large_first": -size_cls, "equal": 0}[policy]
        self.stream = torch.cuda.Stream(priority=prio)
        self.event = torch.cuda.Event()
        self.batch = lbm.Batch(max_batch, self.stream.cuda_stream)
        self.members: dict[int, tuple[Request, lbm.Lattice, float]] = {}
        self.remaining: dict[int, int] = {}
        self.inflight = 0  # steps of the quantum in flight (0: idle)

    def close(self):
        for _, lat, _ in self.members.values():
            lat.close()
        self.members.clear()
        self.batch.close()


class Server:
    """Continuous batching over resident lattices (see the module docstring)."""

    # Lattices of size class c admitted at once.  One 2048 x 1024 lattice fills
    # the GPU by itself (16,384 blocks), so large requests run one after the
    # other at full speed instead of sharing the GPU in lockstep -- which would
    # make an early request finish only with the last one -- while small ones,
    # far from filling it alone, are batched without limit.
    CLASS_CAP = {0: 1 << 30, 1: 8, 2: 2, 3: 1}

    def __init__(self, hbm_budget_bytes: int, quantum: int = 100, max_batch: int = 256,
                 autotune: bool = False, class_cap: dict | None = None, policy: str = "equal",
                 keep_fields: bool = False):
        self.class_cap = dict(self.CLASS_CAP if class_cap is None else class_cap)
        self.keep_fields = keep_fields
        self.policy = policy
        self.budget = int(hbm_budget_bytes)
        self.quantum = int(quantum)
        self.max_batch = max_batch
        self.autotune = autotune
        self.groups: dict[tuple[str, int], Group] = {}
        self.used = 0

    @property
    def active(self) -> int:
        return sum(len(g.members) for g in self.groups.values())

    def group(self, r: Request) -> Group:
        key = (r.precision, size_class(r.nx, r.ny))
        if key not in self.groups:
            self.groups[key] = Group(self.max_batch, key[1], self.policy)
        return self.groups[key]

    def can_admit(self, r: Request) -> bool:
        fp = footprint_bytes(r.nx, r.ny, r.precision)
        if fp > self.budget:
            raise ValueError(f"request {r.rid} needs {fp} B, more than the whole budget")
        cls = size_class(r.nx, r.ny)
        g = self.groups.get((r.precision, cls))
        if g is not None and (g.inflight or len(g.members) >= self.max_batch):
            return False  # membership changes wait for the group's quantum
        in_class = sum(len(h.members) for (_, c), h in self.groups.items() if c == cls)
        return in_class < self.class_cap[cls] and self.used + fp <= self.budget

    def admit(self, r: Request, now: float):
        g = self.group(r)
        lat = lbm.Lattice(r.nx, r.ny, r.params(), precision=r.precision, stream=g.stream.cuda_stream)
        if self.autotune:
            lbm.lbm_autotune(lat.h, 50)
        g.batch.add(lat)
        g.members[r.rid] = (r, lat, now)
        g.remaining[r.rid] = r.steps
        self.used += footprint_bytes(r.nx, r.ny, r.precision)

    def launch(self):
        """Start a quantum on every idle group that has members (asynchronous)."""
        for g in self.groups.values():
            if g.inflight or not g.members:
                continue
            q = min(self.quantum, min(g.remaining.values()))
            g.batch.step(q)
            g.event.record(g.stream)
            g.inflight = q

    def poll(self, now_fn, block: bool = False) -> list[Result]:
        """Finish the quanta that completed (all of them when block=True):
        retire finished requests -- diagnostics read, lattice freed -- and
        report a request whose lattice holds a non-finite value as failed."""
        done = []
        for g in self.groups.values():
            if not g.inflight:
                continue
            if block:
                g.event.synchronize()
            elif not g.event.query():
                continue
            for rid in g.remaining:
                g.remaining[rid] -= g.inflight
            g.inflight = 0
            for rid in [k for k, v in g.remaining.items() if v <= 0]:
                r, lat, start = g.members.pop(rid)
                del g.remaining[rid]
                d = lat.diagnostics(raise_on_diverged=False)
                fields = lat.fields(("H", "T", "fl", "ux", "uy")) if self.keep_fields else None
                done.append(Result(rid, r.arrival, start, now_fn(), d["nan_flag"] == 0, d, fields))
                g.batch.remove(lat)
                lat.close()
                self.used -= footprint_bytes(r.nx, r.ny, r.precision)
        return done

    def busy(self) -> bool:
        return any(g.inflight for g in self.groups.values())

    def close(self):
        for g in self.groups.values():
            g.close()
        self.groups.clear()


def serve(requests, hbm_budget_bytes: int, quantum: int = 100, autotune: bool = False,
          clock=time.perf_counter, max_batch: int = 256, class_cap: dict | None = None,
          policy: str = "equal", keep_fields: bool = False):
    """Serve a request stream with continuous batching; arrivals are replayed
    in real time relative to the start.  Returns (results, makespan_s).
    keep_fields: each result also carries its lattice's final fields."""
    pending = sorted(requests, key=lambda r: r.arrival)
    # Lattices come and go while other groups run: take their memory from the
    # caching allocator, since cudaFree would wait for the whole device.
    lbm.use_torch_allocator()
    srv = Server(hbm_budget_bytes, quantum, max_batch=max_batch, autotune=autotune,
                 class_cap=class_cap, policy=policy, keep_fields=keep_fields)
    t0 = clock()
    now = lambda: clock() - t0  # noqa: E731
    results: list[Result] = []
    i = 0
    waiting: list[Request] = []
    try:
        while i < len(pending) or waiting or srv.active:
            t = now()
            while i < len(pending) and pending[i].arrival <= t:
                waiting.append(pending[i])
                i += 1
            # admission by HBM footprint, first come first served (a request
            # whose group is mid-quantum waits for it; later ones may pass it)
            still = []
            for r in waiting:
                if srv.can_admit(r):
                    srv.admit(r, now())
                else:
                    still.append(r)
            waiting = still
            srv.launch()
            if srv.busy():
                got = srv.poll(now)
                results += got
                if not got:
                    time.sleep(20e-6)
            elif not srv.active and i < len(pending):
                time.sleep(max(0.0, pending[i].arrival - now()))
    finally:
        srv.close()
        lbm.use_default_allocator()
    return results, now()


def sequential_fp32(requests, stream: int | None = None, clock=time.perf_counter):
    """Baseline: one request at a time, FIFO, plain FP32 (lbm_step)."""
    pending = sorted(requests, key=lambda r: r.arrival)
    t0 = clock()
    now = lambda: clock() - t0  # noqa: E731
    results = []
    for r in pending:
        if now() < r.arrival:
            time.sleep(r.arrival - now())
        start = now()
        lat = lbm.Lattice(r.nx, r.ny, r.params(), precision="fp32", stream=stream)
        lat.step(r.steps)
        d = lat.diagnostics(raise_on_diverged=False)
        results.append(Result(r.rid, r.arrival, start, now(), d["nan_flag"] == 0, d))
        lat.close()
    return results, now()


def summarize(results, requests, makespan: float) -> dict:
    by_id = {r.rid: r for r in requests}
    lat = np.array([x.latency for x in results])
    work = sum(by_id[x.rid].cells * by_id[x.rid].steps for x in results)
    return {"requests": len(results), "failed": int(sum(not x.ok for x in results)),
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "mlups": work / makespan / 1e6 if makespan > 0 else None,
            "makespan_s": makespan}


def main(argv=None):
    ap = argparse.ArgumentParser(description="serve a Poisson stream of cavity solves")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--rate", type=float, default=40.0, help="arrivals per second")
    ap.add_argument("--steps", type=int, default=2000, help="step budget of every request")
    ap.add_argument("--quantum", type=int, default=100)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--precisions", default="fp32,bf16sr")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--no-baseline", action="store_true")
    args = ap.parse_args(argv)
    import torch

    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    reqs = poisson_stream(args.requests, args.rate, args.seed, args.steps,
                          tuple(args.precisions.split(",")))
    res, mk = serve(reqs, int(args.budget_gb * 2 ** 30), args.quantum)
    out = {"mode": "continuous batching", **summarize(res, reqs, mk),
           "precisions": args.precisions, "rate_hz": args.rate, "steps": args.steps}
    print(json.dumps(out), flush=True)
    if not args.no_baseline:
        res_b, mk_b = sequential_fp32(reqs, s.cuda_stream)
        print(json.dumps({"mode": "sequential fp32", **summarize(res_b, reqs, mk_b)}), flush=True)


if __name__ == "__main__":
    main()
