"""The paper's two studies, run on the GPU through the C ABI.

* ``stefan_k1_sweep`` -- Sec. 3.1 (Figs. 1-2 as numbers): one-phase melting by
  conduction, T_h = 1, T_m = 0, Ste = 0.01, alpha = 1/6, dx = 1/100, profiles
  at t = 25, for k1 in {0.1, 0.5, 1.0, 1.5} (k1 = 2.0 has no positive
  diffusivity, Eq. 5), B-TriRT with k2 = 2 - k1 (Eq. 6) against SRT
  (k0 = k1 = k2).  Reported per run: the largest temperature error against
  the Neumann solution (Eqs. 7-8), the largest departure of the solid ahead of
  the front from T_m, the interface width (cells with 0 < f_l < 1 in a row)
  and the front position against 2 lambda sqrt(alpha t).
* ``cavity_location_sweep`` -- Sec. 3.2 (Fig. 3b): the melt-fraction history
  of the cavity heated from below at Ra 1e8, Pr 6.2, Ste 0.125, D = 0.5 L,
  512 x 512, for strip centres C = 0.25, 0.375, 0.5 L, up to a given Fourier
  number (full melting needs ~6.6e7 steps per run at Ma 0.1).
* ``cavity_full_melt`` -- the same three cavities advanced together in one
  batch until each is fully melted (melt fraction >= 0.99, the reading of
  "full melting" used here), with the Fourier number at which each crosses
  0.5, 0.9, 0.95 and 0.99: the ordering the paper reports (Sec. 3.2, Sec. 4)
  is that the centred strip melts the cavity first.  Long runs resume from a
  checkpoint of the FP32 (or FP64) populations.
* ``precision_study`` -- the storage precisions against the FP64 path on the
  2048 x 1024 cavity heated from below (Ra 1e8, Pr 1, Ste 1, strip a quarter
  of the width) at several strip centres: the largest melt-fraction difference
  over the run and the relative difference of the time-mean Nusselt number.

Lattice units (reading of Sec. 3.1's mixed units): dt follows from k1 through
Eq. 5, dt = dx^2 (1/k1 - 1/2) / (3 alpha), so t = 25 is 25 / dt steps and the
front X(t) = 2 lambda sqrt(alpha t) becomes X / dx cells.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import lbm, workloads

PAPER_STEFAN = dict(Th=1.0, Tm=0.0, Ste=0.01, alpha=1.0 / 6.0, dx=0.01, t=25.0, k1=(0.1, 0.5, 1.0, 1.5))


def stefan_lambda(Ste: float) -> float:
    """Root of Eq. 8, Ste / (exp(l^2) erf(l)) = l sqrt(pi), by bisection."""
    f = lambda l: l * math.sqrt(math.pi) * math.exp(l * l) * math.erf(l) - Ste  # noqa: E731
    lo, hi = 0.0, 1.0
    while f(hi) < 0:
        hi *= 2
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
    return 0.5 * (lo + hi)


def neumann_T(x, t, alpha, lam, Th=1.0, Tm=0.0):
    """Eq. 7 (x, t in any consistent units)."""
    X = 2 * lam * math.sqrt(alpha * t)
    s = 2 * math.sqrt(alpha * t)
    return np.where(x < X, Th - (Th - Tm) * np.vectorize(math.erf)(x / s) / math.erf(lam), Tm)


def stefan_run(k1: float, model: str, nx: int = 100, precision: str = "fp64", stream=None,
               p=PAPER_STEFAN) -> dict:
    dx, alpha_phys = p["dx"], p["alpha"]
    dt = dx * dx * (1.0 / k1 - 0.5) / (3.0 * alpha_phys)
    steps = int(round(p["t"] / dt))
    alpha_lu = (1.0 / k1 - 0.5) / 3.0
    k2 = 2.0 - k1 if model == "btrirt" else k1
    k0 = 1.0 if model == "btrirt" else k1
    _, ny, prm = workloads.stefan_1024x4(Ste=p["Ste"], alpha=alpha_lu, k2=k2, k0=k0, nx=nx)
    lat = lbm.Lattice(nx, ny, prm, precision=precision, stream=stream)
    lat.step(steps)
    F = lat.fields(("T", "fl", "H"))
    T, fl = F["T"][0], F["fl"][0]
    lam = stefan_lambda(p["Ste"])
    x = (np.arange(nx) + 0.5) * dx
    t = steps * dt
    Tn = neumann_T(x, t, alpha_phys, lam, p["Th"], p["Tm"])
    X = 2 * lam * math.sqrt(alpha_phys * t)
    melted = np.nonzero(fl > 1e-12)[0]
    edge = melted.max() if melted.size else -1
    ahead = T[edge + 1:]
    mushy = ((F["fl"] > 1e-12) & (F["fl"] < 1 - 1e-12)).sum(axis=1)
    d = lat.diagnostics()
    lat.close()
    return {"k1": k1, "model": model, "steps": steps,
            "max_T_error": float(np.abs(T - Tn).max()),
            "solid_departure_from_Tm": float(np.abs(ahead).max(initial=0.0)),
            "interface_width_cells": int(mushy.max()),
            "front_cells": d["front_x"], "front_neumann_cells": X / dx}


def stefan_k1_sweep(precision: str = "fp64", stream=None) -> list[dict]:
    return [stefan_run(k1, m, precision=precision, stream=stream)
            for k1 in PAPER_STEFAN["k1"] for m in ("btrirt", "srt")]


def cavity_location_sweep(fo_end: float = 0.01, n: int = 512, centers=(0.25, 0.375, 0.5),
                          samples: int = 20, precision: str = "fp32", stream=None) -> dict:
    """Melt-fraction history at the paper's cavity parameters (Sec. 3.2)."""
    out = {}
    for C in centers:
        p = workloads.params(Ra=1e8, Pr=6.2, Ste=0.125, strip_center=C, strip_width=0.5)
        lat = lbm.Lattice(n, n, p, precision=precision, stream=stream)
        alpha = lat.derived()["alpha"]
        steps_total = int(round(fo_end * n * n / alpha))
        chunk = max(1, steps_total // samples)
        hist = []
        for _ in range(samples):
            lat.step(chunk)
            d = lat.diagnostics(raise_on_diverged=False)
            hist.append((d["step"] * alpha / (n * n), d["melt_fraction"], d["Nu"], d["nan_flag"]))
        out[C] = hist
        lat.close()
    return out


# The storage study: 2e5 steps of the 2048 x 1024 cavity, sampled every 1000.
PRECISION_STUDY = dict(nx=2048, ny=1024, steps=200_000, every=1000, centers=(0.25, 0.5, 0.75),
                       precisions=("fp32", "fp16", "bf16", "fp16sr", "bf16sr"))


def run_history(lat, steps: int, every: int) -> dict:
    """Advance `lat` by `steps` in pieces of at most `every`, sampling the melt
    fraction after each piece; also the final cumulative heated-wall inflow."""
    melt, done = [], 0
    while done < steps:
        k = min(every, steps - done)
        lat.step(k)
        done += k
        melt.append(lat.diagnostics(raise_on_diverged=False)["melt_fraction"])
    d = lat.diagnostics(raise_on_diverged=False)
    return {"melt": melt, "Q_cum": d["Q_cum"], "final_melt": d["melt_fraction"],
            "nan_flag": d["nan_flag"]}


def compare_to_fp64(ref: dict, run: dict) -> dict:
    """The largest melt-fraction difference over the samples, and the relative
    difference of the time-mean Nusselt number: Nu is the inflow times the same
    constant for both runs, so the mean of Nu over the run compares as the
    cumulative inflow Q_cum does."""
    m64, m = np.asarray(ref["melt"], np.float64), np.asarray(run["melt"], np.float64)
    if m64.shape != m.shape:
        raise ValueError("the two runs were sampled differently")
    return {"melt_err_max": float(np.abs(m - m64).max()) if m.size else 0.0,
            "mean_nu_rel_err": (run["Q_cum"] / ref["Q_cum"] - 1.0) if ref["Q_cum"] != 0.0 else math.nan,
            "final_melt": run["final_melt"], "final_melt_fp64": ref["final_melt"],
            "nan_flag": run["nan_flag"]}


def precision_study(nx: int = 2048, ny: int = 1024, steps: int = 200_000, every: int = 1000,
                    centers=(0.25, 0.5, 0.75), precisions=PRECISION_STUDY["precisions"],
                    stream=None, make_lattice=None) -> list[dict]:
    """Each storage precision against the FP64 path, strip centre by strip
    centre (one row per centre and precision).  make_lattice(C, precision)
    replaces the GPU lattice (host tests)."""
    if make_lattice is None:
        def make_lattice(C, precision):
            p = workloads.params(Ra=1e8, strip_center=C)
            return lbm.Lattice(nx, ny, p, precision=precision, stream=stream)
    rows = []
    for C in centers:
        lat = make_lattice(C, "fp64")
        ref = run_history(lat, steps, every)
        lat.close()
        for prec in precisions:
            lat = make_lattice(C, prec)
            res = run_history(lat, steps, every)
            lat.close()
            rows.append({"C": C, "precision": prec, "steps": steps, "every": every,
                         **compare_to_fp64(ref, res)})
    return rows


FULL_MELT_LEVELS = (0.5, 0.9, 0.95, 0.99)


def crossing_fo(hist, level: float):
    """First Fourier number at which the melt fraction reaches `level`, linear
    between samples; None if it never does.  hist: (Fo, melt, ...) rows."""
    prev = None
    for row in hist:
        fo, m = row[0], row[1]
        if m >= level:
            if prev is None or m <= prev[1]:
                return fo
            return prev[0] + (fo - prev[0]) * (level - prev[1]) / (m - prev[1])
        prev = (fo, m)
    return None


def _paper_cavity(n, C, precision, stream):
    p = workloads.params(Ra=1e8, Pr=6.2, Ste=0.125, strip_center=C, strip_width=0.5)
    return lbm.Lattice(n, n, p, precision=precision, stream=stream)


class SoloSteps:
    """The batch interface over lattices stepped one by one (the single-lattice
    sweep, for a study of one large cavity)."""

    def __init__(self, k=None):
        self.members = []

    def add(self, lat):
        self.members.append(lat)

    def remove(self, lat):
        self.members.remove(lat)

    def step(self, k):
        for lat in self.members:
            lat.step(k)

    def close(self):
        self.members = []


def cavity_full_melt(n: int = 512, centers=(0.25, 0.375, 0.5), levels=FULL_MELT_LEVELS,
                     fo_max: float = 1.0, sample_fo: float = 0.002, precision: str = "fp32",
                     stream=None, checkpoint: str | None = None, max_seconds: float | None = None,
                     make_lattice=None, make_batch=None, href: int | None = None) -> dict:
    """Run the paper's cavities (Sec. 3.2) to full melting, all in one batch.

    Every `sample_fo` of Fourier number each running cavity's diagnostics are
    sampled (Fo, melt fraction, Nu, nan flag); a cavity leaves the batch once
    its melt fraction reaches max(levels), diverges or passes fo_max.  With
    `max_seconds`, the run stops after the first sample past that wall time,
    writes `checkpoint` (populations, step and history of each cavity) and
    returns with complete = False; a later call with the same checkpoint path
    resumes where it stopped and, for FP32 and FP64, ends bitwise where an
    uninterrupted run ends.  The Fourier number is alpha t / href^2 with href
    the cavity height (n for the paper's square cavities)."""
    import os
    import time

    if checkpoint is not None and precision not in ("fp32", "fp64"):
        raise ValueError("checkpoints hold FP32 or FP64 populations exactly; not " + precision)
    make_lattice = make_lattice or (lambda C: _paper_cavity(n, C, precision, stream))
    make_batch = make_batch or (lambda k: lbm.Batch(k, stream))
    lats = [make_lattice(C) for C in centers]
    alpha = lats[0].derived()["alpha"]
    L2 = float(href or n) ** 2
    chunk = max(1, int(round(sample_fo * L2 / alpha)))
    target = max(levels)
    hist = [[] for _ in centers]
    state = ["running"] * len(centers)
    if checkpoint is not None and os.path.exists(checkpoint):
        z = np.load(checkpoint)
        if int(z["n"]) != n or list(z["centers"]) != list(centers) or str(z["precision"]) != precision:
            raise ValueError(f"checkpoint {checkpoint} belongs to another run")
        for i, lat in enumerate(lats):
            lat.set_populations(z[f"f{i}"], z[f"g{i}"], int(z[f"step{i}"]))
            hist[i] = [tuple(r) for r in z[f"hist{i}"].tolist()]
            state[i] = str(z[f"state{i}"])
    else:  # the initial state is the first sample
        for i, lat in enumerate(lats):
            d = lat.diagnostics(raise_on_diverged=False)
            hist[i].append((d["step"] * alpha / L2, d["melt_fraction"], d["Nu"],
                            float(d["nan_flag"])))
    batch = make_batch(len(centers))
    for i, lat in enumerate(lats):
        if state[i] == "running":
            batch.add(lat)
    t0 = time.monotonic()
    complete = True
    while any(s == "running" for s in state):
        batch.step(chunk)
        for i, lat in enumerate(lats):
            if state[i] != "running":
                continue
            d = lat.diagnostics(raise_on_diverged=False)
            fo = d["step"] * alpha / L2
            hist[i].append((fo, d["melt_fraction"], d["Nu"], float(d["nan_flag"])))
            if d["nan_flag"]:
                state[i] = "diverged"
            elif d["melt_fraction"] >= target:
                state[i] = "melted"
            elif fo >= fo_max:
                state[i] = "fo_max"
            if state[i] != "running":
                batch.remove(lat)
        if max_seconds is not None and time.monotonic() - t0 > max_seconds and \
                any(s == "running" for s in state):
            complete = False
            break
    if checkpoint is not None:
        arrays = {"n": n, "centers": np.array(centers), "precision": precision}
        store = np.float32 if precision == "fp32" else np.float64
        for i, lat in enumerate(lats):
            f, g, step = lat.populations()
            arrays.update({f"f{i}": f.astype(store), f"g{i}": g.astype(store), f"step{i}": step,
                           f"hist{i}": np.array(hist[i], dtype=np.float64).reshape(-1, 4),
                           f"state{i}": state[i]})
        tmp = checkpoint + ".tmp.npz"
        np.savez_compressed(tmp, **arrays)
        os.replace(tmp, checkpoint)
    batch.close()
    for lat in lats:
        lat.close()
    return {"complete": complete, "n": n, "steps_per_sample": chunk, "alpha": alpha,
            "runs": {str(C): {"state": state[i],
                              "fo_at": {str(lv): crossing_fo(hist[i], lv) for lv in levels},
                              "final": hist[i][-1] if hist[i] else None,
                              "history": hist[i]}
                     for i, C in enumerate(centers)}}


def production_full_melt(center: float = 0.5, sample_fo: float = 0.002, fo_max: float = 1.0,
                          max_seconds: float | None = None, stream=None, make_lattice=None) -> dict:
    """The 2048 x 1024 production cavity (Ra 1e8, Pr 1, Ste 1, Ma 0.1, FP32
    populations and arithmetic, heated strip a quarter of the width) run to
    full melting on the single-lattice sweep: the melt-fraction and Nusselt
    history against Fo = alpha t / H^2 (H = 1024, the height), and the run's
    throughput over its wall time (sampling included)."""
    import time

    nx, ny, _ = workloads.cavity_2048x1024(center)
    make_lattice = make_lattice or (lambda C: lbm.Lattice(nx, ny, workloads.cavity_2048x1024(C)[2],
                                                          precision="fp32", stream=stream))
    t0 = time.monotonic()
    res = cavity_full_melt(n=nx, centers=(center,), fo_max=fo_max, sample_fo=sample_fo,
                           precision="fp32", stream=stream, max_seconds=max_seconds,
                           make_lattice=make_lattice, make_batch=SoloSteps, href=ny)
    wall = time.monotonic() - t0
    run = res["runs"][str(center)]
    steps = int(round(run["final"][0] * ny * ny / res["alpha"])) if run["final"] else 0
    res.update({"nx": nx, "ny": ny, "steps": steps, "wall_s": wall,
                "mlups_wall": steps * nx * ny / wall / 1e6 if wall > 0 else 0.0})
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description="the paper's Stefan and cavity-location studies")
    ap.add_argument("--study", choices=("stefan", "cavity", "cavity-full", "precision", "production-full"),
                    default="stefan")
    ap.add_argument("--fo", type=float, default=0.01)
    ap.add_argument("--precision", default=None)
    ap.add_argument("--n", type=int, default=512, help="cavity-full: lattice size")
    ap.add_argument("--steps", type=int, default=PRECISION_STUDY["steps"], help="precision: steps per run")
    ap.add_argument("--every", type=int, default=PRECISION_STUDY["every"], help="precision: sample interval")
    ap.add_argument("--size", default="2048x1024", help="precision: lattice size NXxNY")
    ap.add_argument("--fo-max", type=float, default=1.0, help="cavity-full: stop at this Fo")
    ap.add_argument("--checkpoint", default=None, help="cavity-full: resume from / save to")
    ap.add_argument("--max-seconds", type=float, default=None, help="cavity-full: wall budget")
    ap.add_argument("--out", default=None, help="cavity-full: write the result JSON here")
    args = ap.parse_args(argv)
    import torch

    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    if args.study == "stefan":
        for row in stefan_k1_sweep(args.precision or "fp64", s.cuda_stream):
            print(json.dumps(row), flush=True)
    elif args.study == "production-full":
        res = production_full_melt(fo_max=args.fo_max, max_seconds=args.max_seconds, stream=s.cuda_stream)
        if args.out:
            with open(args.out, "w") as fh:
                json.dump(res, fh)
        run = res["runs"]["0.5"]
        print(json.dumps({k: v for k, v in res.items() if k != "runs"} |
                         {"state": run["state"], "fo_at": run["fo_at"], "final": run["final"]}), flush=True)
    elif args.study == "precision":
        nx, ny = (int(v) for v in args.size.split("x"))
        precs = tuple(args.precision.split(",")) if args.precision else PRECISION_STUDY["precisions"]
        for row in precision_study(nx, ny, args.steps, args.every, precisions=precs, stream=s.cuda_stream):
            print(json.dumps(row), flush=True)
    elif args.study == "cavity":
        res = cavity_location_sweep(args.fo, precision=args.precision or "fp32", stream=s.cuda_stream)
        print(json.dumps({str(k): v for k, v in res.items()}), flush=True)
    else:
        res = cavity_full_melt(args.n, fo_max=args.fo_max, precision=args.precision or "fp32",
                               stream=s.cuda_stream, checkpoint=args.checkpoint,
                               max_seconds=args.max_seconds)
        if args.out:
            with open(args.out, "w") as fh:
                json.dump(res, fh)
        summary = {k: v for k, v in res.items() if k != "runs"}
        summary["runs"] = {C: {k: v for k, v in r.items() if k != "history"}
                           for C, r in res["runs"].items()}
        print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    main()
