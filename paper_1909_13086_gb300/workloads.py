"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module holds parameter sets and seeded random arrays only -- none of the
method's arithmetic -- so that the CUDA path and the CPU oracle can be driven
with identical inputs without either depending on the other.

Workloads (all synthetic initial-boundary-value problems; the paper uses no
dataset):
  * ``cavity_64x32``     -- 64 x 32 cavity, Ra 1e4, Pr 1, Ste 1, Ma 0.1, strip of
                            width W/4 in the middle of the bottom wall, k0 = k2 = 1,
                            seeded +-1e-3 perturbation of T (Sec. 3.2 geometry).
  * ``stefan_1024x4``    -- one-phase melting by conduction, 1024 x 4, periodic y,
                            left wall at T_h, u = 0, alpha = 1/6 (Sec. 3.1).
  * ``cavity_2048x1024`` -- production cavity, Ra 1e8, Pr 1, Ste 1, Ma 0.1.
"""
from __future__ import annotations

import numpy as np

CAVITY, STEFAN = 0, 1

_BASE = dict(problem=CAVITY, Ra=1e4, Pr=1.0, Ste=1.0, Ma=0.1,
             strip_center=0.5, strip_width=0.25, k0=1.0, k2=1.0,
             alpha_override=0.0, k0f=1.0, k1f=1.0, flow_on=1,
             init_amp=1e-3, seed=1)


def params(**overrides) -> dict:
    """A complete parameter dict: the 64 x 32 cavity values, then overrides."""
    p = dict(_BASE)
    for k in overrides:
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
    p.update(overrides)
    return p


def cavity_64x32() -> tuple[int, int, dict]:
    return 64, 32, params()


def stefan_1024x4(Ste: float = 1.0, alpha: float = 1.0 / 6.0, k2: float = -1.0,
                  k0: float = 1.0, nx: int = 1024) -> tuple[int, int, dict]:
    """Sec. 3.1 setup in lattice units, thermal diffusivity ``alpha`` given
    directly; k2 < 0 selects k2 = 2 - k1 (Eq. 6)."""
    return nx, 4, params(problem=STEFAN, Ste=Ste, flow_on=0, alpha_override=alpha,
                         k0=k0, k2=k2, init_amp=0.0)


def cavity_2048x1024(strip_center: float = 0.5) -> tuple[int, int, dict]:
    return 2048, 1024, params(Ra=1e8, strip_center=strip_center)


def random_populations(nx: int, ny: int, seed: int, H_mean: float = 0.5,
                       H_spread: float = 1.5, noise: float = 0.01):
    """Seeded arbitrary (non-equilibrium) post-collision populations, shape
    (9, ny, nx) float64 each, for single-step parity checks.  g spreads the
    cell enthalpy across solid, mushy and liquid states; f is a perturbed rest
    state with unit density on average."""
    rng = np.random.default_rng(seed)
    H = H_mean + H_spread * (rng.random((ny, nx)) - 0.5) * 2.0
    g = H[None, :, :] / 9.0 + noise * (rng.random((9, ny, nx)) - 0.5)
    f = 1.0 / 9.0 + noise * (rng.random((9, ny, nx)) - 0.5)
    return f, g
