"""ctypes wrapper of the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is the plain statement of what the GPU
sweep must compute (paper Sec. 2, Eqs. 1-6; Sec. 3, Eqs. 7-8, plus the readings
listed in lbm_oracle.c).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  It never touches the CUDA
library, and the CUDA library never touches it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CAVITY, STEFAN = 0, 1


def compile_cmd() -> list[str]:
    """Compiler command for the oracle: plain C99, FP64 exactly as written."""
    return ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
            "-fopenmp", "-shared", "-fPIC", _SRC, "-o", _LIB, "-lm"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (if older than the source)."""
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
             or os.path.getmtime(_LIB) < os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h")))
    if force or stale:
        subprocess.run(compile_cmd(), check=True)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("problem", ctypes.c_int),
        ("Ra", ctypes.c_double), ("Pr", ctypes.c_double),
        ("Ste", ctypes.c_double), ("Ma", ctypes.c_double),
        ("strip_center", ctypes.c_double), ("strip_width", ctypes.c_double),
        ("k0", ctypes.c_double), ("k2", ctypes.c_double),
        ("alpha_override", ctypes.c_double),
        ("k0f", ctypes.c_double), ("k1f", ctypes.c_double),
        ("flow_on", ctypes.c_int),
        ("init_amp", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


class Derived(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "cs2", "nu", "alpha", "gbeta", "k0", "k1", "k2", "k0f", "k1f", "k2f",
        "Lh", "a", "b", "Href", "heated_len")]


class Diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "step", "melt_fraction", "H_total", "Q_strip", "Q_cum", "Nu",
        "front_x", "max_u", "nan_flag")]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_D9 = ctypes.c_double * 9
_I9 = ctypes.c_int * 9


def _bind(L: ctypes.CDLL) -> ctypes.CDLL:
    """Declare the C signatures of an oracle library (the built one, or a
    variant compiled by ``compile_variant``)."""
    L.orc_splitmix64.restype = ctypes.c_uint64
    L.orc_splitmix64.argtypes = [ctypes.c_uint64]
    L.orc_invert.argtypes = [ctypes.c_double, ctypes.c_double, _D, _D]
    L.orc_geq.argtypes = [ctypes.c_double] * 4 + [_D]
    L.orc_g_collide.argtypes = [_D] + [ctypes.c_double] * 7 + [_D]
    L.orc_feq.argtypes = [ctypes.c_double] * 3 + [_D]
    L.orc_f_collide.argtypes = [_D] + [ctypes.c_double] * 8 + [_D]
    L.orc_stefan_lambda.restype = ctypes.c_double
    L.orc_stefan_lambda.argtypes = [ctypes.c_double]
    L.orc_neumann_T.restype = ctypes.c_double
    L.orc_neumann_T.argtypes = [ctypes.c_double] * 6
    L.orc_derive.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params),
                             ctypes.POINTER(Derived)]
    L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params),
                             ctypes.POINTER(ctypes.c_void_p)]
    L.orc_destroy.argtypes = [ctypes.c_void_p]
    L.orc_destroy.restype = None
    L.orc_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
    L.orc_fields.argtypes = [ctypes.c_void_p] + [_D] * 6
    L.orc_diagnostics.argtypes = [ctypes.c_void_p, ctypes.POINTER(Diag)]
    L.orc_get_derived.argtypes = [ctypes.c_void_p, ctypes.POINTER(Derived)]
    L.orc_get_populations.argtypes = [ctypes.c_void_p, _D, _D]
    L.orc_set_populations.argtypes = [ctypes.c_void_p, _D, _D, ctypes.c_longlong]
    L.orc_cell_update.argtypes = [ctypes.c_void_p, _D, _D, ctypes.c_int, ctypes.c_int,
                                  _D, _D, _D, _D]
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


# ------------------------------------------------------ planted mistakes
# A pin is only worth something if a plausible slip in the oracle breaks it.
# The tests check that by compiling copies of lbm_oracle.c with one mistake
# planted (a text replacement) and running the pin against the copy.
def compile_variant(replacements: list[tuple[str, str]], out_dir: str) -> str:
    """Compile a copy of lbm_oracle.c with each (old, new) replacement applied
    (each ``old`` must occur exactly once) into out_dir; returns the library
    path."""
    src = open(_SRC).read()
    for old, new in replacements:
        if src.count(old) != 1:
            raise ValueError(f"replacement target must occur once: {old!r}")
        src = src.replace(old, new)
    os.makedirs(out_dir, exist_ok=True)
    csrc = os.path.join(out_dir, "lbm_oracle_variant.c")
    with open(csrc, "w") as fh:
        fh.write(src)
    so = os.path.join(out_dir, "liboracle_variant.so")
    cmd = compile_cmd()
    cmd[cmd.index(_SRC)] = csrc
    cmd[cmd.index(_LIB)] = so
    subprocess.run(cmd + ["-I", _HERE], check=True)
    return so


class variant:
    """Context manager: every function of this module uses the library at
    ``path`` (a planted-mistake copy) instead of the oracle, until exit."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = lib()
        _lib = _bind(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def make_params(**kw) -> Params:
    p = Params()
    defaults = dict(problem=CAVITY, Ra=1e4, Pr=1.0, Ste=1.0, Ma=0.1,
                    strip_center=0.5, strip_width=0.25, k0=1.0, k2=1.0,
                    alpha_override=0.0, k0f=1.0, k1f=1.0, flow_on=1,
                    init_amp=1e-3, seed=1)
    defaults.update(kw)
    for k, v in defaults.items():
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------- per cell
def lattice():
    cx, cy, w, opp = _I9(), _I9(), _D9(), _I9()
    lib().orc_lattice(cx, cy, w, opp)
    return (np.array(cx[:]), np.array(cy[:]), np.array(w[:]), np.array(opp[:]))


def splitmix64(v: int) -> int:
    return int(lib().orc_splitmix64(ctypes.c_uint64(v & (2**64 - 1))))


def invert(H: float, Lh: float):
    T, fl = ctypes.c_double(), ctypes.c_double()
    lib().orc_invert(H, Lh, ctypes.byref(T), ctypes.byref(fl))
    return T.value, fl.value


def geq(H, T, ux, uy) -> np.ndarray:
    out = _D9()
    lib().orc_geq(H, T, ux, uy, out)
    return np.array(out[:])


def g_collide(g, H, T, ux, uy, k0, k1, k2) -> np.ndarray:
    gin = _D9(*[float(v) for v in g])
    out = _D9()
    lib().orc_g_collide(gin, H, T, ux, uy, k0, k1, k2, out)
    return np.array(out[:])


def feq(rho, ux, uy) -> np.ndarray:
    out = _D9()
    lib().orc_feq(rho, ux, uy, out)
    return np.array(out[:])


def f_collide(f, rho, ux, uy, Fx, Fy, k0f, k1f, k2f) -> np.ndarray:
    fin = _D9(*[float(v) for v in f])
    out = _D9()
    lib().orc_f_collide(fin, rho, ux, uy, Fx, Fy, k0f, k1f, k2f, out)
    return np.array(out[:])


def stefan_lambda(Ste: float) -> float:
    return float(lib().orc_stefan_lambda(Ste))


def neumann_T(x, t, alpha, lam, Th=1.0, Tm=0.0) -> float:
    return float(lib().orc_neumann_T(x, t, alpha, lam, Th, Tm))


def derive(nx: int, ny: int, **kw) -> Derived:
    d = Derived()
    p = make_params(**kw)
    rc = lib().orc_derive(nx, ny, ctypes.byref(p), ctypes.byref(d))
    if rc != 0:
        raise ValueError(f"orc_derive rejected the parameters (status {rc})")
    return d


# ---------------------------------------------------------------- lattice
class Oracle:
    """One lattice of the FP64 oracle.  Arrays are numpy float64."""

    def __init__(self, nx: int, ny: int, threads: int = 1, **kw):
        self.nx, self.ny = nx, ny
        self.params = make_params(**kw)
        h = ctypes.c_void_p()
        rc = lib().orc_create(nx, ny, ctypes.byref(self.params), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"orc_create failed (status {rc})")
        self._h = h
        self.set_threads(threads)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_threads(self, n: int):
        if lib().orc_set_threads(self._h, int(n)) != 0:
            raise ValueError("bad thread count")

    def step(self, n: int = 1):
        if lib().orc_step(self._h, int(n)) != 0:
            raise RuntimeError("orc_step failed")

    def fields(self) -> dict:
        P = (self.ny, self.nx)
        out = {k: np.empty(P) for k in ("H", "T", "fl", "ux", "uy", "rho")}
        rc = lib().orc_fields(self._h, *[_ptr(out[k]) for k in ("H", "T", "fl", "ux", "uy", "rho")])
        if rc != 0:
            raise RuntimeError(f"orc_fields failed (status {rc})")
        return out

    def diagnostics(self) -> dict:
        d = Diag()
        rc = lib().orc_diagnostics(self._h, ctypes.byref(d))
        if rc != 0:
            raise RuntimeError(f"orc_diagnostics failed (status {rc})")
        return {n: getattr(d, n) for n, _ in Diag._fields_}

    def derived(self) -> dict:
        d = Derived()
        lib().orc_get_derived(self._h, ctypes.byref(d))
        return {n: getattr(d, n) for n, _ in Derived._fields_}

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        lib().orc_get_populations(self._h, _ptr(f), _ptr(g))
        return f, g

    def set_populations(self, f: np.ndarray, g: np.ndarray, step: int = 0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx) and g.shape == f.shape
        if lib().orc_set_populations(self._h, _ptr(f), _ptr(g), int(step)) != 0:
            raise RuntimeError("orc_set_populations failed")

    def cell_update(self, fprev: np.ndarray, gprev: np.ndarray, x: int, y: int):
        """New post-collision populations, fields and inflow of one cell,
        from arbitrary previous populations (shape (9, ny, nx), float64)."""
        fprev = np.ascontiguousarray(fprev, dtype=np.float64)
        gprev = np.ascontiguousarray(gprev, dtype=np.float64)
        fo, go, m = _D9(), _D9(), (ctypes.c_double * 6)()
        q = ctypes.c_double()
        rc = lib().orc_cell_update(self._h, _ptr(fprev), _ptr(gprev), x, y, fo, go, m,
                                   ctypes.byref(q))
        if rc != 0:
            raise RuntimeError("orc_cell_update failed")
        return np.array(fo[:]), np.array(go[:]), np.array(m[:]), q.value


if __name__ == "__main__":  # pragma: no cover - manual build helper
    print(build(force="--force" in sys.argv))
