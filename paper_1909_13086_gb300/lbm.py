"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (``libbtrirt.so``).

Argument marshalling only: every step of the solver runs in the CUDA library.
The functions keep the C names (``lbm_create``, ``lbm_set_params``,
``lbm_step``, ``lbm_read_fields``, ``lbm_diagnostics``, ...); ``Lattice`` is a
small convenience wrapper over them.  PyTorch, when present, lends the CUDA
stream and the caching allocator -- plumbing only.

There is no CPU fallback: if the library is missing or cannot be loaded this
module raises on first use.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbtrirt.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_DIVERGED, LBM_ERR_STATE, LBM_ERR_TIMEOUT = \
    0, -1, -2, -3, -4, -5, -6
LBM_FP64, LBM_FP32, LBM_FP16, LBM_BF16, LBM_FP16_SR, LBM_BF16_SR = 0, 1, 2, 3, 4, 5
LBM_CAVITY, LBM_STEFAN = 0, 1
LBM_STREAM_TWO_BUFFERS, LBM_STREAM_ONE_BUFFER = 0, 1
FIELD_BITS = {"H": 1, "T": 2, "fl": 4, "ux": 8, "uy": 16, "rho": 32}
FIELD_NAMES = ("H", "T", "fl", "ux", "uy", "rho")
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16": LBM_FP16, "bf16": LBM_BF16,
              "fp16sr": LBM_FP16_SR, "bf16sr": LBM_BF16_SR}


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


class lbm_params(ctypes.Structure):
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


class lbm_derived(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "nu", "alpha", "gbeta", "k0", "k1", "k2", "k0f", "k1f", "k2f", "Lh", "a", "b",
        "Href", "heated_len")]


class lbm_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong)] + [(n, ctypes.c_double) for n in (
        "melt_fraction", "H_total", "Q_strip", "Q_cum", "Nu", "front_x", "max_u")] + [
        ("nan_flag", ctypes.c_int)]


class lbm_launch_stats(ctypes.Structure):
    _fields_ = [("sweeps_direct", ctypes.c_longlong), ("sweeps_replayed", ctypes.c_longlong),
                ("graphs_captured", ctypes.c_longlong)]


EXPORTED = ("lbm_create", "lbm_set_params", "lbm_get_derived", "lbm_step", "lbm_set_diag_every",
            "lbm_set_launch", "lbm_get_launch_stats", "lbm_set_staging", "lbm_set_streaming", "lbm_set_wait_limit",
            "lbm_read_fields", "lbm_diagnostics", "lbm_read_populations", "lbm_write_populations",
            "lbm_destroy", "lbm_last_error", "lbm_set_allocator", "lbm_version", "lbm_step_static",
            "lbm_batch_create", "lbm_batch_add", "lbm_batch_remove", "lbm_batch_count",
            "lbm_batch_step", "lbm_batch_destroy", "lbm_autotune", "lbm_set_history",
            "lbm_read_history", "lbm_batch_set_launch", "lbm_batch_set_streaming", "lbm_batch_autotune")

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def lib() -> ctypes.CDLL:
    """Load ``libbtrirt.so`` (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with paper_1909_13086_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    L.lbm_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                             ctypes.POINTER(H)]
    L.lbm_set_params.argtypes = [H, ctypes.POINTER(lbm_params)]
    L.lbm_get_derived.argtypes = [H, ctypes.POINTER(lbm_derived)]
    L.lbm_step.argtypes = [H, ctypes.c_longlong]
    L.lbm_set_diag_every.argtypes = [H, ctypes.c_longlong]
    L.lbm_set_launch.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.lbm_get_launch_stats.argtypes = [H, ctypes.POINTER(lbm_launch_stats)]
    L.lbm_set_staging.argtypes = [H, ctypes.c_int]
    L.lbm_set_streaming.argtypes = [H, ctypes.c_int]
    L.lbm_batch_set_streaming.argtypes = [H, ctypes.c_int]
    L.lbm_set_wait_limit.argtypes = [H, ctypes.c_longlong, ctypes.c_int]
    L.lbm_read_fields.argtypes = [H, ctypes.c_uint] + [_D] * 6
    L.lbm_diagnostics.argtypes = [H, ctypes.POINTER(lbm_diag)]
    L.lbm_read_populations.argtypes = [H, _D, _D, ctypes.POINTER(ctypes.c_longlong)]
    L.lbm_write_populations.argtypes = [H, _D, _D, ctypes.c_longlong]
    L.lbm_destroy.argtypes = [H]
    L.lbm_last_error.argtypes = [H]
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_set_allocator.argtypes = [ALLOC_FN, FREE_FN, ctypes.c_void_p]
    L.lbm_version.restype = ctypes.c_char_p
    L.lbm_set_history.argtypes = [H, ctypes.c_longlong]
    L.lbm_read_history.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), _D, _D, _D,
                                   ctypes.POINTER(ctypes.c_int)]
    L.lbm_autotune.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_float)]
    L.lbm_batch_create.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    L.lbm_batch_add.argtypes = [ctypes.c_void_p, H]
    L.lbm_batch_remove.argtypes = [ctypes.c_void_p, H]
    L.lbm_batch_count.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
    L.lbm_batch_step.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
    L.lbm_batch_destroy.argtypes = [ctypes.c_void_p]
    L.lbm_batch_set_launch.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.lbm_batch_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_float)]
    L.lbm_step_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.POINTER(lbm_params), ctypes.c_longlong,
                                  ctypes.c_void_p, ctypes.POINTER(lbm_diag)]
    for name in EXPORTED:
        if name not in ("lbm_last_error", "lbm_version"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, h=None) -> int:
    if rc != LBM_OK:
        raise LbmError(rc, lib().lbm_last_error(h).decode())
    return rc


def _dptr(a):
    if a is None:
        return None
    assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def make_params(d: dict) -> lbm_params:
    p = lbm_params()
    for k, v in d.items():
        setattr(p, k, v)
    return p


# ------------------------------------------------------------ C-ABI mirrors
def lbm_version() -> str:
    return lib().lbm_version().decode()


def lbm_create(nx: int, ny: int, precision: int, stream: int | None = None):
    h = ctypes.c_void_p()
    _check(lib().lbm_create(nx, ny, precision, ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h


def lbm_set_params(h, params: dict | lbm_params) -> None:
    p = params if isinstance(params, lbm_params) else make_params(params)
    _check(lib().lbm_set_params(h, ctypes.byref(p)), h)


def lbm_get_derived(h) -> dict:
    d = lbm_derived()
    _check(lib().lbm_get_derived(h, ctypes.byref(d)), h)
    return {n: getattr(d, n) for n, _ in lbm_derived._fields_}


def lbm_step(h, n: int) -> None:
    _check(lib().lbm_step(h, int(n)), h)


def lbm_set_diag_every(h, k: int) -> None:
    _check(lib().lbm_set_diag_every(h, int(k)), h)


def lbm_set_launch(h, rows: int = 1, prefetch: int = 16, graph_chunk: int = 128) -> None:
    """Launch shape (the defaults are the library's FP32 ones; with 16-bit
    storage the library starts from 3 rows and prefetch 32)."""
    _check(lib().lbm_set_launch(h, int(rows), int(prefetch), int(graph_chunk)), h)


def lbm_set_staging(h, bands: int = -1) -> None:
    _check(lib().lbm_set_staging(h, int(bands)), h)


def lbm_set_streaming(h, mode: int = LBM_STREAM_ONE_BUFFER) -> None:
    _check(lib().lbm_set_streaming(h, int(mode)), h)


def lbm_set_wait_limit(h, tries: int = 1 << 20, force_timeout: bool = False) -> None:
    _check(lib().lbm_set_wait_limit(h, int(tries), 1 if force_timeout else 0), h)


def lbm_get_launch_stats(h) -> dict:
    st = lbm_launch_stats()
    _check(lib().lbm_get_launch_stats(h, ctypes.byref(st)), h)
    return {n: getattr(st, n) for n, _ in lbm_launch_stats._fields_}


def lbm_read_fields(h, mask: int, H=None, T=None, fl=None, ux=None, uy=None, rho=None) -> None:
    _check(lib().lbm_read_fields(h, mask, _dptr(H), _dptr(T), _dptr(fl), _dptr(ux), _dptr(uy),
                                 _dptr(rho)), h)


def lbm_diagnostics(h, raise_on_diverged: bool = True) -> dict:
    d = lbm_diag()
    rc = lib().lbm_diagnostics(h, ctypes.byref(d))
    if rc != LBM_OK and not (rc == LBM_ERR_DIVERGED and not raise_on_diverged):
        _check(rc, h)
    return {n: getattr(d, n) for n, _ in lbm_diag._fields_}


def lbm_read_populations(h, f: np.ndarray | None, g: np.ndarray | None) -> int:
    step = ctypes.c_longlong()
    _check(lib().lbm_read_populations(h, _dptr(f), _dptr(g), ctypes.byref(step)), h)
    return step.value


def lbm_write_populations(h, f: np.ndarray, g: np.ndarray, step: int) -> None:
    _check(lib().lbm_write_populations(h, _dptr(f), _dptr(g), int(step)), h)


def lbm_step_static(src_ptr: int, dst_ptr: int, nx: int, ny: int, precision: int, params: dict,
                    step: int, stream: int | None = None, want_diag: bool = True) -> dict | None:
    """One sweep on caller-owned device buffers (tile-major layout), no
    allocation inside the library; returns the diagnostics of step + 1."""
    p = make_params(params)
    d = lbm_diag()
    rc = lib().lbm_step_static(ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr), nx, ny, precision,
                               ctypes.byref(p), int(step), ctypes.c_void_p(stream or 0),
                               ctypes.byref(d) if want_diag else None)
    _check(rc)
    return {n: getattr(d, n) for n, _ in lbm_diag._fields_} if want_diag else None


def lbm_set_history(h, capacity: int) -> None:
    _check(lib().lbm_set_history(h, int(capacity)), h)


def lbm_read_history(h, max_entries: int) -> dict:
    step = (ctypes.c_longlong * max(1, max_entries))()
    Q, Nu, melt = (np.empty(max(1, max_entries)) for _ in range(3))
    n = ctypes.c_int()
    _check(lib().lbm_read_history(h, int(max_entries), step, _dptr(Q), _dptr(Nu), _dptr(melt),
                                  ctypes.byref(n)), h)
    k = n.value
    return {"step": np.array(step[:k], dtype=np.int64), "Q": Q[:k], "Nu": Nu[:k], "melt": melt[:k]}


def lbm_autotune(h, steps_per_trial: int = 200) -> dict:
    rows, pf, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(lib().lbm_autotune(h, int(steps_per_trial), ctypes.byref(rows), ctypes.byref(pf),
                              ctypes.byref(us)), h)
    return {"rows": rows.value, "prefetch": pf.value, "us_per_step": us.value}


def lbm_batch_create(max_lattices: int, stream: int | None = None):
    b = ctypes.c_void_p()
    _check(lib().lbm_batch_create(int(max_lattices), ctypes.c_void_p(stream or 0), ctypes.byref(b)))
    return b


def lbm_batch_add(b, h) -> None:
    _check(lib().lbm_batch_add(b, h))


def lbm_batch_remove(b, h) -> None:
    _check(lib().lbm_batch_remove(b, h))


def lbm_batch_count(b) -> int:
    c = ctypes.c_int()
    _check(lib().lbm_batch_count(b, ctypes.byref(c)))
    return c.value


def lbm_batch_step(b, n: int) -> None:
    _check(lib().lbm_batch_step(b, int(n)))


def lbm_batch_set_launch(b, rows: int = 0, prefetch: int = -1, interleave: int = 0) -> None:
    _check(lib().lbm_batch_set_launch(b, int(rows), int(prefetch), int(interleave)))


def lbm_batch_set_streaming(b, mode: int = LBM_STREAM_ONE_BUFFER) -> None:
    _check(lib().lbm_batch_set_streaming(b, int(mode)))


def lbm_batch_autotune(b, steps_per_trial: int = 50) -> dict:
    rows, pf, il, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(lib().lbm_batch_autotune(b, int(steps_per_trial), ctypes.byref(rows), ctypes.byref(pf),
                                    ctypes.byref(il), ctypes.byref(us)))
    return {"rows": rows.value, "prefetch": pf.value, "interleave": il.value, "us_per_step": us.value}


def lbm_batch_destroy(b) -> None:
    _check(lib().lbm_batch_destroy(b))


def lbm_destroy(h) -> None:
    _check(lib().lbm_destroy(h))


_torch_hooks = None


def use_torch_allocator() -> None:
    """Route the library's device allocations through PyTorch's caching
    allocator (device memory as plumbing; the library stays torch-free)."""
    global _torch_hooks
    import torch

    def _alloc(nbytes, ctx):
        try:
            dev = torch.cuda.current_device()
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev,
                                                      torch.cuda.current_stream(dev))
        except Exception:  # allocation failure -> NULL, reported as LBM_ERR_OOM
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    _torch_hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(lib().lbm_set_allocator(_torch_hooks[0], _torch_hooks[1], None))


def use_default_allocator() -> None:
    """Back to cudaMalloc / cudaFree for later lbm_create calls."""
    _check(lib().lbm_set_allocator(ALLOC_FN(), FREE_FN(), None))


# ------------------------------------------------------------ convenience
class Lattice:
    """One lattice on the current CUDA device.  ``params`` is a dict with the
    fields of ``lbm_params`` (see ``workloads.params``)."""

    def __init__(self, nx: int, ny: int, params: dict, precision: str = "fp32",
                 stream: int | None = None):
        self.nx, self.ny = nx, ny
        self.precision = precision
        self.h = lbm_create(nx, ny, PRECISIONS[precision], stream)
        lbm_set_params(self.h, params)

    def close(self):
        if getattr(self, "h", None) is not None:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    def derived(self) -> dict:
        return lbm_get_derived(self.h)

    def diagnostics(self, raise_on_diverged: bool = True) -> dict:
        return lbm_diagnostics(self.h, raise_on_diverged)

    def fields(self, names=FIELD_NAMES) -> dict:
        out = {k: np.empty((self.ny, self.nx)) for k in names}
        mask = 0
        for k in names:
            mask |= FIELD_BITS[k]
        lbm_read_fields(self.h, mask, *[out.get(k) for k in FIELD_NAMES])
        return out

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        step = lbm_read_populations(self.h, f, g)
        return f, g, step

    def set_populations(self, f: np.ndarray, g: np.ndarray, step: int = 0):
        lbm_write_populations(self.h, np.ascontiguousarray(f, np.float64),
                              np.ascontiguousarray(g, np.float64), step)


class Batch:
    """Lattices advanced together by one fused launch per step."""

    def __init__(self, max_lattices: int = 64, stream: int | None = None):
        self.b = lbm_batch_create(max_lattices, stream)
        self.members = []

    def add(self, lat: Lattice):
        lbm_batch_add(self.b, lat.h)
        self.members.append(lat)

    def remove(self, lat: Lattice):
        lbm_batch_remove(self.b, lat.h)
        self.members.remove(lat)

    def step(self, n: int = 1):
        lbm_batch_step(self.b, n)

    def close(self):
        if getattr(self, "b", None) is not None:
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
