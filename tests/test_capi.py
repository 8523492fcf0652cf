"""The C-ABI library loads and exports every entry point the header declares
(no GPU needed: no compute call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lbm_\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def built():
    from paper_1909_13086_gb300 import build

    build.build()
    from paper_1909_13086_gb300 import lbm

    return lbm


def test_header_declares_the_api():
    names = declared_functions()
    for n in ("lbm_create", "lbm_set_params", "lbm_step", "lbm_read_fields", "lbm_diagnostics",
              "lbm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    L = built.lib()
    for n in declared_functions():
        assert hasattr(L, n), n
    assert set(declared_functions()) == set(built.EXPORTED)
    assert built.lbm_version().endswith("sm_103a")


def test_exports_nothing_else(built):
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", built.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert syms == set(declared_functions())


def test_struct_layouts_match_header(built):
    import ctypes

    # lbm_params: int + 4 doubles + 2 + 2 + 1 + 2 doubles + int + double + uint64
    assert ctypes.sizeof(built.lbm_params) == 4 + 4 + 8 * 11 + 4 + 4 + 8 + 8
    assert ctypes.sizeof(built.lbm_derived) == 14 * 8
    assert ctypes.sizeof(built.lbm_diag) == 8 + 7 * 8 + 8


def test_argument_errors_need_no_gpu(built):
    import ctypes

    L = built.lib()
    h = ctypes.c_void_p()
    assert L.lbm_create(1, 1, 1, None, ctypes.byref(h)) == built.LBM_ERR_ARG
    assert b"nx and ny" in L.lbm_last_error(None)
    assert L.lbm_create(8, 8, 7, None, ctypes.byref(h)) == built.LBM_ERR_ARG
    assert (built.LBM_FP64, built.LBM_FP32, built.LBM_FP16, built.LBM_BF16) == (0, 1, 2, 3)
    assert L.lbm_create(8, 65536, 1, None, ctypes.byref(h)) == built.LBM_ERR_ARG   # ny > 65535
    assert L.lbm_create(65536, 40000, 1, None, ctypes.byref(h)) == built.LBM_ERR_ARG  # > 2^31 cells
    assert L.lbm_step(None, 1) == built.LBM_ERR_ARG
    assert L.lbm_set_streaming(None, built.LBM_STREAM_ONE_BUFFER) == built.LBM_ERR_ARG
    assert L.lbm_batch_set_streaming(None, built.LBM_STREAM_TWO_BUFFERS) == built.LBM_ERR_ARG
    assert L.lbm_destroy(None) == built.LBM_OK


def test_streaming_constants_match_header(built):
    import re

    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    m = re.search(r"enum \{ LBM_STREAM_TWO_BUFFERS = (\d+), LBM_STREAM_ONE_BUFFER = (\d+) \};", text)
    assert m and (int(m.group(1)), int(m.group(2))) == (built.LBM_STREAM_TWO_BUFFERS, built.LBM_STREAM_ONE_BUFFER)
