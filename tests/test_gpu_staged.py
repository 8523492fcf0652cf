"""The staged sweep of 16-bit storage (tile rows streamed through shared
memory by TMA bulk copies, bands of rows per block) computes exactly what the
row-per-block sweep computes: populations and diagnostics bitwise, for the
cavity (ragged tiles, side walls, heated strip, one or many bands) and the
Stefan problem (periodic rows, flow off).  Its bounded waits report a timeout
as LBM_ERR_TIMEOUT, without a fault, and the handle stays usable."""
import numpy as np
import pytest

from paper_1909_13086_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu

_STREAMS = []


@pytest.fixture(scope="module")
def stream():
    import torch

    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    _STREAMS.append(s)
    return s.cuda_stream


def state(lat):
    f, g, step = lat.populations()
    return f, g, step, lat.diagnostics()


CASES = [
    ("cavity 300x77", 300, 77, workloads.params(Ra=1e6, strip_center=0.4)),
    ("cavity 256x128", 256, 128, workloads.params(Ra=1e7, strip_center=0.2)),
    ("cavity 130x9", 130, 9, workloads.params(Ra=1e5, strip_center=0.5, strip_width=0.6)),
    ("cavity 2x12", 2, 12, workloads.params(Ra=1e5)),
    ("stefan 300x8", 300, 8, workloads.stefan_1024x4(Ste=0.5, nx=300)[2]),
]


# band counts per case: the automatic choice, 1, and 3 where the lattice has
# the 12 rows that 3 bands need (bands are capped at ny / 4)
SHAPES = [(c, bands) for c in CASES for bands in (-1, 1, 3) if bands < 0 or c[2] >= 4 * bands]


@pytest.mark.parametrize("prec", ["fp16sr", "bf16sr", "fp16", "bf16"])
@pytest.mark.parametrize("case,bands", SHAPES, ids=[f"{c[0]}-bands{b}" for c, b in SHAPES])
def test_staged_equals_row_per_block(stream, prec, case, bands):
    name, nx, ny, p = case
    ref = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    lbm.lbm_set_staging(ref.h, 0)
    lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    lbm.lbm_set_staging(lat.h, bands)
    for n in (1, 37, 200):  # direct launches and graph-replayed pieces
        ref.step(n)
        lat.step(n)
        a, b = state(ref), state(lat)
        assert a[2] == b[2]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (name, n)
        assert a[3] == b[3], (name, n)


def test_staged_timeout_is_reported_and_recoverable(stream):
    """Every block first waits on a barrier that nothing completes: the wait
    runs out after a few tries, the blocks let their copies land and return,
    and lbm_diagnostics reports LBM_ERR_TIMEOUT.  After lbm_set_params the
    handle steps exactly like a fresh one."""
    nx, ny, p = 256, 128, workloads.params(Ra=1e6)
    lat = lbm.Lattice(nx, ny, p, precision="bf16sr", stream=stream)
    lbm.lbm_set_staging(lat.h, -1)
    lbm.lbm_set_wait_limit(lat.h, 16, force_timeout=True)
    lat.step(3)
    with pytest.raises(lbm.LbmError) as e:
        lat.diagnostics()
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    lbm.lbm_set_wait_limit(lat.h, 1 << 20, force_timeout=False)
    lbm.lbm_set_params(lat.h, p)
    lat.step(50)
    fresh = lbm.Lattice(nx, ny, p, precision="bf16sr", stream=stream)
    lbm.lbm_set_staging(fresh.h, 0)
    fresh.step(50)
    a, b = state(fresh), state(lat)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[3] == b[3]


def test_staging_argument_checks(stream):
    lat = lbm.Lattice(64, 32, workloads.params(), precision="fp16sr", stream=stream)
    for bad in (-2, 70000):
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_staging(lat.h, bad)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_wait_limit(lat.h, -1)
    # FP32 lattices ignore the setting
    f32 = lbm.Lattice(64, 32, workloads.params(), precision="fp32", stream=stream)
    lbm.lbm_set_staging(f32.h, 3)
    f32.step(10)
    assert f32.diagnostics()["step"] == 10
