"""Sweeps replayed from captured CUDA graphs compute exactly what direct
launches compute: populations, diagnostics and the history ring bitwise, for
call lengths below, at and above the longest piece, odd and even (so both
buffer parities start a piece), with diagnostic sweeps inside a call, and for
batches."""
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


def assert_same(a, b):
    assert a[2] == b[2]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[3] == b[3]


@pytest.mark.parametrize("n", [2, 20, 127, 129, 200])
@pytest.mark.parametrize("prec", ["fp32", "bf16sr"])
def test_replayed_pieces_equal_direct_launches(stream, n, prec):
    p = workloads.params(Ra=1e6, strip_center=0.4)
    direct = lbm.Lattice(300, 77, p, precision=prec, stream=stream)
    lbm.lbm_set_launch(direct.h, 1, 24 if prec == "bf16sr" else 4, 0)   # every sweep launched directly
    graphed = lbm.Lattice(300, 77, p, precision=prec, stream=stream)
    for call in range(4):  # odd n: each parity is seen twice, so both get captured
        direct.step(n)
        graphed.step(n)
        assert_same(state(direct), state(graphed))
    st = lbm.lbm_get_launch_stats(graphed.h)
    assert st["graphs_captured"] >= 1 and st["sweeps_replayed"] >= n - (n > 128)
    assert st["sweeps_direct"] + st["sweeps_replayed"] == 4 * n
    assert lbm.lbm_get_launch_stats(direct.h)["sweeps_replayed"] == 0


def test_pieces_end_at_diagnostic_sweeps(stream):
    """diag_every = 7 with calls of 50 steps: pieces of 7 (replayed) and the
    calls' tails; the history ring's melt fractions land on the same steps."""
    p = workloads.params(Ra=1e6, strip_center=0.6)
    lats = []
    for chunk in (0, 128):
        lat = lbm.Lattice(256, 128, p, precision="fp32", stream=stream)
        lbm.lbm_set_launch(lat.h, 1, 4, chunk)
        lbm.lbm_set_diag_every(lat.h, 7)
        lbm.lbm_set_history(lat.h, 256)
        for _ in range(4):
            lat.step(50)
        lats.append(lat)
    assert_same(state(lats[0]), state(lats[1]))
    h0 = lbm.lbm_read_history(lats[0].h, 256)
    h1 = lbm.lbm_read_history(lats[1].h, 256)
    assert np.array_equal(h0["step"], h1["step"]) and np.array_equal(h0["Q"], h1["Q"])
    assert np.array_equal(np.isnan(h0["melt"]), np.isnan(h1["melt"]))
    m = ~np.isnan(h0["melt"])
    assert np.array_equal(h0["melt"][m], h1["melt"][m])
    assert set(h0["step"][m]) == {s for s in range(1, 201) if s % 7 == 0 or s % 50 == 0}
    assert lbm.lbm_get_launch_stats(lats[1].h)["sweeps_replayed"] > 100


@pytest.mark.parametrize("prec", ["fp32", "fp16sr"])
def test_batch_pieces_replayed_equal_solo(stream, prec):
    """A serving quantum of 100 steps repeated: from the second quantum on the
    batch replays one captured 100-step piece; members stay bitwise equal to
    lattices stepped alone with direct launches."""
    cases = [(256, 128, dict(Ra=1e6, strip_center=0.2)), (300, 77, dict(Ra=1e5, strip_center=0.65)),
             (64, 32, dict())]
    solo = []
    for nx, ny, kw in cases:
        lat = lbm.Lattice(nx, ny, workloads.params(**kw), precision=prec, stream=stream)
        lbm.lbm_set_launch(lat.h, 1, 4, 0)
        for _ in range(4):
            lat.step(100)
        solo.append(lat)
    members = [lbm.Lattice(nx, ny, workloads.params(**kw), precision=prec, stream=stream)
               for nx, ny, kw in cases]
    b = lbm.Batch(4, stream)
    for lat in members:
        b.add(lat)
    for _ in range(4):
        b.step(100)
    for s, m in zip(solo, members):
        assert_same(state(s), state(m))
