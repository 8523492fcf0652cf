"""One-buffer streaming (lbm_set_streaming): the push and local sweeps of the
AA pattern, run in place in one buffer, must give bitwise the populations,
diagnostics, history and fields of two-buffer streaming -- for both problems,
with and without flow, every storage type, ragged lattices, odd and even call
lengths (direct and graph-replayed pieces, diagnostic steps inside the
one-buffer part), mode switches, launch shapes, batches and checkpoints."""
import numpy as np
import pytest

from paper_1909_13086_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu
ONE, TWO = lbm.LBM_STREAM_ONE_BUFFER, lbm.LBM_STREAM_TWO_BUFFERS


@pytest.fixture(scope="module")
def stream():
    import torch

    torch.cuda.set_device(0)
    return torch.cuda.Stream().cuda_stream


CASES = [
    ("cavity 300x77", 300, 77, workloads.params(Ra=1e6, strip_center=0.4)),
    ("cavity 130x9", 130, 9, workloads.params(Ra=1e5, strip_center=0.5, strip_width=0.6)),
    ("cavity 2x12", 2, 12, workloads.params(Ra=1e5)),
    ("cavity 257x33 flow off", 257, 33, workloads.params(Ra=1e5, flow_on=0)),
    ("stefan 300x8", 300, 8, workloads.stefan_1024x4(Ste=0.5, nx=300)[2]),
]


def state(lat):
    f, g, step = lat.populations()
    return f, g, step, lat.diagnostics(raise_on_diverged=False)


def assert_same(a, b, what):
    assert a[2] == b[2], what
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), what
    assert a[3] == b[3], what


def pair(stream, nx, ny, p, prec, diag_every=10):
    ref = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    lbm.lbm_set_streaming(lat.h, ONE)
    for L in (ref, lat):
        lbm.lbm_set_diag_every(L.h, diag_every)
    return ref, lat


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16sr", "fp16sr", "fp16", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_one_buffer_equals_two_buffers(stream, prec, case):
    name, nx, ny, p = case
    ref, lat = pair(stream, nx, ny, p, prec)
    for n in (1, 2, 3, 37, 200, 201, 200):  # odd and even calls; pieces direct, then replayed
        ref.step(n)
        lat.step(n)
        assert_same(state(ref), state(lat), (name, prec, n))
        # every call closes over two buffers, so the fields are recomputed from the
        # previous step's populations after calls of any length
        fa, fb = ref.fields(), lat.fields()
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), (name, prec, n, k)
    s = lbm.lbm_get_launch_stats(lat.h)
    assert s["sweeps_replayed"] > 0


def test_history_and_mode_switches(stream):
    nx, ny, p = 200, 60, workloads.params(Ra=1e6, strip_center=0.3)
    ref = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    lat = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    for L in (ref, lat):
        lbm.lbm_set_history(L.h, 1000)
        lbm.lbm_set_diag_every(L.h, 100)
    for mode, n in ((ONE, 123), (TWO, 77), (ONE, 299), (ONE, 1)):
        ref.step(n)   # the same calls: each call's last step enters the history with its melt fraction
        lbm.lbm_set_streaming(lat.h, mode)
        lat.step(n)
    assert_same(state(ref), state(lat), "switches")
    ha, hb = lbm.lbm_read_history(ref.h, 500), lbm.lbm_read_history(lat.h, 500)
    for k in ha:
        assert np.array_equal(np.asarray(ha[k]), np.asarray(hb[k]), equal_nan=True), k


@pytest.mark.parametrize("prec", ["fp32", "bf16sr"])
@pytest.mark.parametrize("rows,prefetch", [(1, 0), (1, 16), (2, 8), (3, 32), (4, 2)])
def test_launch_shapes(stream, prec, rows, prefetch):
    nx, ny, p = 260, 45, workloads.params(Ra=1e5, strip_center=0.6)
    ref, lat = pair(stream, nx, ny, p, prec, diag_every=0)
    lbm.lbm_set_launch(lat.h, rows, prefetch, 16)
    ref.step(121)
    lat.step(121)
    assert_same(state(ref), state(lat), (prec, rows, prefetch))


def test_checkpoint_batch_and_autotune(stream):
    """Checkpoint at step 200, resume on a fresh handle, tune, step, then step
    inside a batch: the same path with either streaming mode."""
    nx, ny, p = 256, 128, workloads.params(Ra=1e7, strip_center=0.65)
    out = []
    for mode in (TWO, ONE):
        lat = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
        lbm.lbm_set_streaming(lat.h, mode)
        lat.step(200)
        f, g, step = lat.populations()
        lat2 = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
        lbm.lbm_set_streaming(lat2.h, mode)
        lat2.set_populations(f, g, step)
        t = lbm.lbm_autotune(lat2.h, 20)     # one-buffer sweeps are tuned on a scratch lattice of that mode
        assert t["rows"] in (1, 2, 3, 4)
        lat2.step(100)
        b = lbm.Batch(2, stream)             # a batch steps its members over two buffers
        b.add(lat2)
        b.step(33)
        b.close()
        out.append(state(lat2))
    assert_same(out[0], out[1], "checkpoint + batch")


def test_full_size_one_buffer_fp32(stream):
    nx, ny, p = workloads.cavity_2048x1024()
    ref, lat = pair(stream, nx, ny, p, "fp32", diag_every=100)
    ref.step(301)
    lat.step(301)
    assert_same(state(ref), state(lat), "2048x1024")


def test_bad_mode(stream):
    lat = lbm.Lattice(64, 32, workloads.params(), precision="fp32", stream=stream)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_streaming(lat.h, 2)


BATCH = [(256, 128, dict(Ra=1e6, strip_center=0.2)), (300, 77, dict(Ra=1e5, strip_center=0.65)),
         (64, 32, dict()), (130, 9, dict(Ra=1e7, strip_center=0.5, strip_width=0.4, seed=9))]


@pytest.mark.parametrize("prec", ["fp32", "bf16sr", "fp64"])
@pytest.mark.parametrize("shape", [(0, -1, 1), (1, 0, 0), (3, 8, 1), (4, 2, 0)])
def test_batch_one_buffer_equals_two_buffers(stream, prec, shape):
    """Mixed sizes, one member a step ahead (its buffer parity differs from the
    others'), calls of odd and even length; the uniform-size case with the
    interleaved block order as well."""
    rows, pf, il = shape
    out = []
    for mode in (TWO, ONE):
        lats = [lbm.Lattice(nx, ny, workloads.params(**kw), precision=prec, stream=stream)
                for nx, ny, kw in BATCH]
        lats[1].step(1)
        same = [lbm.Lattice(128, 64, workloads.params(Ra=1e6, strip_center=c, seed=k), precision=prec,
                            stream=stream) for k, c in enumerate((0.2, 0.5, 0.8))]
        res = []
        for group in (lats, same):
            b = lbm.Batch(8, stream)
            for lat in group:
                b.add(lat)
            lbm.lbm_batch_set_streaming(b.b, mode)
            lbm.lbm_batch_set_launch(b.b, rows, pf, il)
            for n in (150, 37, 2, 1, 150, 37):  # pieces direct, then replayed
                b.step(n)
            b.close()
            res += [state(lat) for lat in group]
        out.append(res)
    for k, (a, b_) in enumerate(zip(*out)):
        assert_same(a, b_, (prec, shape, k))


def test_batch_bad_mode(stream):
    b = lbm.Batch(2, stream)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_set_streaming(b.b, 3)
    b.close()


@pytest.mark.parametrize("nx,ny,steps", [(2, 65535, 4), (262144, 2, 4), (129, 65535, 3)])
def test_extreme_shapes(stream, nx, ny, steps):
    """The tallest lattice the launch allows, a 2,048-tile strip and a ragged
    two-tile width at full height: the push sweep's targets across tile and
    wall edges at every size, against two-buffer streaming (FP32, bitwise)."""
    p = workloads.params(Ra=1e5, init_amp=0.1)
    ref, lat = pair(stream, nx, ny, p, "fp32", diag_every=0)
    ref.step(steps)
    lat.step(steps)
    assert_same(state(ref), state(lat), (nx, ny))
