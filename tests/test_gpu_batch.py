"""Batched stepping: lattices advanced together by one fused launch per step
must end bitwise where they end when stepped alone, whatever else is in the
batch, through membership changes, graph-replayed chunks and odd step counts;
and a member of a mixed batch must match the FP64 CPU oracle."""
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


CASES = [  # uneven grids, strip positions and Rayleigh numbers
    (256, 128, dict(Ra=1e6, strip_center=0.2)),
    (300, 77, dict(Ra=1e5, strip_center=0.65)),
    (64, 32, dict()),
    (130, 70, dict(Ra=1e7, strip_center=0.5, strip_width=0.4, seed=9)),
]


def make(stream, prec, nx, ny, kw):
    return lbm.Lattice(nx, ny, workloads.params(**kw), precision=prec, stream=stream)


def state(lat):
    f, g, step = lat.populations()
    return f, g, step, lat.diagnostics()


def assert_same(a, b):
    fa, ga, sa, da = a
    fb, gb, sb, db = b
    assert sa == sb
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert da == db


@pytest.mark.parametrize("prec", ["fp32", "fp16sr", "bf16"])
def test_batch_equals_solo(stream, prec):
    solo = [make(stream, prec, nx, ny, kw) for nx, ny, kw in CASES]
    for lat in solo:
        lat.step(150)
        lat.step(37)
    members = [make(stream, prec, nx, ny, kw) for nx, ny, kw in CASES]
    b = lbm.Batch(8, stream)
    for lat in members:
        b.add(lat)
    b.step(150)  # two graph-replayed chunks of 64 and 22 direct steps
    b.step(37)   # odd: every member's buffer parity flips
    for s, m in zip(solo, members):
        assert_same(state(s), state(m))


def test_batch_membership_changes(stream):
    prec = "fp32"
    a, c, d = (make(stream, prec, *CASES[k][:2], CASES[k][2]) for k in (0, 1, 2))
    b = lbm.Batch(4, stream)
    b.add(a)
    b.add(c)
    b.step(100)
    b.add(d)            # joins mid-run
    b.step(71)
    b.remove(a)         # leaves; stepped alone afterwards
    a.step(13)
    b.step(129)
    assert lbm.lbm_batch_count(b.b) == 2
    ref_a = make(stream, prec, *CASES[0][:2], CASES[0][2])
    ref_a.step(184)
    ref_c = make(stream, prec, *CASES[1][:2], CASES[1][2])
    ref_c.step(300)
    ref_d = make(stream, prec, *CASES[2][:2], CASES[2][2])
    ref_d.step(200)
    for ref, got in ((ref_a, a), (ref_c, c), (ref_d, d)):
        assert_same(state(ref), state(got))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_launch_shape_keeps_heated_wall_flux(stream, prec):
    """Rows per block change the number of blocks that fold the heated-wall
    inflow (row bands for the Stefan problem, tile columns for the cavity):
    the flux stays that of the default shape -- exactly for the cavity, whose
    heated wall is one row; to working-precision rounding for the Stefan
    problem, whose heated column's rows a thread sums before the FP64 fold."""
    cases = [(128, 4, workloads.stefan_1024x4(nx=128)[2]),
             (300, 77, workloads.params(Ra=1e6, strip_center=0.4))]
    for nx, ny, p in cases:
        tol = 1e-12 if prec == "fp64" or p["problem"] == lbm.LBM_CAVITY else 1e-6
        ref = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
        ref.step(40)
        lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
        lbm.lbm_set_launch(lat.h, 3, 4, 16)
        lat.step(40)
        fr, gr, sr, dr = state(ref)
        fl, gl, sl, dl = state(lat)
        assert sr == sl and np.array_equal(fr, fl) and np.array_equal(gr, gl)
        for k in ("Q_strip", "Q_cum", "Nu"):
            assert dl[k] == pytest.approx(dr[k], rel=tol, abs=1e-14), (nx, k)
        if prec == "fp32":
            assert dl["melt_fraction"] == dr["melt_fraction"] and dl["H_total"] == dr["H_total"]
            if p["problem"] == lbm.LBM_CAVITY:
                assert dl == dr


def test_batch_rejects_mixed_members(stream):
    b = lbm.Batch(2, stream)
    b.add(make(stream, "fp32", 64, 32, {}))
    with pytest.raises(lbm.LbmError):
        b.add(make(stream, "fp64", 64, 32, {}))
    with pytest.raises(lbm.LbmError):
        b.add(lbm.Lattice(128, 4, workloads.stefan_1024x4(nx=128)[2], stream=stream))
    b.add(make(stream, "fp32", 70, 40, {}))
    with pytest.raises(lbm.LbmError):
        b.add(make(stream, "fp32", 64, 32, {}))  # full


def test_autotune_leaves_state_and_caches(stream):
    nx, ny, p = 256, 128, workloads.params(Ra=1e6, strip_center=0.35)
    lat = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    lat.step(10)
    before = state(lat)
    t1 = lbm.lbm_autotune(lat.h, 50)
    assert t1["rows"] in (1, 2, 3, 4) and t1["prefetch"] in (0, 2, 4, 8, 16, 24, 32, 48)
    assert t1["us_per_step"] > 0
    assert_same(before, state(lat))          # the handle's state is untouched
    other = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    t2 = lbm.lbm_autotune(other.h, 50)
    assert t2["us_per_step"] == 0.0 and (t2["rows"], t2["prefetch"]) == (t1["rows"], t1["prefetch"])
    # a tuned lattice computes exactly what an untuned one does, diagnostics
    # included (FP32 sums are exact fixed-point sums, independent of grouping)
    ref = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    ref.step(60)
    lat.step(50)
    assert_same(state(ref), state(lat))


@pytest.mark.parametrize("batched", [False, True])
def test_history_ring_matches_step_by_step_diagnostics(stream, batched):
    """The device history (heated-wall inflow every step, melt fraction on the
    diagnostic steps) equals what step-by-step diagnostics report, also when the
    steps run as replayed graphs or inside a batch."""
    nx, ny, p = 200, 90, workloads.params(Ra=1e6, strip_center=0.45)
    ref = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    want = {}
    for _ in range(300):
        ref.step(1)
        d = ref.diagnostics()
        want[d["step"]] = (d["Q_strip"], d["Nu"], d["melt_fraction"])
    lat = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    lbm.lbm_set_history(lat.h, 512)
    lbm.lbm_set_diag_every(lat.h, 50)
    if batched:
        b = lbm.Batch(2, stream)
        b.add(lat)
        b.step(200)  # inside a batch diag_every does not apply: only the last step
        b.step(100)
        diag_steps = {200, 300}
    else:
        lat.step(300)
        diag_steps = {50, 100, 150, 200, 250, 300}
    h = lbm.lbm_read_history(lat.h, 1000)
    assert list(h["step"]) == list(range(1, 301))
    for s, q, nu, m in zip(h["step"], h["Q"], h["Nu"], h["melt"]):
        assert q == want[s][0] and nu == pytest.approx(want[s][1], rel=1e-14)
        if s in diag_steps:
            assert m == pytest.approx(want[s][2], rel=1e-6, abs=1e-12)
        else:
            assert np.isnan(m)
    assert lbm.lbm_read_history(lat.h, 10)["step"][0] == 291


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_member_matches_oracle(orc, stream, prec):
    """A member of a mixed batch (other sizes, Rayleigh numbers and strip
    positions around it) against the oracle: T and f_l within 1e-5 (FP32),
    every field within 1e-12 of its scale (FP64)."""
    if prec == "fp32":
        cases = [(256, 128, dict(Ra=1e6, strip_center=0.2))] + CASES[1:]
        steps = 300
    else:
        cases = [(64, 32, dict()), (130, 70, dict(Ra=1e7, strip_center=0.5, strip_width=0.4, seed=9)),
                 (67, 19, dict(Ra=1e5, strip_center=0.8))]
        steps = 400
    members = [make(stream, prec, nx, ny, kw) for nx, ny, kw in cases]
    b = lbm.Batch(8, stream)
    for lat in members:
        b.add(lat)
    b.step(steps)
    for k in ((0,) if prec == "fp32" else range(len(cases))):
        nx, ny, kw = cases[k]
        ref = orc.Oracle(nx, ny, threads=8, **workloads.params(**kw))
        ref.step(steps)
        want, got = ref.fields(), members[k].fields()
        if prec == "fp32":
            for name in ("T", "fl"):
                assert np.abs(got[name] - want[name]).max() <= 1e-5, (k, name)
        else:
            scale = {"H": 1.0, "T": 1.0, "fl": 1.0, "rho": 1.0, "ux": 0.1 / 3 ** 0.5, "uy": 0.1 / 3 ** 0.5}
            for name, sc in scale.items():
                err = np.abs(got[name] - want[name]).max() / max(np.abs(want[name]).max(), sc)
                assert err <= 1e-12, (k, name, err)
        d, dr = members[k].diagnostics(), ref.diagnostics()
        assert d["step"] == steps
        assert d["Q_cum"] == pytest.approx(dr["Q_cum"], rel=1e-5 if prec == "fp32" else 1e-12)


@pytest.mark.parametrize("rows,prefetch,interleave", [(1, 0, 1), (4, 16, 1), (1, 4, 0), (3, 8, 0)])
def test_batch_launch_shapes_equal_solo(stream, rows, prefetch, interleave):
    """Rows per block, prefetch distance and the interleaved block order of a
    one-size batch change no result: members end bitwise where solo runs do,
    diagnostics included (FP32 sums are exact fixed-point sums)."""
    cases = [(256, 128, dict(Ra=1e6, strip_center=c, seed=k)) for k, c in enumerate((0.2, 0.5, 0.8))]
    solo = [make(stream, "fp32", nx, ny, kw) for nx, ny, kw in cases]
    for lat in solo:
        lat.step(130)
    members = [make(stream, "fp32", nx, ny, kw) for nx, ny, kw in cases]
    b = lbm.Batch(4, stream)
    for lat in members:
        b.add(lat)
    lbm.lbm_batch_set_launch(b.b, rows, prefetch, interleave)
    b.step(130)
    for s, m in zip(solo, members):
        assert_same(state(s), state(m))


def test_batch_autotune_leaves_state_and_caches(stream):
    cases = [(256, 128, dict(Ra=1e6, strip_center=0.35)), (300, 77, dict(Ra=1e5)),
             (256, 128, dict(Ra=1e7, strip_center=0.65))]
    members = [make(stream, "fp32", nx, ny, kw) for nx, ny, kw in cases]
    b = lbm.Batch(4, stream)
    for lat in members:
        b.add(lat)
    b.step(10)
    before = [state(m) for m in members]
    t1 = lbm.lbm_batch_autotune(b.b, 30)
    assert t1["rows"] in (1, 2, 3, 4) and t1["prefetch"] in (0, 4, 8, 16) and t1["interleave"] == 0
    assert t1["us_per_step"] > 0
    for s0, m in zip(before, members):
        assert_same(s0, state(m))                     # the members' states are untouched
    other = [make(stream, "fp32", nx, ny, kw) for nx, ny, kw in cases]
    b2 = lbm.Batch(4, stream)
    for lat in other:
        b2.add(lat)
    t2 = lbm.lbm_batch_autotune(b2.b, 30)              # same composition: from the cache
    assert t2["us_per_step"] == 0.0
    assert (t2["rows"], t2["prefetch"], t2["interleave"]) == (t1["rows"], t1["prefetch"], t1["interleave"])
    b.step(90)
    solo = [make(stream, "fp32", nx, ny, kw) for nx, ny, kw in cases]
    for lat in solo:
        lat.step(100)
    for s, m in zip(solo, members):
        assert_same(state(s), state(m))


@pytest.mark.parametrize("rows", [1, 2, 3, 4])
def test_batch_row_bands_in_both_directions_match_oracle(orc, stream, rows):
    """Short members (1 to 10 row bands, ragged last bands) sweep their bands
    in the direction their own buffer parity picks: one member joined three
    steps late, so that members run in opposite directions within the same
    launches.  Every member against the oracle (FP64, 1e-12)."""
    p = workloads.params(Ra=1e5, strip_center=0.45, strip_width=0.3)
    heights = (3, 4, 5, 7, 10)
    members = [lbm.Lattice(130, ny, p, precision="fp64", stream=stream) for ny in heights]
    late = lbm.Lattice(130, 6, p, precision="fp64", stream=stream)
    late.step(3)
    b = lbm.Batch(8, stream)
    for lat in members + [late]:
        b.add(lat)
    lbm.lbm_batch_set_launch(b.b, rows, 2, 0)
    b.step(9)
    scale = {"H": 1.0, "T": 1.0, "fl": 1.0, "rho": 1.0, "ux": 0.1 / 3 ** 0.5, "uy": 0.1 / 3 ** 0.5}
    for ny, lat, steps in list(zip(heights, members, [9] * len(heights))) + [(6, late, 12)]:
        ref = orc.Oracle(130, ny, **p)
        ref.step(steps)
        want, got = ref.fields(), lat.fields()
        for name, sc in scale.items():
            err = np.abs(got[name] - want[name]).max() / max(np.abs(want[name]).max(), sc)
            assert err <= 1e-12, (ny, rows, name, err)
        assert lat.diagnostics()["Q_cum"] == pytest.approx(ref.diagnostics()["Q_cum"], rel=1e-12, abs=1e-15)
    b.close()
