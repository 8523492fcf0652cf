"""Continuous-batching server: every result is the one the request gets when
solved alone and, for the small FP32 requests, the oracle's; admission
respects the HBM budget; a failing request does not disturb the others."""
import numpy as np
import pytest

from paper_1909_13086_gb300 import lbm, serving

pytestmark = pytest.mark.gpu

_STREAMS = []


@pytest.fixture(scope="module")
def stream():
    import torch

    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    _STREAMS.append(s)
    return s.cuda_stream


def small_stream(n=8, steps=300):
    return serving.poisson_stream(n, rate_hz=200.0, seed=3, steps=steps,
                                  precisions=("fp32", "bf16sr", "fp16sr"),
                                  grids=((256, 128), (512, 256), (300, 77)), ras=(1e5, 1e6, 1e7))


def solo(r, stream):
    lat = lbm.Lattice(r.nx, r.ny, r.params(), precision=r.precision, stream=stream)
    lat.step(r.steps)
    d = lat.diagnostics(raise_on_diverged=False)
    f, g, _ = lat.populations()
    lat.close()
    return d, f, g


def test_each_result_equals_its_solo_run(stream):
    reqs = small_stream()
    results, makespan = serving.serve(reqs, 8 * 2 ** 30, quantum=100)
    assert len(results) == len(reqs) and all(x.ok for x in results)
    by_id = {r.rid: r for r in reqs}
    for x in results:
        d, _, _ = solo(by_id[x.rid], stream)
        assert x.diag == d  # bitwise: the batch computes exactly the solo steps


def test_admission_respects_hbm_budget(stream, monkeypatch):
    reqs = small_stream(6, 200)
    for r in reqs:  # equal footprints: the budget holds exactly two
        r.nx, r.ny, r.precision = 256, 128, "fp32"
    one = serving.footprint_bytes(256, 128, "fp32")
    budget = 2 * one + 1
    peaks = []
    orig = serving.Server.admit

    def admit(self, r, now):
        orig(self, r, now)
        assert self.used <= self.budget
        peaks.append(self.active)

    monkeypatch.setattr(serving.Server, "admit", admit)
    results, _ = serving.serve(reqs, budget, quantum=50)
    assert len(results) == len(reqs)
    assert max(peaks) <= 2


def test_failed_request_is_isolated(stream):
    reqs = small_stream(3, 200)
    for r in reqs:  # all in one group: same precision and size class
        r.precision, r.nx, r.ny = "fp32", 256, 128
    srv = serving.Server(8 * 2 ** 30, quantum=100)
    try:
        for r in reqs:
            srv.admit(r, 0.0)
        bad_rid = reqs[0].rid
        (g,) = srv.groups.values()
        _, lat, _ = g.members[bad_rid]
        f, gg, step = lat.populations()
        gg[0, 5, 5] = np.nan
        lat.set_populations(f, gg, step)
        seen = 0
        while srv.active:
            srv.launch()
            for x in srv.poll(lambda: 0.0, block=True):
                seen += 1
                if x.rid == bad_rid:
                    assert not x.ok and x.diag["nan_flag"] == 1
                else:
                    assert x.ok
                    d, _, _ = solo(next(r for r in reqs if r.rid == x.rid), stream)
                    assert x.diag == d
        assert seen == 3
    finally:
        srv.close()


def test_served_fp32_results_match_oracle(orc):
    """Requests served together with others (mixed sizes, precisions and
    Rayleigh numbers): every small FP32 one ends, field by field, within 1e-5
    of the oracle in T and f_l."""
    reqs = small_stream(10, 300)
    results, _ = serving.serve(reqs, 8 * 2 ** 30, quantum=100, keep_fields=True)
    by_id = {r.rid: r for r in reqs}
    checked = 0
    for x in results:
        r = by_id[x.rid]
        if r.precision != "fp32" or r.nx * r.ny > 256 * 128:
            continue
        ref = orc.Oracle(r.nx, r.ny, threads=8, **r.params())
        ref.step(r.steps)
        want = ref.fields()
        for name in ("T", "fl"):
            assert np.abs(x.fields[name] - want[name]).max() <= 1e-5, (r.rid, name)
        assert x.diag["Q_cum"] == pytest.approx(ref.diagnostics()["Q_cum"], rel=1e-5)
        checked += 1
    assert checked >= 1
