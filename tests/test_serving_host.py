"""Host logic of the serving loop (no GPU): stream generation, footprints,
summaries."""
import numpy as np

from paper_1909_13086_gb300 import serving


def test_poisson_stream_is_seeded_and_poisson():
    a = serving.poisson_stream(2000, rate_hz=50.0, seed=7)
    b = serving.poisson_stream(2000, rate_hz=50.0, seed=7)
    assert [(r.arrival, r.nx, r.Ra, r.center, r.precision) for r in a] == \
        [(r.arrival, r.nx, r.Ra, r.center, r.precision) for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert abs(gaps.mean() - 1 / 50.0) < 0.1 / 50.0       # exponential mean 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1      # coefficient of variation 1
    assert {(r.nx, r.ny) for r in a} == set(serving.GRIDS)
    assert {r.center for r in a} == set(serving.CENTERS)
    for r in a:  # strip of width W/4 stays on the wall
        assert 0.0 <= r.center - 0.125 and r.center + 0.125 <= 1.0


def test_footprint_counts_both_buffers_of_18_tiled_planes():
    assert serving.footprint_bytes(2048, 1024, "fp32") >= 2 * 18 * 2048 * 1024 * 4
    assert serving.footprint_bytes(2048, 1024, "bf16sr") < serving.footprint_bytes(2048, 1024, "fp32")
    # ragged widths are padded to 128-cell tiles
    assert serving.footprint_bytes(130, 10, "fp32") >= 2 * 18 * 256 * 10 * 4


def test_summary_percentiles_and_mlups():
    reqs = [serving.Request(i, 0.0, 100, 10, 1e6, 0.5, "fp32", 10) for i in range(100)]
    res = [serving.Result(i, 0.0, 0.0, float(i + 1), True, {}) for i in range(100)]
    s = serving.summarize(res, reqs, makespan=100.0)
    assert s["p50_s"] == np.percentile(np.arange(1, 101), 50)
    assert s["p99_s"] == np.percentile(np.arange(1, 101), 99)
    assert s["mlups"] == 100 * 1000 * 10 / 100.0 / 1e6
