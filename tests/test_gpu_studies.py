"""The paper's Sec. 3.1 study as numbers: with k1 + k2 = 2 (Eq. 6) the solid
ahead of the front stays at T_m and the interface is one cell wide for every
k1 of the paper's list, while SRT departs from both whenever k1 != 1."""
import pytest

from paper_1909_13086_gb300 import studies

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sweep():
    import torch

    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    rows = studies.stefan_k1_sweep("fp64", s.cuda_stream)
    return {(r["k1"], r["model"]): r for r in rows}


@pytest.mark.parametrize("k1", [0.1, 0.5, 1.0, 1.5])
def test_btrirt_keeps_solid_at_tm_and_one_cell_interface(sweep, k1):
    r = sweep[(k1, "btrirt")]
    assert r["solid_departure_from_Tm"] <= 1e-12
    assert r["interface_width_cells"] <= 1
    assert abs(r["front_cells"] - r["front_neumann_cells"]) <= 1.0
    assert r["max_T_error"] <= 0.05


@pytest.mark.parametrize("k1", [0.1, 0.5, 1.5])
def test_srt_departs_when_k1_is_not_1(sweep, k1):
    r = sweep[(k1, "srt")]
    assert r["solid_departure_from_Tm"] > 1e-6 or r["interface_width_cells"] > 1


def test_srt_equals_btrirt_at_k1_1(sweep):
    a, b = sweep[(1.0, "srt")], sweep[(1.0, "btrirt")]
    assert a["max_T_error"] == b["max_T_error"] and a["front_cells"] == b["front_cells"]


def test_full_melt_study_resumes_bitwise(tmp_path):
    """Sec. 3.2's cavities in one batch: a run stopped after every sample and
    resumed from its FP32 checkpoint ends exactly where an uninterrupted run
    ends (128 x 128 here, a few thousandths of the Fourier time)."""
    import torch

    torch.cuda.set_device(0)
    s = torch.cuda.Stream().cuda_stream
    kw = dict(n=128, fo_max=0.001, sample_fo=0.00025, stream=s)
    straight = studies.cavity_full_melt(**kw)
    calls = 0
    while True:
        calls += 1
        res = studies.cavity_full_melt(checkpoint=str(tmp_path / "ck.npz"), max_seconds=0.0, **kw)
        if res["complete"]:
            break
        assert calls < 10
    assert calls >= 4
    assert res["runs"] == straight["runs"]
    for r in straight["runs"].values():
        assert r["state"] == "fo_max"
        h = r["history"]
        assert h[0][0] == 0.0 and all(row[3] == 0.0 for row in h)
        assert h[-1][1] > h[0][1]  # melting has started
