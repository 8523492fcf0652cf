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
