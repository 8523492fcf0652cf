"""Host logic of the full-melting study (Sec. 3.2): threshold crossings, the
batch membership as cavities finish, and checkpoint / resume -- on CPU, with a
fake lattice whose melt fraction grows at a fixed rate per step."""
import numpy as np
import pytest

from paper_1909_13086_gb300 import studies


class FakeLattice:
    def __init__(self, rate, n=8):
        self.rate, self.n, self.step_ = rate, n, 0
        self.f = np.zeros((9, n, n))
        self.g = np.zeros((9, n, n))

    def derived(self):
        return {"alpha": 0.01}

    def advance(self, k):
        self.step_ += k
        self.f += k          # the "state" remembers every step taken
        self.g -= 0.5 * k

    def diagnostics(self, raise_on_diverged=True):
        return {"step": self.step_, "melt_fraction": min(1.0, self.rate * self.step_),
                "Nu": 2.0, "nan_flag": 0}

    def populations(self):
        return self.f.copy(), self.g.copy(), self.step_

    def set_populations(self, f, g, step):
        self.f, self.g, self.step_ = np.array(f, np.float64), np.array(g, np.float64), step

    def close(self):
        pass


class FakeBatch:
    def __init__(self, k, log):
        self.members, self.log = [], log

    def add(self, lat):
        self.members.append(lat)

    def remove(self, lat):
        self.members.remove(lat)

    def step(self, k):
        self.log.append(len(self.members))
        for m in self.members:
            m.advance(k)

    def close(self):
        pass


RATES = {0.25: 1.0 / 4000, 0.375: 1.0 / 3000, 0.5: 1.0 / 2000}


def run(tmp_path=None, max_seconds=None, fo_max=10.0, log=None):
    log = [] if log is None else log
    return studies.cavity_full_melt(
        n=8, centers=tuple(RATES), fo_max=fo_max, sample_fo=0.05, precision="fp32",
        checkpoint=None if tmp_path is None else str(tmp_path / "ck.npz"), max_seconds=max_seconds,
        make_lattice=lambda C: FakeLattice(RATES[C]), make_batch=lambda k: FakeBatch(k, log))


def test_crossing_interpolates_and_reports_never():
    h = [(0.1, 0.2, 1.0, 0.0), (0.2, 0.6, 1.0, 0.0), (0.3, 0.95, 1.0, 0.0)]
    assert studies.crossing_fo(h, 0.5) == pytest.approx(0.175)
    assert studies.crossing_fo(h, 0.2) == 0.1            # reached at the first sample
    assert studies.crossing_fo(h, 0.99) is None
    assert studies.crossing_fo([], 0.5) is None


def test_cavities_leave_the_batch_as_they_melt():
    log = []
    res = run(log=log)
    # chunk = 0.05 * 64 / 0.01 = 320 steps; Fo = step / 6400, melt = 6400 rate Fo,
    # so 0.99 is reached after 7 (C = 0.5), 10 (0.375) and 13 (0.25) samples
    assert res["steps_per_sample"] == 320
    assert log == [3] * 7 + [2] * 3 + [1] * 3
    r = res["runs"]
    assert [r[str(C)]["state"] for C in RATES] == ["melted"] * 3
    for C, rate in RATES.items():
        h = r[str(C)]["history"]
        assert h[0] == (0.0, 0.0, 2.0, 0.0)           # the initial state comes first
        for lv in (0.5, 0.9):                          # linear between the samples
            assert r[str(C)]["fo_at"][str(lv)] == pytest.approx(lv / (6400 * rate))
    fo99 = [r[str(C)]["fo_at"]["0.99"] for C in RATES]
    assert fo99[2] < fo99[1] < fo99[0]                 # the centred strip melts first


def test_fo_max_stops_unmelted_cavities():
    res = run(fo_max=0.1)
    assert {r["state"] for r in res["runs"].values()} == {"fo_max"}


def test_resume_from_checkpoint_equals_uninterrupted(tmp_path):
    straight = run()
    calls = 0
    while True:
        calls += 1
        res = run(tmp_path, max_seconds=0.0)   # stops after every sample
        if res["complete"]:
            break
        assert calls < 30
    assert calls == 13  # one sample per call
    assert res["runs"] == straight["runs"]
    z = np.load(tmp_path / "ck.npz")
    assert z["f0"].dtype == np.float32 and int(z["step0"]) == 13 * 320
    assert np.all(z["f0"] == 13 * 320) and str(z["state2"]) == "melted"


def test_checkpoint_of_another_run_and_16_bit_are_rejected(tmp_path):
    run(tmp_path, max_seconds=0.0)
    with pytest.raises(ValueError):
        studies.cavity_full_melt(
            n=8, centers=(0.25, 0.5), sample_fo=0.5, checkpoint=str(tmp_path / "ck.npz"),
            make_lattice=lambda C: FakeLattice(RATES[C]), make_batch=lambda k: FakeBatch(k, []))
    with pytest.raises(ValueError):
        studies.cavity_full_melt(n=8, precision="bf16sr", checkpoint=str(tmp_path / "x.npz"))


class FakeRun:
    """Melt fraction and inflow growing at fixed rates; `bias` stands in for a
    storage precision's departure from the FP64 run."""
    def __init__(self, bias):
        self.bias, self.n = bias, 0

    def step(self, k):
        self.n += k

    def diagnostics(self, raise_on_diverged=True):
        return {"melt_fraction": 1e-5 * self.n * (1.0 + self.bias), "Q_cum": 2.0 * self.n * (1.0 + self.bias),
                "nan_flag": 0}

    def close(self):
        pass


def test_precision_study_compares_each_precision_with_fp64():
    bias = {"fp64": 0.0, "fp32": 1e-3, "bf16sr": -0.02}
    rows = studies.precision_study(steps=2500, every=1000, centers=(0.25, 0.5),
                                   precisions=("fp32", "bf16sr"),
                                   make_lattice=lambda C, prec: FakeRun(bias[prec]))
    assert [(r["C"], r["precision"]) for r in rows] == [(0.25, "fp32"), (0.25, "bf16sr"),
                                                         (0.5, "fp32"), (0.5, "bf16sr")]
    for r in rows:
        b = bias[r["precision"]]
        # samples after 1000, 2000 and the last 500 steps: the largest gap is at the end
        assert r["melt_err_max"] == pytest.approx(abs(b) * 1e-5 * 2500)
        assert r["mean_nu_rel_err"] == pytest.approx(b)
        assert r["final_melt_fp64"] == pytest.approx(1e-5 * 2500)


def test_compare_to_fp64_rejects_different_sampling():
    with pytest.raises(ValueError):
        studies.compare_to_fp64({"melt": [0.1, 0.2], "Q_cum": 1.0, "final_melt": 0.2, "nan_flag": 0},
                                {"melt": [0.1], "Q_cum": 1.0, "final_melt": 0.1, "nan_flag": 0})


class FakeSoloLattice(FakeLattice):
    """A lattice stepped on its own (the single-lattice path)."""
    def step(self, k):
        self.advance(k)


def test_production_full_melt_uses_the_cavity_height_for_fo():
    """Fo = alpha t / H^2 with H = 1024 (not the width), one sample every
    0.002 of Fo, the run ends at melt fraction 0.99 and reports its steps."""
    rate = 1.0 / 2e7   # melt fraction per step: 0.99 after 1.98e7 steps
    res = studies.production_full_melt(sample_fo=0.002, make_lattice=lambda C: FakeSoloLattice(rate))
    H2, alpha = 1024.0 ** 2, 0.01
    assert res["steps_per_sample"] == round(0.002 * H2 / alpha)
    run = res["runs"]["0.5"]
    assert run["state"] == "melted" and res["complete"]
    # the crossing of 0.5, interpolated between samples, sits at 1e7 steps
    assert run["fo_at"]["0.5"] == pytest.approx(1e7 * alpha / H2, rel=1e-9)
    assert res["steps"] == round(run["final"][0] * H2 / alpha)
    assert res["nx"] == 2048 and res["ny"] == 1024 and res["mlups_wall"] > 0
