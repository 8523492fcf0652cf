"""CUDA path vs the FP64 CPU oracle, through the C ABI.

Bars: FP64 GPU path within 1e-12 of the oracle relative to each field's (or
population plane set's) largest magnitude; FP32 path within 1e-5 max-abs in T
and f_l after 1000 steps.  Sizes: the 64 x 32 cavity, ragged lattices that do
not fill a 256-wide block, the 1024 x 4 Stefan problem, and the full 2048 x
1024 production cavity in the launch configuration the benchmark times
(sampled cells after a pull sweep; every cell after a call of one-buffer
sweeps).
"""
import math

import numpy as np
import pytest

from paper_1909_13086_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu

FIELDS = ("H", "T", "fl", "ux", "uy", "rho")


_STREAMS = []


@pytest.fixture(scope="module")
def stream():
    """A dedicated CUDA stream lent to the library (kept alive for the module)."""
    import torch

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    _STREAMS.append(s)
    return s.cuda_stream


# Characteristic scale of each field: Delta T = 1 for H and T, 1 for f_l and
# rho, the free-fall velocity U = Ma c_s (Ma = 0.1) for u.  Errors are taken
# relative to max(|field|, scale): a velocity of 1e-6 is formed from O(0.1)
# populations, so its rounding is ~1e-17 absolute, not 1e-12 of 1e-6.
SCALE = {"H": 1.0, "T": 1.0, "fl": 1.0, "rho": 1.0, "ux": 0.1 / math.sqrt(3), "uy": 0.1 / math.sqrt(3)}


def rel_err(got, want, scale=0.0):
    s = max(np.abs(want).max(), scale)
    return np.abs(got - want).max() / (s if s > 0 else 1.0)


def assert_fields_fp64(got, want, tol=1e-12, names=FIELDS):
    for k in names:
        e = rel_err(got[k], want[k], SCALE[k])
        assert e <= tol, f"field {k}: relative error {e:.3e} > {tol:.1e}"


def run_pair(orc, nx, ny, p, steps, prec, stream, threads=4):
    ref = orc.Oracle(nx, ny, threads=threads, **p)
    ref.step(steps)
    lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    lat.step(steps)
    return ref, lat


# ------------------------------------------------------------ FP64 parity
def test_fp64_cavity_64x32_2000_steps(orc, stream):
    nx, ny, p = workloads.cavity_64x32()
    ref, lat = run_pair(orc, nx, ny, p, 2000, "fp64", stream)
    assert_fields_fp64(lat.fields(), ref.fields())
    f, g, step = lat.populations()
    fr, gr = ref.populations()
    assert step == 2000
    assert rel_err(f, fr) <= 1e-12 and rel_err(g, gr) <= 1e-12
    d, dr = lat.diagnostics(), ref.diagnostics()
    for k in ("melt_fraction", "H_total", "Q_strip", "Q_cum", "Nu", "front_x", "max_u"):
        assert d[k] == pytest.approx(dr[k], rel=1e-12, abs=1e-15), k
    assert d["step"] == 2000 and d["nan_flag"] == 0


@pytest.mark.parametrize("nx,ny,steps", [(67, 19, 400), (300, 37, 300), (2, 2, 50), (513, 3, 100)])
def test_fp64_ragged_lattices(orc, stream, nx, ny, steps):
    p = workloads.params(Ra=1e5, strip_center=0.45, strip_width=0.3)
    ref, lat = run_pair(orc, nx, ny, p, steps, "fp64", stream)
    assert_fields_fp64(lat.fields(), ref.fields())
    d, dr = lat.diagnostics(), ref.diagnostics()
    assert d["Q_cum"] == pytest.approx(dr["Q_cum"], rel=1e-12)
    assert d["melt_fraction"] == pytest.approx(dr["melt_fraction"], rel=1e-12, abs=1e-16)


def test_fp64_step_zero_and_every_step(orc, stream):
    """Fields and diagnostics agree at step 0 and after each of the first steps."""
    nx, ny, p = 48, 20, workloads.params(Ra=1e5)
    ref = orc.Oracle(nx, ny, **p)
    lat = lbm.Lattice(nx, ny, p, precision="fp64", stream=stream)
    for n in range(6):
        if n:
            ref.step(1)
            lat.step(1)
        assert_fields_fp64(lat.fields(), ref.fields())
        d, dr = lat.diagnostics(), ref.diagnostics()
        assert d["step"] == n
        for k in ("melt_fraction", "H_total", "Q_strip", "Q_cum"):
            assert d[k] == pytest.approx(dr[k], rel=1e-12, abs=1e-15), (n, k)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("problem", ["cavity", "stefan"])
def test_single_step_from_random_state(orc, stream, prec, tol, problem):
    """Arbitrary non-equilibrium populations (solid, mushy and liquid cells,
    every wall rule) advanced by one step on both sides."""
    if problem == "cavity":
        nx, ny, p = 70, 33, workloads.params(Ra=1e6, strip_center=0.4, strip_width=0.35)
    else:
        nx, ny, p = workloads.stefan_1024x4(Ste=0.5, alpha=0.1, k2=0.7, k0=1.2, nx=90)
    f, g = workloads.random_populations(nx, ny, seed=11)
    if prec == "fp32":  # both sides start from the same FP32-representable state
        f, g = f.astype(np.float32).astype(np.float64), g.astype(np.float32).astype(np.float64)
    ref = orc.Oracle(nx, ny, **p)
    ref.set_populations(f, g, step=7)
    ref.step(1)
    lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    lat.set_populations(f, g, step=7)
    lat.step(1)
    fo, go, step = lat.populations()
    fr, gr = ref.populations()
    assert step == 8
    assert np.abs(go - gr).max() <= tol * max(1.0, np.abs(gr).max())
    if p["flow_on"]:
        assert np.abs(fo - fr).max() <= tol * max(1.0, np.abs(fr).max())
    got, want = lat.fields(), ref.fields()
    for k in FIELDS:
        assert np.abs(got[k] - want[k]).max() <= tol * max(1.0, np.abs(want[k]).max()), k
    assert lat.diagnostics()["Q_strip"] == pytest.approx(ref.diagnostics()["Q_strip"], rel=10 * tol,
                                                         abs=10 * tol)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("nx", [2, 31, 33, 128, 129, 256])
def test_side_wall_columns_from_random_state(orc, stream, prec, tol, nx):
    """Side-wall warps of the cavity take the fast loads and bounce their wall
    lane back: checked where a warp touches both walls (2, 31), where the last
    column is a lone lane of a later warp (33, 129) and where it ends a tile
    (128, 256), one step from arbitrary populations."""
    ny, p = 9, workloads.params(Ra=1e6, strip_center=0.5, strip_width=0.5)
    f, g = workloads.random_populations(nx, ny, seed=nx)
    if prec == "fp32":
        f, g = f.astype(np.float32).astype(np.float64), g.astype(np.float32).astype(np.float64)
    ref = orc.Oracle(nx, ny, **p)
    ref.set_populations(f, g, step=3)
    ref.step(1)
    lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    lat.set_populations(f, g, step=3)
    lat.step(1)
    fo, go, _ = lat.populations()
    fr, gr = ref.populations()
    assert np.abs(go - gr).max() <= tol * max(1.0, np.abs(gr).max())
    assert np.abs(fo - fr).max() <= tol * max(1.0, np.abs(fr).max())


# ------------------------------------------------------------ FP32 parity
def test_fp32_cavity_1000_steps(orc, stream):
    nx, ny, p = workloads.cavity_64x32()
    ref, lat = run_pair(orc, nx, ny, p, 1000, "fp32", stream)
    got, want = lat.fields(), ref.fields()
    for k in ("T", "fl"):
        e = np.abs(got[k] - want[k]).max()
        assert e <= 1e-5, f"{k}: max-abs error {e:.3e}"
    d, dr = lat.diagnostics(), ref.diagnostics()
    assert d["melt_fraction"] == pytest.approx(dr["melt_fraction"], abs=1e-5)


# ------------------------------------------------------------ Stefan
def test_stefan_fp64_field_parity(orc, stream):
    nx, ny, p = workloads.stefan_1024x4(Ste=1.0)
    ref, lat = run_pair(orc, nx, ny, p, 10000, "fp64", stream, threads=8)
    assert_fields_fp64(lat.fields(), ref.fields(), names=("H", "T", "fl"))
    assert lat.diagnostics()["front_x"] == pytest.approx(ref.diagnostics()["front_x"], rel=1e-12)


def fp32_drift_bound(n, H_max):
    """Four standard deviations of the enthalpy drift that FP32 storage of the
    populations allows after n steps: each step rounds the stored values once,
    so the error of a cell's H walks randomly with steps of about
    ulp(H_max) / sqrt(12) -- the latent-heat population g_0 ~ f_l L dominates
    H_max = 1 + L.  For the 64 x 32 cavity (L = 1) at 1000 steps this is
    8.7e-6, inside the 1e-5 bar; after 1e4 steps it is 2.8e-5 at Ste 1 and
    1.1e-4 at Ste 0.1 (L = 10)."""
    ulp = 2.0 ** (math.floor(math.log2(H_max)) - 23)
    return 4.0 * math.sqrt(n) * ulp / math.sqrt(12.0)


@pytest.mark.parametrize("Ste", [0.1, 1.0])
def test_stefan_fp32_field_parity_1e4_steps(orc, stream, Ste):
    """The FP32 path over 1e4 steps of the 1024 x 4 Stefan problem, cell by
    cell against the oracle.  T everywhere within the FP32 storage drift
    bound.  The phase field: the same cells solid, mushy and liquid; in the
    mushy cell f_l is the heat that has crossed into it from its liquid
    neighbour (at T_n above T_m) divided by L, so a drift dT of that
    neighbour's temperature is a relative error dT / T_n of the flux it
    integrates, and the same error in f_l (Stefan condition, Eqs. 7-8)."""
    nx, ny, p = workloads.stefan_1024x4(Ste=Ste)
    n = 10000
    ref, lat = run_pair(orc, nx, ny, p, n, "fp32", stream, threads=8)
    got, want = lat.fields(("H", "T", "fl")), ref.fields()
    tol_T = max(1e-5, fp32_drift_bound(n, 1.0 + 1.0 / Ste))
    e = np.abs(got["T"] - want["T"]).max()
    assert e <= tol_T, f"T: max-abs error {e:.3e} > {tol_T:.3e}"
    fl, flr = got["fl"], want["fl"]
    assert np.array_equal(fl == 0.0, flr == 0.0) and np.array_equal(fl == 1.0, flr == 1.0)
    front_err = 0.0
    for row in range(ny):
        (mushy,) = np.nonzero((flr[row] > 0.0) & (flr[row] < 1.0))
        assert mushy.size == 1 and mushy[0] > 0
        x = mushy[0]
        tol_fl = tol_T / want["T"][row, x - 1]
        assert abs(fl[row, x] - flr[row, x]) <= tol_fl, (row, fl[row, x] - flr[row, x], tol_fl)
        front_err = max(front_err, tol_fl)
    assert lat.diagnostics()["front_x"] == pytest.approx(ref.diagnostics()["front_x"], abs=front_err)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("Ste", [0.1, 1.0])
def test_stefan_front_matches_neumann(orc, stream, prec, Ste):
    """Front within one cell of X = 2 lambda sqrt(alpha t) from 1e3 steps on,
    and within 1 % (2 % at Ste 0.1, where X(1e5) is only 57 cells) at 1e5."""
    nx, ny, p = workloads.stefan_1024x4(Ste=Ste)
    lam = orc.stefan_lambda(Ste)
    alpha = p["alpha_override"]
    lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    done = 0
    for n in (1000, 3000, 10000, 30000, 100000):
        lat.step(n - done)
        done = n
        X = 2 * lam * math.sqrt(alpha * n)
        xf = lat.diagnostics()["front_x"]
        assert abs(xf - X) <= 1.0, (n, xf, X)
    assert xf == pytest.approx(X, rel=0.02 if Ste < 0.5 else 0.01)
    T = lat.fields(("T",))["T"][0]
    x = np.arange(nx) + 0.5
    liquid = x < X - 1.0
    Tn = np.array([orc.neumann_T(xx, done, alpha, lam) for xx in x[liquid]])
    assert np.abs(T[liquid] - Tn).max() <= 1e-2


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("fp32", 1e-6)])
def test_one_cell_interface_on_gpu(stream, prec, tol):
    """Eq. 6: with k1 + k2 = 2 the solid ahead of the front stays at H_s and
    the interface is one cell wide (checked every 50 steps)."""
    alpha = (1.0 / 1.5 - 0.5) / 3.0  # k1 = 1.5 through Eq. 5
    nx, ny, p = workloads.stefan_1024x4(Ste=0.1, alpha=alpha, k2=0.5, nx=256)
    lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    eps = 1e-12 if prec == "fp64" else 1e-5
    for _ in range(40):
        lat.step(50)
        F = lat.fields(("H", "fl"))
        fl, H = F["fl"], F["H"]
        assert ((fl > eps) & (fl < 1 - eps)).sum(axis=1).max() <= 1
        for row in range(ny):
            melted = np.nonzero(fl[row] > eps)[0]
            edge = melted.max() if melted.size else -1
            assert np.abs(H[row, edge + 1:]).max(initial=0.0) <= tol


# ------------------------------------------------------------ invariants
def test_mirror_symmetry_gpu(stream):
    nx, ny = 128, 64
    p = workloads.params(Ra=1e5, init_amp=0.0)
    lat = lbm.Lattice(nx, ny, p, precision="fp64", stream=stream)
    lat.step(1500)
    F = lat.fields()
    assert F["fl"].max() > 0
    for k in ("H", "T", "fl", "uy", "rho"):
        a = F[k]
        assert np.abs(a - a[:, ::-1]).max() <= max(1e-12 * np.abs(a).max(), 1e-14), k
    assert np.abs(F["ux"] + F["ux"][:, ::-1]).max() <= max(1e-12 * np.abs(F["ux"]).max(), 1e-14)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_energy_budget_gpu(stream, prec):
    nx, ny, p = workloads.cavity_64x32()
    lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    h0 = lat.diagnostics()["H_total"]
    lat.step(3000)
    d = lat.diagnostics()
    tol = 1e-12 if prec == "fp64" else 1e-4
    assert abs(d["H_total"] - h0 - d["Q_cum"]) <= tol * d["Q_cum"]


def test_checkpoint_resume_is_bitwise(stream):
    nx, ny, p = 96, 40, workloads.params(Ra=1e5)
    for prec in ("fp64", "fp32"):
        a = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
        a.step(400)
        fa, ga, _ = a.populations()
        b = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
        b.step(200)
        f, g, step = b.populations()
        c = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
        c.set_populations(f, g, step)
        c.step(200)
        fc, gc, stepc = c.populations()
        assert stepc == 400
        assert np.array_equal(fa, fc) and np.array_equal(ga, gc)


def test_deterministic_diagnostics(stream):
    nx, ny, p = 700, 300, workloads.params(Ra=1e6)
    runs = []
    for _ in range(2):
        lat = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
        lat.step(100)
        runs.append(lat.diagnostics())
    assert runs[0] == runs[1]


# ------------------------------------------------------------ errors
def test_errors_and_edge_cases(stream):
    nx, ny, p = workloads.cavity_64x32()
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(1, 8, p, stream=stream)
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(nx, ny, dict(p, k0=2.5), stream=stream)
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(nx, ny, dict(p, Ste=0.0), stream=stream)
    lat = lbm.Lattice(nx, ny, p, stream=stream)
    lat.step(0)
    assert lat.diagnostics()["step"] == 0
    with pytest.raises(lbm.LbmError):
        lat.step(-1)
    f, g, _ = lat.populations()
    lat.set_populations(f, g, 5)
    with pytest.raises(lbm.LbmError) as e:
        lat.fields()
    assert e.value.status == lbm.LBM_ERR_STATE
    with pytest.raises(lbm.LbmError) as e:
        lat.diagnostics()
    assert e.value.status == lbm.LBM_ERR_STATE
    # a non-finite state is reported, not hidden
    g = g.copy()
    g[0, 3, 4] = np.nan
    lat.set_populations(f, g, 0)
    lat.step(1)
    d = lat.diagnostics(raise_on_diverged=False)
    assert d["nan_flag"] == 1
    with pytest.raises(lbm.LbmError) as e:
        lat.diagnostics()
    assert e.value.status == lbm.LBM_ERR_DIVERGED


def test_torch_allocator_hook(orc, stream):
    import torch

    lbm.use_torch_allocator()
    try:
        before = torch.cuda.memory_allocated()
        nx, ny, p = workloads.cavity_64x32()
        lat = lbm.Lattice(nx, ny, p, precision="fp64", stream=stream)
        assert torch.cuda.memory_allocated() > before
        lat.step(100)
        ref = orc.Oracle(nx, ny, **p)
        ref.step(100)
        assert_fields_fp64(lat.fields(), ref.fields())
        lat.close()
        assert torch.cuda.memory_allocated() == before
    finally:
        lbm.use_default_allocator()


def test_allocation_failure_is_reported(stream):
    """An allocator that refuses every request (a full device or a spent arena)
    makes lbm_create and lbm_batch_create fail with LBM_ERR_OOM; nothing is
    freed that was not allocated, and the library works again once the default
    allocator is back."""
    asked, freed = [], []

    def _alloc(nbytes, ctx):
        asked.append(nbytes)
        return None

    def _free(ptr, ctx):
        freed.append(ptr)

    hooks = (lbm.ALLOC_FN(_alloc), lbm.FREE_FN(_free))
    lbm._check(lbm.lib().lbm_set_allocator(hooks[0], hooks[1], None))
    try:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(64, 32, lbm.PRECISIONS["fp32"], stream)
        assert e.value.status == lbm.LBM_ERR_OOM and asked
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_batch_create(4, stream)
        assert e.value.status == lbm.LBM_ERR_OOM
        assert freed == []
    finally:
        lbm.use_default_allocator()
    nx, ny, p = workloads.cavity_64x32()
    lat = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    lat.step(10)
    assert lat.diagnostics()["step"] == 10
    lat.close()


# ------------------------------------------------------------ full size
def test_full_size_sampled_parity_fp32(orc, stream):
    """2048 x 1024 production cavity, FP32, the benchmark's launch shape: one
    step from the GPU's own step-(n-1) populations recomputed by the oracle on
    sampled cells (every boundary row and column, the strip edges, random
    interior cells)."""
    nx, ny, p = workloads.cavity_2048x1024()
    lat = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    lat.step(30)
    fprev, gprev, _ = lat.populations()
    lat.step(1)
    fnew, gnew, _ = lat.populations()
    F = lat.fields()
    ref = orc.Oracle(nx, ny, **p)
    rng = np.random.default_rng(5)
    d = ref.derived()
    cells = [(x, y) for x in (0, 1, nx - 2, nx - 1) for y in range(0, ny, 97)]
    cells += [(x, y) for y in (0, 1, ny - 2, ny - 1) for x in range(0, nx, 61)]
    for xs in (int(math.floor(d["a"])) + k for k in (-2, -1, 0, 1)):
        cells += [(xs, 0), (xs, 1), (nx - 1 - xs, 0)]
    cells += [(int(x), int(y)) for x, y in zip(rng.integers(0, nx, 400), rng.integers(0, ny, 400))]
    for x, y in cells:
        fo, go, m, _ = ref.cell_update(fprev, gprev, x, y)
        assert np.abs(go - gnew[:, y, x]).max() <= 1e-5, (x, y)
        assert np.abs(fo - fnew[:, y, x]).max() <= 1e-5, (x, y)
        for k, name in enumerate(FIELDS):
            assert abs(m[k] - F[name][y, x]) <= 1e-5, (x, y, name)


@pytest.mark.parametrize("calls,n", [(1, 5), (3, 100)])
def test_full_size_one_buffer_sweeps_vs_oracle_fp32(orc, stream, calls, n):
    """2048 x 1024 production cavity, FP32, in the benchmark's streaming and
    launch shape (diagnostics every 100th step): from the GPU's own populations
    after 100 steps, `calls` calls of n steps -- 5: push, local, push, local
    sweeps in one buffer, then a pull sweep into the other; three calls of
    100: the same 100-step piece ending in a diagnostic sweep, launched
    directly, then from its graph -- against the oracle's steps from the same
    populations, every population of every cell, and the fields."""
    nx, ny, p = workloads.cavity_2048x1024()
    lat = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    lbm.lbm_set_streaming(lat.h, lbm.LBM_STREAM_ONE_BUFFER)  # the FP32 default, stated
    lbm.lbm_set_diag_every(lat.h, 100)
    lat.step(100)
    f0, g0, s0 = lat.populations()
    ref = orc.Oracle(nx, ny, threads=8, **p)
    ref.set_populations(f0, g0, s0)
    del f0, g0
    for _ in range(calls):
        lat.step(n)
    if calls > 2:
        assert lbm.lbm_get_launch_stats(lat.h)["sweeps_replayed"] > 0
    ref.step(calls * n)
    f1, g1, s1 = lat.populations()
    fo, go = ref.populations()
    assert s1 == s0 + calls * n
    assert np.abs(g1 - go).max() <= 1e-5
    assert np.abs(f1 - fo).max() <= 1e-5
    del f1, g1, fo, go
    F, Fo = lat.fields(), ref.fields()
    for name in ("T", "fl", "ux", "uy"):
        assert np.abs(F[name] - Fo[name]).max() <= 1e-5, name


def test_fp32_mass_conserved_over_a_long_run(stream):
    """The closed cavity conserves mass (Eq. 2's flow analogue: the collision
    keeps sum f_i, bounce-back walls return what leaves).  In FP32 the rounded
    D2Q9 weights sum to 1 + 7.45e-9; had each collision carried that excess,
    the 64 x 32 cavity's mean density would have grown by ~4e-4 over 5e4
    steps.  It must stay within 3e-5 of 1."""
    nx, ny, p = workloads.cavity_64x32()
    lat = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    assert abs(lat.fields()["rho"].mean() - 1.0) <= 1e-7
    lat.step(50000)
    assert lat.diagnostics()["nan_flag"] == 0
    assert abs(lat.fields()["rho"].mean() - 1.0) <= 3e-5


def test_full_size_budget_and_bounds_fp32(stream):
    nx, ny, p = workloads.cavity_2048x1024()
    lat = lbm.Lattice(nx, ny, p, precision="fp32", stream=stream)
    d0 = lat.diagnostics()
    lat.step(2000)
    d = lat.diagnostics()
    assert d["nan_flag"] == 0 and d["Q_cum"] > 0
    assert 0.0 <= d["melt_fraction"] <= 1.0 and d["melt_fraction"] > d0["melt_fraction"]
    assert abs(d["H_total"] - d0["H_total"] - d["Q_cum"]) <= 1e-3 * d["Q_cum"]
    assert d["max_u"] < 0.3


# ------------------------------------------------------------ launch paths
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_graph_replay_matches_direct_launches(stream, prec):
    """lbm_step replays captured chunk graphs; the state, the heated-wall
    totals and the diagnostics must be bitwise those of one launch per sweep,
    including diagnostic sweeps inside the chunks and odd chunk lengths."""
    nx, ny, p = 300, 77, workloads.params(Ra=1e5, strip_center=0.4)
    out = []
    for chunk, diag_every in ((0, 0), (128, 0), (0, 50), (32, 50), (7, 3)):
        lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
        lbm.lbm_set_launch(lat.h, 1, 4, chunk)
        lbm.lbm_set_diag_every(lat.h, diag_every)
        lat.step(413)
        lat.step(290)
        f, g, step = lat.populations()
        out.append((f, g, step, lat.diagnostics()))
    f0, g0, s0, d0 = out[0]
    for f, g, s, d in out[1:]:
        assert s == s0 == 703
        assert np.array_equal(f, f0) and np.array_equal(g, g0)
        assert d == d0


@pytest.mark.parametrize("problem", ["cavity", "stefan"])
@pytest.mark.parametrize("ny", [3, 4, 5, 7, 10])
def test_row_band_order_both_directions(orc, stream, problem, ny):
    """Successive sweeps visit the row bands in opposite directions, the two
    wall bands first; every band count (1 to 10 bands, a ragged last band)
    and both directions (odd and even steps) match the oracle."""
    nx = 130
    if problem == "cavity":
        p = workloads.params(Ra=1e5, strip_center=0.45, strip_width=0.3)
    else:
        p = workloads.stefan_1024x4(Ste=1.0, nx=nx)[2]
    ref = orc.Oracle(nx, ny, **p)
    ref.step(9)
    want = ref.fields()
    for rows in (1, 2, 3, 4):
        lat = lbm.Lattice(nx, ny, p, precision="fp64", stream=stream)
        lbm.lbm_set_launch(lat.h, rows, 2, 0)
        lat.step(9)
        assert_fields_fp64(lat.fields(), want)
        assert lat.diagnostics()["Q_cum"] == pytest.approx(ref.diagnostics()["Q_cum"], rel=1e-12, abs=1e-15)
        lat.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16sr"])
def test_launch_shape_does_not_change_populations(stream, prec):
    nx, ny, p = 260, 45, workloads.params(Ra=1e5)
    ref = None
    for rows, pf in ((1, 0), (1, 4), (3, 2), (8, 64)):
        lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
        lbm.lbm_set_launch(lat.h, rows, pf, 16)
        lat.step(120)
        f, g, _ = lat.populations()
        if ref is None:
            ref = (f, g)
        else:
            assert np.array_equal(f, ref[0]) and np.array_equal(g, ref[1])


# ------------------------------------------------------------ 16-bit storage
def _w():
    return np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _bf16(x32):
    """Round float32 values to bfloat16 (nearest, ties to even), back as float32."""
    b = np.ascontiguousarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


# FP16 storage scales g by 2^6 and f - w by 2^10 (exact powers of two)
F16_SCALE = {"g": 64.0, "f": 1024.0}


def _encode(f, g, prec):
    """What the 16-bit storage holds, decoded: f_i as w_i + q(f_i - w_i), g_i as
    q(g_i), with the FP32 arithmetic the device uses."""
    if prec == "fp16":
        def qs(a, sc):
            return ((a * np.float32(sc)).astype(np.float16).astype(np.float32) / np.float32(sc))
        qf, qg = (lambda a: qs(a, F16_SCALE["f"])), (lambda a: qs(a, F16_SCALE["g"]))
    else:
        qf = qg = _bf16
    w = _w().astype(np.float32)[:, None, None]
    f32, g32 = f.astype(np.float32), g.astype(np.float32)
    return ((qf(f32 - w) + w).astype(np.float64), qg(g32).astype(np.float64))


def _ulp16(a, prec, kind="g"):
    """One unit in the last place of the (scaled) 16-bit format at |a|."""
    mant = 10 if prec == "fp16" else 7
    tiny = 2.0 ** -14 / F16_SCALE[kind] if prec == "fp16" else 2.0 ** -126
    return 2.0 ** (np.floor(np.log2(np.maximum(np.abs(a), tiny))) - mant)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_16bit_single_step_matches_oracle_to_one_ulp(orc, stream, prec):
    """From a state the 16-bit storage holds exactly, one step on the GPU (FP32
    arithmetic, result rounded to 16 bits) equals the FP64 oracle's step rounded
    the same way, to one unit in the last place of the 16-bit format."""
    nx, ny, p = 70, 33, workloads.params(Ra=1e6, strip_center=0.4, strip_width=0.35)
    f, g = workloads.random_populations(nx, ny, seed=12)
    f, g = _encode(f, g, prec)
    ref = orc.Oracle(nx, ny, **p)
    ref.set_populations(f, g, step=3)
    ref.step(1)
    lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    lat.set_populations(f, g, step=3)
    f_in, g_in, _ = lat.populations()
    assert np.array_equal(f_in, f) and np.array_equal(g_in, g)  # lossless round trip
    lat.step(1)
    fo, go, _ = lat.populations()
    fr, gr = ref.populations()
    w = _w()[:, None, None]
    assert np.all(np.abs(go - gr) <= _ulp16(gr, prec, "g") + 1e-6 * np.abs(gr) + 1e-30)
    assert np.all(np.abs((fo - w) - (fr - w)) <= _ulp16(fr - w, prec, "f") + 1e-6 * np.abs(fr) + 1e-30)


@pytest.mark.parametrize("prec,melt_tol,nu_tol,budget_tol",
                         [("fp16sr", 2e-4, 5e-3, 5e-3), ("bf16sr", 1e-3, 3e-2, 3e-2)])
def test_16bit_stochastic_rounding_tracks_fp64(stream, prec, melt_tol, nu_tol, budget_tol):
    """64 x 32 cavity, 2000 steps, history every 100 steps: with stochastic
    rounding the 16-bit runs follow the FP64 run -- melt fraction within
    melt_tol at every sample (target 1e-3), mean Nu within nu_tol, and the
    enthalpy budget closes to budget_tol (the rounding is unbiased but its
    noise, ~ulp/2 per stored value and step, random-walks in sum H)."""
    nx, ny, p = workloads.cavity_64x32()
    hist = {}
    for pr in ("fp64", prec):
        lat = lbm.Lattice(nx, ny, p, precision=pr, stream=stream)
        h0 = lat.diagnostics()["H_total"]
        rows = []
        for _ in range(20):
            lat.step(100)
            d = lat.diagnostics()
            rows.append((d["melt_fraction"], d["Nu"], d["H_total"] - h0 - d["Q_cum"], d["Q_cum"]))
        hist[pr] = np.array(rows)
    a, r = hist[prec], hist["fp64"]
    assert np.abs(a[:, 0] - r[:, 0]).max() <= melt_tol
    assert abs(a[:, 1].mean() - r[:, 1].mean()) <= nu_tol * r[:, 1].mean()
    assert np.abs(a[:, 2]).max() <= budget_tol * a[-1, 3]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_16bit_round_to_nearest_stagnates(stream, prec):
    """Negative control: rounding to nearest loses the per-step enthalpy
    increments below half an ulp, so melting lags the FP64 run by more than
    the 1e-3 target and the enthalpy budget does not close."""
    nx, ny, p = workloads.cavity_64x32()
    out = {}
    for pr in ("fp64", prec):
        lat = lbm.Lattice(nx, ny, p, precision=pr, stream=stream)
        h0 = lat.diagnostics()["H_total"]
        lat.step(2000)
        d = lat.diagnostics()
        out[pr] = (d["melt_fraction"], abs(d["H_total"] - h0 - d["Q_cum"]) / d["Q_cum"])
    assert out["fp64"][0] - out[prec][0] > 1e-3
    assert out[prec][1] > 1e-2


# ------------------------------------------------------------ extreme shapes
@pytest.mark.parametrize("prec", ["fp16sr", "bf16sr"])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_16bit_stochastic_rounding_keeps_non_finite_values(stream, prec, bad):
    """The paired stochastic-rounding conversion stores a NaN or an infinity as
    a non-finite value, so a diverging cell is still reported steps later."""
    nx, ny, p = workloads.cavity_64x32()
    lat = lbm.Lattice(nx, ny, p, precision=prec, stream=stream)
    lat.step(10)
    f, g, step = lat.populations()
    g[0, 12, 20] = bad
    lat.set_populations(f, g, step)
    lat.step(5)
    d = lat.diagnostics(raise_on_diverged=False)
    assert d["nan_flag"] == 1
    f, g, _ = lat.populations()
    assert not np.isfinite(g).all()


@pytest.mark.parametrize("nx,ny,steps", [(2, 65535, 3), (262144, 2, 3), (129, 65535, 2)])
def test_extreme_shapes_match_oracle(orc, stream, nx, ny, steps):
    """The tallest lattice the launch allows (65,535 rows: 65,535 blocks in y),
    a 2^18-cell-wide strip of 2,048 tiles, and a ragged two-tile width at full
    height, against the oracle (FP64)."""
    p = workloads.params(Ra=1e5, init_amp=0.1)
    ref, lat = run_pair(orc, nx, ny, p, steps, "fp64", stream, threads=8)
    assert_fields_fp64(lat.fields(), ref.fields())
    d, dr = lat.diagnostics(), ref.diagnostics()
    assert d["Q_cum"] == pytest.approx(dr["Q_cum"], rel=1e-12, abs=1e-15)
    assert d["melt_fraction"] == pytest.approx(dr["melt_fraction"], rel=1e-12, abs=1e-15)
