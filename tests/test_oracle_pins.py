"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each checks a property that a
plausible slip (a dropped term, a wrong sign or index, a transposed operand)
would break -- moment identities (Eq. 4), the moment-space form of the block
collision (Eq. 2, "can be written as an MRT form"), the SRT/BGK reduction,
Guo's forcing, conservation in a closed box, the exact enthalpy budget, the
Neumann solution (Eqs. 7-8) for the front, the profile and the heated-wall
flux (hence Q and Nu), the one-cell interface of Eq. 6, mirror symmetry, the
diffusivity of Eq. 5, the viscosity of the flow operator (a decaying shear
wave at Pr != 1), the solid treatment u = f_l u*, hydrostatic balance, the
distribution of the seeded initial perturbation, and published generator
outputs.  The last test plants such slips in copies of the oracle and checks
that the matching pins fail on them.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CS2 = 1.0 / 3.0


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ lattice
def test_d2q9_table(orc):
    cx, cy, w, opp = orc.lattice()
    c = np.stack([cx, cy], 1).astype(float)
    # weights from Sec. 2 (golden)
    table = {int(r[0]): int(r[1]) / int(r[2]) for r in read_golden("d2q9_weights.txt")}
    for i in range(9):
        assert w[i] == pytest.approx(table[int(cx[i] ** 2 + cy[i] ** 2)], rel=0, abs=1e-17)
    assert sorted(map(tuple, c.astype(int))) == sorted(
        [(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)])
    # opposites
    for i in range(9):
        assert cx[opp[i]] == -cx[i] and cy[opp[i]] == -cy[i]
    # isotropy up to fourth order with c_s^2 = 1/3
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, CS2 * np.eye(2), atol=1e-16)
    M3 = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(M3, 0.0, atol=1e-16)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(2)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(M4, iso, atol=1e-16)


def test_splitmix64_published_outputs(orc):
    G = 0x9E3779B97F4A7C15
    for seed, k, out in read_golden("splitmix64.txt"):
        v = (int(seed) + (int(k) - 1) * G) % 2 ** 64
        assert orc.splitmix64(v) == int(out)


# ------------------------------------------------------------ H -> (T, f_l)
def test_inversion_reconstructs_total_enthalpy(orc):
    """Eq. 1 defines H = C_p T + f_l L; the inversion must return the (T, f_l)
    of that definition: solid below H_s, liquid above H_s + L, T = T_m between."""
    rng = np.random.default_rng(0)
    for Lh in (1.0, 8.0, 100.0):
        for H in np.concatenate([rng.uniform(-2, Lh + 2, 400), [0.0, Lh, -1e-300, Lh * (1 + 1e-16)]]):
            T, fl = orc.invert(H, Lh)
            assert 0.0 <= fl <= 1.0
            assert T + fl * Lh == pytest.approx(H, rel=1e-15, abs=1e-15)
            if 0.0 < fl < 1.0:
                assert T == 0.0
            if T < 0.0:
                assert fl == 0.0
            if T > 0.0:
                assert fl == 1.0
    # continuity at both kinks
    for Lh in (1.0, 8.0):
        for Hk in (0.0, Lh):
            a = orc.invert(Hk - 1e-12, Lh)
            b = orc.invert(Hk + 1e-12, Lh)
            assert abs(a[0] - b[0]) < 1e-11 and abs(a[1] - b[1]) < 1e-11


# ---------------------------------------------------------------- Eq. 4
def test_geq_moments(orc):
    cx, cy, w, _ = orc.lattice()
    c = np.stack([cx, cy], 1).astype(float)
    rng = np.random.default_rng(1)
    for _ in range(50):
        H, T = rng.uniform(-1, 3), rng.uniform(-1, 2)
        u = rng.uniform(-0.1, 0.1, 2)
        g = orc.geq(H, T, u[0], u[1])
        assert g.sum() == pytest.approx(H, abs=1e-14)
        assert np.allclose(c.T @ g, T * u, atol=1e-15)
        assert np.allclose(np.einsum("ia,ib,i->ab", c, c, g), T * CS2 * np.eye(2), atol=1e-15)


def test_feq_moments(orc):
    cx, cy, w, _ = orc.lattice()
    c = np.stack([cx, cy], 1).astype(float)
    rng = np.random.default_rng(2)
    for _ in range(50):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.1, 0.1, 2)
        f = orc.feq(rho, u[0], u[1])
        assert f.sum() == pytest.approx(rho, abs=1e-14)
        assert np.allclose(c.T @ f, rho * u, atol=1e-15)
        assert np.allclose(np.einsum("ia,ib,i->ab", c, c, f),
                           rho * CS2 * np.eye(2) + rho * np.outer(u, u), atol=1e-15)


# --------------------------------------------------------- Eq. 2 (MRT form)
def _projectors(orc):
    """Orthogonal projectors (inner product sum a_i b_i / w_i) onto the
    0th-, 1st-, 2nd-order and ghost subspaces of D2Q9 population space."""
    cx, cy, w, _ = orc.lattice()
    cx = cx.astype(float)
    cy = cy.astype(float)
    Winv = np.diag(1.0 / w)

    def proj(cols):
        B = np.stack(cols, 1)
        return B @ np.linalg.solve(B.T @ Winv @ B, B.T @ Winv)

    P0 = proj([w])
    P1 = proj([w * cx, w * cy])
    P2 = proj([w * (cx * cx - CS2), w * cx * cy, w * (cy * cy - CS2)])
    Pg = np.eye(9) - P0 - P1 - P2
    return P0, P1, P2, Pg


def test_g_collision_is_block_relaxation(orc):
    """The non-equilibrium part's first moment relaxes with k1, its second
    moment with k2 and everything else with k0 (Eq. 2 as an MRT operator)."""
    P0, P1, P2, Pg = _projectors(orc)
    rng = np.random.default_rng(3)
    for _ in range(40):
        g = rng.uniform(-0.2, 0.6, 9)
        H = g.sum()
        T = rng.uniform(-0.5, 1.5)
        u = rng.uniform(-0.05, 0.05, 2)
        k0, k1, k2 = rng.uniform(0.1, 1.9, 3)
        geq = orc.geq(H, T, u[0], u[1])
        n = g - geq
        n_post = orc.g_collide(g, H, T, u[0], u[1], k0, k1, k2) - geq
        expect = (1 - k0) * (P0 @ n) + (1 - k1) * (P1 @ n) + (1 - k2) * (P2 @ n) + (1 - k0) * (Pg @ n)
        assert np.allclose(n_post, expect, atol=1e-14, rtol=0)
        assert orc.g_collide(g, H, T, u[0], u[1], k0, k1, k2).sum() == pytest.approx(H, abs=1e-14)


def test_g_collision_reduces_to_srt(orc):
    """k0 = k1 = k2 = k gives the single-relaxation-time (BGK) update."""
    rng = np.random.default_rng(4)
    for _ in range(40):
        g = rng.uniform(-0.2, 0.6, 9)
        H, T = g.sum(), rng.uniform(-0.5, 1.5)
        u = rng.uniform(-0.05, 0.05, 2)
        k = rng.uniform(0.1, 1.9)
        geq = orc.geq(H, T, u[0], u[1])
        bgk = g - k * (g - geq)
        assert np.allclose(orc.g_collide(g, H, T, u[0], u[1], k, k, k), bgk, atol=1e-15, rtol=0)


def _guo_source(orc, u, F, tau):
    """Guo, Zheng & Shi (Phys. Rev. E 65, 046308, 2002) forcing term with
    lattice units c_s^2 = 1/3: (1 - 1/(2 tau)) w_i [3(c_i - u).F + 9(c_i.u)(c_i.F)]."""
    cx, cy, w, _ = orc.lattice()
    S = np.empty(9)
    for i in range(9):
        ci = np.array([cx[i], cy[i]], float)
        S[i] = (1 - 0.5 / tau) * w[i] * (3 * (ci - u) @ F + 9 * (ci @ u) * (ci @ F))
    return S


def test_f_collision_reduces_to_bgk_guo(orc):
    rng = np.random.default_rng(5)
    for _ in range(40):
        f = rng.uniform(0.0, 0.3, 9)
        rho = f.sum()
        u = rng.uniform(-0.05, 0.05, 2)
        F = rng.uniform(-1e-3, 1e-3, 2)
        k = rng.uniform(0.2, 1.9)
        feq = orc.feq(rho, u[0], u[1])
        expect = f - k * (f - feq) + _guo_source(orc, u, F, 1.0 / k)
        got = orc.f_collide(f, rho, u[0], u[1], F[0], F[1], k, k, k)
        assert np.allclose(got, expect, atol=1e-15, rtol=0)


def test_f_collision_moments_and_source(orc):
    """Block flow collision: mass kept; first moment of the post-collision
    populations is j + F when u = (j + F/2)/rho; the source's moments are
    0, (1 - k1f/2) F and (1 - k2f/2)(uF + Fu), with no ghost part."""
    cx, cy, w, _ = orc.lattice()
    c = np.stack([cx, cy], 1).astype(float)
    P0, P1, P2, Pg = _projectors(orc)
    rng = np.random.default_rng(6)
    for _ in range(40):
        f = rng.uniform(0.0, 0.3, 9)
        rho = f.sum()
        j = c.T @ f
        F = rng.uniform(-1e-3, 1e-3, 2)
        u = (j + 0.5 * F) / rho
        k0f, k1f, k2f = rng.uniform(0.2, 1.9, 3)
        post = orc.f_collide(f, rho, u[0], u[1], F[0], F[1], k0f, k1f, k2f)
        assert post.sum() == pytest.approx(rho, abs=1e-14)
        assert np.allclose(c.T @ post, j + F, atol=1e-14)
        S = post - orc.f_collide(f, rho, u[0], u[1], 0.0, 0.0, k0f, k1f, k2f)
        assert abs(S.sum()) < 1e-15
        assert np.allclose(c.T @ S, (1 - 0.5 * k1f) * F, atol=1e-15)
        uF = np.outer(u, F) + np.outer(F, u)
        assert np.allclose(np.einsum("ia,ib,i->ab", c, c, S), (1 - 0.5 * k2f) * uF, atol=1e-15)
        assert np.allclose(Pg @ S, 0.0, atol=1e-15)
        # the non-source part relaxes blockwise like Eq. 2
        feq = orc.feq(rho, u[0], u[1])
        n = f - feq
        n_post = post - S - feq
        expect = (1 - k0f) * (P0 @ n + Pg @ n) + (1 - k1f) * (P1 @ n) + (1 - k2f) * (P2 @ n)
        assert np.allclose(n_post, expect, atol=1e-14)


# ------------------------------------------------------------ Eqs. 5-8
def test_eq5_k1_round_trip_and_paper_k1_list(orc):
    params = read_golden("paper_parameters.txt")
    k1s = [float(v) for k, v in params if k == "stefan_k1"]
    for k1 in k1s:
        alpha = CS2 * (1.0 / k1 - 0.5)
        if k1 >= 2.0:
            # Eq. 5 leaves no positive diffusivity at k1 = 2, so that entry of the
            # paper's list cannot be run; a negative diffusivity is rejected.
            assert alpha <= 0.0
            with pytest.raises(ValueError):
                orc.derive(64, 4, problem=orc.STEFAN, flow_on=0, alpha_override=-1e-3, k2=-1.0)
            continue
        d = orc.derive(64, 4, problem=orc.STEFAN, flow_on=0, alpha_override=alpha, k2=-1.0)
        assert d.k1 == pytest.approx(k1, rel=1e-14)
        assert d.k1 + d.k2 == pytest.approx(2.0, rel=1e-15)   # Eq. 6 on request


def test_cavity_parameter_mapping(orc):
    """nu, alpha, g beta reproduce Ra and Pr; the cavity strip sits at C +- D/2."""
    for nx, ny, Ra, Pr in [(64, 32, 1e4, 1.0), (2048, 1024, 1e8, 1.0), (512, 512, 1e8, 6.2)]:
        d = orc.derive(nx, ny, Ra=Ra, Pr=Pr, Ma=0.1)
        assert d.gbeta * 1.0 * ny ** 3 / (d.nu * d.alpha) == pytest.approx(Ra, rel=1e-12)
        assert d.nu / d.alpha == pytest.approx(Pr, rel=1e-14)
        assert math.sqrt(d.gbeta * ny) == pytest.approx(0.1 / math.sqrt(3), rel=1e-14)
        assert d.a == pytest.approx(nx * 0.375) and d.b == pytest.approx(nx * 0.625)
    d = orc.derive(64, 32, Ra=1e4, Pr=1.0, Ma=0.1)
    assert d.k1 == pytest.approx(1.80042, abs=1e-5)        # k1 of the 64x32 case


def test_stefan_root_eq8(orc):
    from scipy.optimize import brentq
    from scipy.special import erf
    for Ste in (0.01, 0.1, 0.125, 1.0, 3.0):
        lam = orc.stefan_lambda(Ste)
        ref = brentq(lambda l: Ste / (math.exp(l * l) * erf(l)) - l * math.sqrt(math.pi), 1e-9, 5.0,
                     xtol=1e-15)
        assert lam == pytest.approx(ref, rel=1e-12)
    # small-Ste limit: lambda^2 -> Ste/2
    assert orc.stefan_lambda(1e-6) ** 2 == pytest.approx(0.5e-6, rel=1e-5)


def test_neumann_solution_eq7(orc):
    """Eq. 7 satisfies the heat equation in the melt, T = T_h at the wall,
    T = T_m at the front, and the Stefan condition L dX/dt = -alpha dT/dx."""
    for Ste in (0.1, 1.0):
        lam = orc.stefan_lambda(Ste)
        alpha, Lh, t = 1.0 / 6.0, 1.0 / Ste, 2000.0
        X = 2 * lam * math.sqrt(alpha * t)
        T = lambda x, tt: orc.neumann_T(x, tt, alpha, lam)
        assert T(0.0, t) == pytest.approx(1.0, abs=1e-15)
        assert T(X * (1 - 1e-12), t) == pytest.approx(0.0, abs=1e-9)
        assert T(X * 1.5, t) == 0.0
        h = 1e-2
        for x in (0.2 * X, 0.5 * X, 0.8 * X):
            dTdt = (T(x, t + h) - T(x, t - h)) / (2 * h)
            d2Tdx2 = (T(x + h, t) - 2 * T(x, t) + T(x - h, t)) / h ** 2
            assert dTdt == pytest.approx(alpha * d2Tdx2, rel=1e-4, abs=1e-10)
        dXdt = lam * math.sqrt(alpha / t)
        dTdx = (T(X - 1e-4, t) - T(X - 2e-4, t)) / 1e-4
        assert Lh * dXdt == pytest.approx(-alpha * dTdx, rel=1e-3)


# ---------------------------------------------------------- whole lattice
def _liquid_state(orc, nx, ny, H0):
    """Post-collision populations of a resting state with enthalpy field H0."""
    _, _, w, _ = orc.lattice()
    Lh = 1.0
    g = np.empty((9, ny, nx))
    f = np.empty((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            T, _fl = orc.invert(H0[y, x], Lh)
            g[:, y, x] = orc.geq(H0[y, x], T, 0.0, 0.0)
            f[:, y, x] = w
    return f, g


def test_closed_box_conserves_mass_and_enthalpy(orc):
    """Adiabatic no-slip walls (no heated strip): sum rho and sum H are
    invariants of the whole step, with melting and convection going on."""
    nx, ny = 48, 24
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    H0 = np.where(Y < ny // 2, 1.0 + 0.8 * np.sin(2 * np.pi * X / nx) ** 2, -0.3)
    o = orc.Oracle(nx, ny, Ra=1e5, Pr=1.0, Ste=1.0, Ma=0.1, strip_width=0.0)
    f, g = _liquid_state(orc, nx, ny, H0)
    o.set_populations(f, g)
    o.step(1)
    F0 = o.fields()
    m0, h0 = F0["rho"].sum(), F0["H"].sum()
    o.step(1999)
    F = o.fields()
    # Exact in exact arithmetic.  In FP64 the near-uniform rounding of each
    # cell's sums repeats step after step, so the drift grows linearly, about a
    # quarter ulp per cell per step: the gate allows two ulps per step.  A lost
    # or doubled wall population would show up as O(1e-3) per step.
    tol = 1999 * 2 * np.finfo(float).eps
    assert abs(F["rho"].sum() - m0) <= tol * abs(m0)
    assert abs(F["H"].sum() - h0) <= tol * np.abs(F0["H"]).sum()
    assert np.abs(F["uy"]).max() > 1e-5          # convection did happen
    fl0 = (H0 > 0).mean()
    assert abs(F["fl"].mean() - fl0) > 1e-3      # so did phase change


def test_heated_strip_energy_budget(orc):
    """sum H(n) - sum H(0) equals the summed heated-wall inflow (to rounding)."""
    o = orc.Oracle(64, 32)
    h0 = o.diagnostics()["H_total"]
    o.step(2000)
    d = o.diagnostics()
    assert d["Q_cum"] > 100.0
    assert abs(d["H_total"] - h0 - d["Q_cum"]) <= 1e-12 * d["Q_cum"]
    assert d["nan_flag"] == 0.0
    assert 0.0 < d["melt_fraction"] < 1.0 and d["Nu"] > 0.0
    assert d["front_x"] == pytest.approx(d["melt_fraction"] * 64, rel=1e-13)


def test_step_by_step_budget_and_monotone_melt(orc):
    o = orc.Oracle(64, 32)
    prev = o.diagnostics()
    for _ in range(300):
        o.step(1)
        d = o.diagnostics()
        assert abs(d["H_total"] - prev["H_total"] - d["Q_strip"]) <= 1e-12 * max(1.0, abs(d["H_total"]))
        assert d["Q_strip"] > 0.0
        prev = d


def test_mirror_symmetry_centred_strip(orc):
    nx, ny = 40, 20
    o = orc.Oracle(nx, ny, Ra=1e5, init_amp=0.0)
    o.step(600)
    F = o.fields()
    assert F["fl"].max() > 0.0
    # Mirror images round differently (sums run in the same lattice order), so
    # the bound is 1e-12 of the field's scale or 1e-14 absolute for the
    # velocities, whose O(1e-16) rounding comes from O(0.1) populations.
    for k in ("H", "T", "fl", "uy", "rho"):
        a = F[k]
        tol = max(1e-12 * np.abs(a).max(), 1e-14)
        assert np.abs(a - a[:, ::-1]).max() <= tol, k
    assert np.abs(F["ux"] + F["ux"][:, ::-1]).max() <= max(1e-12 * np.abs(F["ux"]).max(), 1e-14)


def test_thread_count_does_not_change_results(orc):
    a = orc.Oracle(33, 17, threads=1, Ra=1e5)
    b = orc.Oracle(33, 17, threads=4, Ra=1e5)
    a.step(50)
    b.step(50)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert a.diagnostics() == b.diagnostics()


def test_diffusion_rate_matches_eq5(orc):
    """A cosine mode of T in a liquid at rest decays as exp(-alpha k^2 t) with
    alpha = c_s^2 (1/k1 - 1/2) (Eq. 5), for several k1 and any k2, k0.
    Bounce-back rows next to the adiabatic top and bottom walls diffuse the
    tangential mode slightly differently, so the domain is tall (128 rows) and
    the gate 1 %."""
    nx, ny = 64, 128
    _, _, w, _ = orc.lattice()
    x = np.arange(nx) + 0.5
    kw = math.pi / nx
    for k1, k0, k2 in [(0.5, 1.0, 1.0), (1.0, 0.7, 1.0), (1.5, 1.0, 0.5)]:
        alpha = CS2 * (1.0 / k1 - 0.5)
        o = orc.Oracle(nx, ny, threads=4, Ste=1.0, flow_on=0, alpha_override=alpha, k0=k0,
                       k2=k2, strip_width=0.0, init_amp=0.0)
        T0 = 1.0 + 0.1 * np.cos(kw * x)
        g = np.zeros((9, ny, nx))
        for xx in range(nx):
            g[:, :, xx] = orc.geq(T0[xx] + 1.0, T0[xx], 0.0, 0.0)[:, None]
        f = np.broadcast_to(w[:, None, None], (9, ny, nx)).copy()
        o.set_populations(f, g)
        n = int(round(0.3 / (alpha * kw * kw)))
        o.step(n)
        T = o.fields()["T"].mean(axis=0)
        amp = 2.0 / nx * np.sum((T - T.mean()) * np.cos(kw * x))
        assert amp == pytest.approx(0.1 * math.exp(-alpha * kw * kw * n), rel=1e-2)


def test_hydrostatic_balance_sets_force_sign(orc):
    """Uniformly warm liquid at rest: the buoyancy force F = g beta (T - T_m) y
    must be balanced by a density gradient d rho/dy = F_y / c_s^2, and the
    fluid must come to rest."""
    nx, ny = 12, 24
    o = orc.Oracle(nx, ny, Ra=4096.0, Pr=1.0, Ste=1.0, alpha_override=0.1, strip_width=0.0,
                   init_amp=0.0)
    d = o.derived()
    H0 = np.full((ny, nx), 1.5)
    f, g = _liquid_state(orc, nx, ny, H0)
    o.set_populations(f, g)
    o.step(4000)
    F = o.fields()
    Fy = d["gbeta"] * 0.5
    drho = np.diff(F["rho"][:, nx // 2])[2:-2].mean()
    assert Fy > 1e-3
    assert drho == pytest.approx(Fy / CS2, rel=1e-3)
    assert np.abs(F["uy"]).max() < 1e-4 * Fy * ny


def test_hot_fluid_rises(orc):
    nx, ny = 32, 32
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    H0 = 1.0 + 0.5 * np.exp(-((X - 16) ** 2 + (Y - 10) ** 2) / 20.0)
    o = orc.Oracle(nx, ny, Ra=1e5, strip_width=0.0, init_amp=0.0)
    f, g = _liquid_state(orc, nx, ny, H0)
    o.set_populations(f, g)
    o.step(200)
    F = o.fields()
    blob = F["uy"][8:13, 13:19]
    assert blob.min() > 0.0                      # the warm blob moves up
    assert blob.mean() > 0.5 * F["uy"].max()


# ---------------------------------------------------- Stefan (Sec. 3.1)
def _stefan(orc, nx, Ste, k1, k2, k0=1.0):
    alpha = CS2 * (1.0 / k1 - 0.5)
    o = orc.Oracle(nx, 4, problem=orc.STEFAN, Ste=Ste, flow_on=0, alpha_override=alpha,
                   k0=k0, k2=k2, init_amp=0.0)
    return o, alpha


@pytest.mark.parametrize("Ste", [0.1, 1.0])
def test_stefan_front_and_profile_match_neumann(orc, Ste):
    nx, n_end = 256, 20000
    o, alpha = _stefan(orc, nx, Ste, k1=1.0, k2=-1.0)
    lam = orc.stefan_lambda(Ste)
    done = 0
    for n in (1000, 5000, 20000):
        o.step(n - done)
        done = n
        X = 2 * lam * math.sqrt(alpha * n)
        xf = o.diagnostics()["front_x"]
        assert abs(xf - X) <= 1.0, (n, xf, X)
    assert xf == pytest.approx(X, rel=0.02 if Ste < 0.5 else 0.01)
    T = o.fields()["T"][0]
    x = np.arange(nx) + 0.5
    liquid = x < X - 1.0
    Tn = np.array([orc.neumann_T(xx, n_end, alpha, lam) for xx in x[liquid]])
    assert np.abs(T[liquid] - Tn).max() <= 1e-2


@pytest.mark.parametrize("k1,k0", [(1.5, 1.0), (0.5, 1.0), (1.5, 0.6), (0.8, 1.3)])
def test_one_cell_interface_with_k1_plus_k2_eq_2(orc, k1, k0):
    """Eq. 6 (k1 + k2 = 2): the solid ahead of the front stays exactly at T_m
    (H = H_s) and every row has at most one mushy cell, at every step."""
    # "Exactly" means to rounding: the leak into the solid is an FP64 rounding
    # residue (~1e-17), so a cell counts as mushy above 1e-12 liquid fraction.
    o, _ = _stefan(orc, 128, Ste=0.1, k1=k1, k2=2.0 - k1, k0=k0)
    eps = 1e-12
    for _ in range(1500):
        o.step(1)
        F = o.fields()
        fl, H = F["fl"], F["H"]
        mushy = (fl > eps) & (fl < 1 - eps)
        assert mushy.sum(axis=1).max() <= 1
        for row in range(4):
            melted = np.nonzero(fl[row] > eps)[0]
            edge = melted.max() if melted.size else -1
            assert np.abs(H[row, edge + 1:]).max(initial=0.0) <= 1e-14
    assert o.diagnostics()["front_x"] > 3.0


@pytest.mark.parametrize("k", [0.5, 1.5])
def test_srt_leaks_into_solid_when_k_not_1(orc, k):
    """Negative control (Sec. 3.1, SRT): with k0 = k1 = k2 = k != 1 the solid
    ahead of the front is disturbed.  The leak has the sign of 1 - k: for
    k < 1 enthalpy runs ahead and the interface widens past one cell; for
    k > 1 the solid ahead is pulled below T_m."""
    o, _ = _stefan(orc, 128, Ste=0.1, k1=k, k2=k, k0=k)
    o.step(1500)
    F = o.fields()
    fl, H = F["fl"], F["H"]
    if k < 1:
        mushy = (fl > 1e-6) & (fl < 1 - 1e-6)
        assert mushy.sum(axis=1).min() >= 2
    else:
        assert H.min() < -1e-6


# ------------------------------------------- flow viscosity (reading A2)
def check_shear_wave_decays_at_nu(orc):
    """A shear wave u_y = U sin(2 pi (x + 1/2)/nx) in liquid at rest between the
    no-slip side walls (an eigenmode of the viscous term that vanishes on both
    half-way walls and carries no net flux) decays as exp(-nu k^2 t): the flow
    operator's second-moment rate k2f = 1/(nu/c_s^2 + 1/2) sets the kinematic
    viscosity, as Eq. 5 does for the diffusivity.  Pr = 6.2, so nu = 6.2 alpha
    and a rate taken from alpha would decay six times slower.  No buoyancy
    (Ra = 0), no heated wall; the box is tall so that the top and bottom walls
    do not reach the measured middle rows in 300 steps."""
    nx, ny, Pr, nu, U = 32, 512, 6.2, 0.1, 1e-3
    o = orc.Oracle(nx, ny, threads=4, Ra=0.0, Pr=Pr, Ste=1.0, alpha_override=nu / Pr,
                   strip_width=0.0, init_amp=0.0)
    x = np.arange(nx) + 0.5
    kw = 2.0 * math.pi / nx
    f = np.empty((9, ny, nx))
    g = np.empty((9, ny, nx))
    for xx in range(nx):
        uy = U * math.sin(kw * x[xx])
        f[:, :, xx] = orc.feq(1.0, 0.0, uy)[:, None]
        g[:, :, xx] = orc.geq(1.5, 0.5, 0.0, uy)[:, None]   # liquid: H > L = 1
    o.set_populations(f, g)
    n = 300
    o.step(n)
    F = o.fields()
    assert F["fl"].min() == 1.0
    mid = F["uy"][ny // 2 - 16: ny // 2 + 16].mean(axis=0)
    amp = 2.0 / nx * np.sum(mid * np.sin(kw * x))
    decay = math.exp(-nu * kw * kw * n)
    assert amp == pytest.approx(U * decay, rel=1e-2)
    # the largest speed is at least the wave's crest in the middle rows and a
    # little more where the flow turns at the top and bottom walls (about 7 %
    # here); |u_x| alone or |u|^2 would be far off
    crest = U * np.sin(kw * x).max() * decay
    assert 0.99 * crest <= o.diagnostics()["max_u"] <= 1.15 * crest


def test_shear_wave_decays_at_the_flow_viscosity(orc):
    check_shear_wave_decays_at_nu(orc)


# ------------------------------------------ solid treatment (reading A3)
def check_velocity_is_fl_times_ustar(orc):
    """u = f_l u*, u* = (j + F/2)/rho: zero in every solid cell, u* itself in
    every liquid cell, f_l u* in the mushy ones.  u* is formed here from the
    populations streamed by hand (interior cells, no wall) and the force
    F = g beta (T - T_m) y of the enthalpy streamed the same way, T taken from
    Eq. 1's definition of H."""
    nx, ny, Lh = 40, 24, 1.0
    o = orc.Oracle(nx, ny, Ra=1e6, Pr=0.7, Ste=1.0 / Lh, strip_width=0.0, init_amp=0.0)
    gbeta = o.derived()["gbeta"]
    cx, cy, _, _ = orc.lattice()
    rng = np.random.default_rng(5)
    H = rng.uniform(-0.6, 1.6, (ny, nx))    # solid, mushy and liquid cells
    f = np.empty((9, ny, nx))
    g = np.empty((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            u = rng.uniform(-0.05, 0.05, 2)
            T0 = min(H[y, x], 0.0) + max(H[y, x] - Lh, 0.0)
            g[:, y, x] = orc.geq(H[y, x], T0, 0.0, 0.0) + 0.01 * (rng.random(9) - 0.5)
            f[:, y, x] = orc.feq(1.0 + 0.02 * (rng.random() - 0.5), u[0], u[1]) \
                + 0.002 * (rng.random(9) - 0.5)
    o.set_populations(f, g)
    o.step(1)
    F = o.fields()
    fs = np.stack([f[i, 1 - cy[i]: ny - 1 - cy[i], 1 - cx[i]: nx - 1 - cx[i]] for i in range(9)])
    gs = np.stack([g[i, 1 - cy[i]: ny - 1 - cy[i], 1 - cx[i]: nx - 1 - cx[i]] for i in range(9)])
    rho = fs.sum(0)
    jx = np.tensordot(cx, fs, 1)
    jy = np.tensordot(cy, fs, 1)
    Hs = gs.sum(0)
    T = np.minimum(Hs, 0.0) + np.maximum(Hs - Lh, 0.0)
    fl = np.clip(Hs / Lh, 0.0, 1.0)
    usx, usy = jx / rho, (jy + 0.5 * gbeta * T) / rho
    ux, uy = F["ux"][1:-1, 1:-1], F["uy"][1:-1, 1:-1]
    solid, liquid = fl == 0.0, fl == 1.0
    mushy = ~solid & ~liquid
    assert solid.sum() > 100 and liquid.sum() > 100 and mushy.sum() > 100
    assert np.array_equal(F["fl"][1:-1, 1:-1], fl)
    assert np.all(ux[solid] == 0.0) and np.all(uy[solid] == 0.0)
    # the half-force shift is ~3e-5 here, so 1e-15 separates u* from j/rho
    assert np.abs(ux[liquid] - usx[liquid]).max() <= 1e-15
    assert np.abs(uy[liquid] - usy[liquid]).max() <= 1e-15
    assert np.abs(uy[mushy] - fl[mushy] * usy[mushy]).max() <= 1e-15
    assert np.abs(usy[liquid]).max() > 1e-2   # the liquid does move


def test_velocity_is_liquid_fraction_times_ustar(orc):
    check_velocity_is_fl_times_ustar(orc)


# --------------------------------- heated-wall inflow and Nu (reading A17)
def neumann_wall_flux(orc, Ste, alpha, n):
    """Heat flux per unit wall length at time n of the Neumann solution
    (Eqs. 7-8): -alpha dT/dx at x = 0 = alpha dT / (erf(lambda) sqrt(pi alpha t))."""
    lam = orc.stefan_lambda(Ste)
    return alpha * 1.0 / (math.erf(lam) * math.sqrt(math.pi * alpha * n))


WALL_FLUX_CASES = [  # (problem, Ste, checkpoints, tolerance)
    ("stefan", 1.0, (2000, 8000), 1e-2),
    ("stefan", 0.1, (8000,), 3e-2),
    ("cavity", 1.0, (2000, 6000), 1e-2),
]


def check_wall_flux_and_nu(orc, problem, Ste, steps, tol):
    """The inflow the oracle reports for a step, Q = sum over heated crossings
    of (2 w_i T_h - 2 g*_opp), is the heat entering through the T_h wall: for
    one-phase melting from a wall held at T_h it follows Neumann's flux times
    the wall length.  Stefan problem: left wall, ny cells long, Nu = Q nx /
    (alpha dT ny).  Cavity with its whole bottom wall heated and the flow off:
    the same solution along y, the wall nx cells long, Nu = Q ny / (alpha dT
    nx) (reference length = cavity height)."""
    alpha = 1.0 / 6.0
    if problem == "stefan":
        nx, ny = 256, 4
        o = orc.Oracle(nx, ny, problem=orc.STEFAN, Ste=Ste, flow_on=0, alpha_override=alpha,
                       k0=1.0, k2=-1.0, init_amp=0.0)
        wall, href = ny, nx
    else:
        # wide enough that the two side-wall columns, where half-way
        # bounce-back of the diagonal populations is not a mirror image,
        # shift the total by well under the gate
        nx, ny = 64, 160
        o = orc.Oracle(nx, ny, threads=4, problem=orc.CAVITY, Ste=Ste, flow_on=0,
                       alpha_override=alpha, strip_center=0.5, strip_width=1.0, k0=1.0,
                       k2=-1.0, init_amp=0.0)
        wall, href = nx, ny
    done = 0
    for n in steps:
        o.step(n - done)
        done = n
        d = o.diagnostics()
        q = neumann_wall_flux(orc, Ste, alpha, n)
        assert d["Q_strip"] == pytest.approx(q * wall, rel=tol), (problem, n)
        assert d["Nu"] == pytest.approx(q * wall * href / (alpha * wall), rel=tol), (problem, n)


@pytest.mark.parametrize("problem,Ste,steps,tol", WALL_FLUX_CASES)
def test_heated_wall_flux_and_nusselt_follow_neumann(orc, problem, Ste, steps, tol):
    check_wall_flux_and_nu(orc, problem, Ste, steps, tol)


# ------------------------------------------ initial state (reading A15)
def test_initial_perturbation_is_uniform_on_plus_minus_amp(orc):
    """H0 = amp (2r - 1) with r uniform on [0, 1): inside [-amp, amp], mean
    zero and uniform (Kolmogorov-Smirnov), no two neighbouring cells alike;
    cells with H0 > 0 are mushy at T_m, the others subcooled solid, f at rest."""
    from scipy import stats
    amp = 1e-3
    o = orc.Oracle(256, 128, Ra=1e6, init_amp=amp, seed=3)
    F = o.fields()
    H = F["H"].ravel()
    assert H.min() >= -amp and H.max() < amp
    assert abs(H.mean()) < 4 * amp / math.sqrt(3 * H.size)
    assert stats.kstest(H, stats.uniform(loc=-amp, scale=2 * amp).cdf).pvalue > 1e-3
    assert np.all(F["H"][:, 1:] != F["H"][:, :-1]) and np.all(F["H"][1:] != F["H"][:-1])
    assert np.all(F["T"][F["H"] > 0] == 0.0) and np.all(F["fl"][F["H"] <= 0] == 0.0)
    assert np.array_equal(F["T"][F["H"] <= 0], F["H"][F["H"] <= 0])
    assert np.all(F["rho"] == 1.0) and np.all(F["ux"] == 0.0) and np.all(F["uy"] == 0.0)
    f, _ = o.populations()
    _, _, w, _ = orc.lattice()
    assert np.array_equal(f, np.broadcast_to(w[:, None, None], f.shape))
    other = orc.Oracle(256, 128, Ra=1e6, init_amp=amp, seed=4).fields()["H"]
    assert np.abs(other - F["H"]).max() > amp   # the seed matters


def test_nan_flag_marks_a_non_finite_cell(orc):
    o = orc.Oracle(40, 20, Ra=1e5)
    o.step(3)
    assert o.diagnostics()["nan_flag"] == 0.0
    f, g = o.populations()
    g[4, 7, 11] = np.nan
    o.set_populations(f, g, 3)
    o.step(1)
    assert o.diagnostics()["nan_flag"] == 1.0


# ------------------------------------------------- planted mistakes
# Each pin above must fail on an oracle with the matching plausible slip.
MUTATIONS = {
    "k2f from alpha": (
        [("d->k2f = 1.0 / (d->nu / CS2 + 0.5);", "d->k2f = 1.0 / (d->alpha / CS2 + 0.5);")],
        [check_shear_wave_decays_at_nu]),
    "f_l factor dropped": (
        [("ux = fl * (jx + 0.5 * Fx) / rho;", "ux = (jx + 0.5 * Fx) / rho;"),
         ("uy = fl * (jy + 0.5 * Fy) / rho;", "uy = (jy + 0.5 * Fy) / rho;")],
        [check_velocity_is_fl_times_ustar]),
    "half-force shift dropped": (
        [("uy = fl * (jy + 0.5 * Fy) / rho;", "uy = fl * jy / rho;")],
        [check_velocity_is_fl_times_ustar]),
    "Href and heated length swapped in Nu": (
        [("s->Q_last * s->d.Href / (s->d.alpha * RHO0 * CP * (TH - TM) * s->d.heated_len)",
          "s->Q_last * s->d.heated_len / (s->d.alpha * RHO0 * CP * (TH - TM) * s->d.Href)")],
        [lambda orc: check_wall_flux_and_nu(orc, *WALL_FLUX_CASES[0]),
         lambda orc: check_wall_flux_and_nu(orc, *WALL_FLUX_CASES[2])]),
    "inflow counted once instead of twice": (
        [("qin += 2.0 * W[i] * CP * TH - 2.0 * gprev[ko];", "qin += W[i] * CP * TH - gprev[ko];")],
        [lambda orc: check_wall_flux_and_nu(orc, *WALL_FLUX_CASES[0])]),
    # and some older pins, each against the slip it is meant to catch
    "Eq. 4 rest term w_0 C_p T dropped": (
        [("out[0] = H - CP * T + W[0] * CP * T;", "out[0] = H - CP * T;")],
        [test_geq_moments]),
    "Eq. 2 k1 and k2 exchanged": (
        [("out[i] = p[i] - k0 * n[i] - (k1 - k0) * W[i] * cM1 / CS2 -\n"
          "                 (k2 - k0) * W[i] * q_contract(i, M2) / (2.0 * CS2 * CS2);",
          "out[i] = p[i] - k0 * n[i] - (k2 - k0) * W[i] * cM1 / CS2 -\n"
          "                 (k1 - k0) * W[i] * q_contract(i, M2) / (2.0 * CS2 * CS2);")],
        [test_g_collision_is_block_relaxation]),
    "anti-bounce-back sign": (
        [("g[i] = -gprev[ko] + 2.0 * W[i] * CP * TH;", "g[i] = gprev[ko] + 2.0 * W[i] * CP * TH;")],
        [test_heated_strip_energy_budget]),
    "Stefan rows not periodic": (
        [("if (s->p.problem == ORC_STEFAN) sy = ((sy % ny) + ny) % ny; /* periodic y */", "")],
        [lambda orc: test_stefan_front_and_profile_match_neumann(orc, 1.0)]),
    "initial perturbation on [0, 2 amp)": (
        [("const double delta = p->init_amp * (2.0 * r - 1.0);",
          "const double delta = p->init_amp * (2.0 * r);")],
        [test_initial_perturbation_is_uniform_on_plus_minus_amp]),
    "buoyancy sign": (
        [("Fy = RHO0 * s->d.gbeta * (T - TM);", "Fy = -RHO0 * s->d.gbeta * (T - TM);")],
        [test_hot_fluid_rises, test_hydrostatic_balance_sets_force_sign]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_fail_on_planted_mistakes(orc, tmp_path, name):
    replacements, checks = MUTATIONS[name]
    path = orc.compile_variant(replacements, str(tmp_path))
    with orc.variant(path):
        for check in checks:
            with pytest.raises(AssertionError):
                check(orc)
