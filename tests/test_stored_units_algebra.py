"""The 16-bit storage modes collide in stored units: f as the scaled deviation
delta_i = (f_i - w_i) kF from the rest state, g as g_i kG.  The block collision
of delta is that of f with B0 = k0 (rho - 1) kF in place of k0 rho (a + k0 = 1
cancels the rest state), and g collides with T kG and H kG.  These tests write
that algebra out in FP64 (as the sweep evaluates it, in moment space) and check
it against the oracle's own collisions (Eq. 2 with the equilibrium of Eq. 4 for
g; the same block operator with forcing for f), on the host."""
import numpy as np
import pytest

from oracle import oracle as O

C = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)], float)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def emit(p, a, B0, B1, B2):
    """p_i <- a p_i + w_i [B0 + 3 c_i.B1 + 9/2 Q_i:B2], Q_i = c_i c_i - I/3."""
    out = np.empty(9)
    for i in range(9):
        cx, cy = C[i]
        q = cx * cx * B2[0] + 2 * cx * cy * B2[1] + cy * cy * B2[2] - (B2[0] + B2[2]) / 3
        out[i] = a * p[i] + W[i] * (B0 + 3 * (cx * B1[0] + cy * B1[1]) + 4.5 * q)
    return out


def moments(p):
    return (C[:, 0] @ p, C[:, 1] @ p, (C[:, 0] ** 2) @ p, (C[:, 0] * C[:, 1]) @ p, (C[:, 1] ** 2) @ p)


def f_collide_stored(d, rho, ux, uy, Fy, k0, k1, k2, kF):
    """The f collision on delta = (f - w) kF, as the sweep writes it."""
    jx, jy, xx, xy, yy = moments(d)
    R0 = d.sum()                       # (rho - 1) kF
    rk = rho * kF
    rux, ruy = rk * ux, rk * uy
    rxx, rxy, ryy, r3 = rux * ux, rux * uy, ruy * uy, R0 / 3
    d1, d2 = k1 - k0, k2 - k0
    s1, s2 = 1 - 0.5 * k1, 1 - 0.5 * k2
    Fk = Fy * kF
    A1x = d1 * (jx - rux)
    A1y = d1 * (jy - ruy) - s1 * Fk
    A2xx = d2 * (xx - r3 - rxx)
    A2xy = d2 * (xy - rxy) - s2 * ux * Fk
    A2yy = d2 * (yy - r3 - ryy) - s2 * 2 * uy * Fk
    return emit(d, 1 - k0, k0 * R0, (k0 * rux - A1x, k0 * ruy - A1y),
                (k0 * rxx - A2xx, k0 * rxy - A2xy, k0 * ryy - A2yy))


def g_collide_stored(gs, T, ux, uy, k0, k1, k2, kG):
    """The g collision on g kG, with T kG and H kG."""
    Hs = gs.sum()
    Ts = T * kG
    jx, jy, xx, xy, yy = moments(gs)
    d1, d2 = k1 - k0, k2 - k0
    k0T = k0 * Ts
    B1 = (k0T * ux - d1 * (jx - Ts * ux), k0T * uy - d1 * (jy - Ts * uy))
    B2 = (-d2 * (xx - Ts / 3), -d2 * xy, -d2 * (yy - Ts / 3))
    out = emit(gs, 1 - k0, k0T, B1, B2)
    out[0] += k0 * (Hs - Ts)
    return out


@pytest.mark.parametrize("kF,kG", [(1024.0, 64.0), (1.0, 1.0)])
def test_stored_unit_collisions_equal_the_oracle(kF, kG):
    rng = np.random.default_rng(3)
    for _ in range(200):
        f = W * (1 + 0.05 * rng.standard_normal(9))
        rho = f.sum()
        ux, uy, Fy = 0.05 * rng.standard_normal(3)
        k0, k1, k2 = rng.uniform(0.3, 1.9, 3)
        want = O.f_collide(f, rho, ux, uy, 0.0, Fy, k0, k1, k2)
        got = f_collide_stored((f - W) * kF, rho, ux, uy, Fy, k0, k1, k2, kF)
        assert np.allclose(got / kF + W, want, rtol=0, atol=1e-15 * max(1.0, kF / 64))

        g = rng.uniform(-0.2, 1.5, 9) * W
        H = g.sum()
        T, _ = O.invert(H, 1.0)
        g0, g1, g2 = rng.uniform(0.3, 1.9, 3)
        want = O.g_collide(g, H, T, ux, uy, g0, g1, g2)
        got = g_collide_stored(g * kG, T, ux, uy, g0, g1, g2, kG)
        assert np.allclose(got / kG, want, rtol=0, atol=1e-15)


def test_rest_state_is_a_fixed_point_in_stored_units():
    """delta = 0 (rho = 1, u = 0, no force) stays 0: the rest state needs no
    storage at all, which is why the 16-bit codecs store deviations."""
    d = f_collide_stored(np.zeros(9), 1.0, 0.0, 0.0, 0.0, 1.0, 1.2, 0.8, 1024.0)
    assert np.array_equal(d, np.zeros(9))
