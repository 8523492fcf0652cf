"""Index arithmetic of the sweep's fast loads, replayed on the host.

Interior rows of a lattice are pulled with one base pointer per lane plus
compile-time offsets (plane p: p*128; row above / below: -/+2304; column
left / right: -/+1), with the tile's first / last lane using a base shifted
into the neighbouring tile.  Warps of the cavity that touch a side wall take
the same loads with the wall lane's out-of-lattice neighbour pointer clamped to
its own cell, and then overwrite its wall directions.  These tests recompute,
for every lane of every warp over many widths, the element each of the 18
loads reads and check that it lies inside the population buffer -- and, for a
clamped lane, inside its own tile's three rows -- so that no width can make a
fast-path load leave the allocation."""
import numpy as np
import pytest

TW, PLANES = 128, 18
RS = PLANES * TW

# (cx, cy) of D2Q9 directions 0..8, as the sweep numbers them
C = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]


def pop_index(x, y, p, ny):
    return ((x // TW) * ny + y) * RS + p * TW + (x % TW)


def load_offsets():
    """(base, offset) of the 18 loads: base 0 = own, 1 = left-shifted, 2 =
    right-shifted; offset in elements relative to that base."""
    out = []
    for P in (0, 9):
        for i, (cx, cy) in enumerate(C):
            base = 1 if cx == 1 else (2 if cx == -1 else 0)
            out.append((base, (P + i) * TW - cx - cy * RS, P + i, cx, cy))
    return out


def check_width(nx, ny):
    ntx = (nx + TW - 1) // TW
    total = ntx * ny * RS
    offs = load_offsets()
    for bx in range(ntx):
        for warp in range(TW // 32):
            xw = bx * TW + warp * 32
            fastcol = xw >= 1 and xw + 31 <= nx - 2
            sidewall = not fastcol          # cavity: every other warp touches a wall
            for lane in range(32):
                lx = warp * 32 + lane
                x = bx * TW + lx
                if x >= nx:
                    continue                # inactive lane
                for y in range(1, ny - 1):  # interior rows only take the fast loads
                    i0 = pop_index(x, y, 0, ny)
                    iL = pop_index(x - 1, y, 0, ny) + 1 if (lx == 0 and x > 0) else i0
                    iR = pop_index(x + 1, y, 0, ny) - 1 if (lx == TW - 1 and x < nx - 1) else i0
                    bases = (i0, iL, iR)
                    for base, off, plane, cx, cy in offs:
                        e = bases[base] + off
                        assert 0 <= e < total, (nx, ny, x, y, plane)
                        wall_lane = (cx == 1 and x == 0) or (cx == -1 and x == nx - 1)
                        if wall_lane:
                            # clamped: stays in the cell's own tile, rows y-1..y+1
                            lo = pop_index(bx * TW, y - 1, 0, ny)
                            hi = pop_index(bx * TW, y + 1, 0, ny) + RS
                            assert lo <= e < hi, (nx, ny, x, y, plane)
                            assert sidewall
                        else:
                            # a true neighbour: the source cell's own plane element
                            want = pop_index(x - cx, y - cy, plane, ny)
                            assert e == want, (nx, ny, x, y, plane)


@pytest.mark.parametrize("nx", [2, 3, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 300, 383, 384])
def test_fast_loads_stay_in_the_buffer(nx):
    check_width(nx, 5)


def test_fast_loads_for_every_width_up_to_four_tiles():
    for nx in range(2, 4 * TW + 2):
        check_width(nx, 3)
