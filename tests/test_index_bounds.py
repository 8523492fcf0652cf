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


def plane_ofs(p, lx, paired):
    """Element of plane p (0..8 f, 9..17 g) of column lx within a tile row:
    planar for FP32 / FP64; for 16-bit storage (paired) f_i and g_i share the
    32-bit word i * TW + lx, f in the low half (element 2 w), g in the high
    half (element 2 w + 1)."""
    return 2 * ((p % 9) * TW + lx) + (1 if p >= 9 else 0) if paired else p * TW + lx


def pop_index(x, y, p, ny, paired=False):
    return ((x // TW) * ny + y) * RS + plane_ofs(p, x % TW, paired)


def load_offsets(paired=False):
    """(base, offset) of the 18 loads: base 0 = own, 1 = left-shifted, 2 =
    right-shifted; offset in elements relative to that base.  Paired: word
    offsets (row RS / 2 words, direction TW words) doubled, + 1 for g."""
    out = []
    for P in (0, 9):
        for i, (cx, cy) in enumerate(C):
            base = 1 if cx == 1 else (2 if cx == -1 else 0)
            if paired:
                off = 2 * (i * TW - cx - cy * (RS // 2)) + (1 if P else 0)
            else:
                off = (P + i) * TW - cx - cy * RS
            out.append((base, off, P + i, cx, cy))
    return out


def check_width(nx, ny, paired=False):
    ntx = (nx + TW - 1) // TW
    total = ntx * ny * RS
    offs = load_offsets(paired)
    cs = 2 if paired else 1
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
                    i0 = pop_index(x, y, 0, ny, paired)
                    iL = pop_index(x - 1, y, 0, ny, paired) + cs if (lx == 0 and x > 0) else i0
                    iR = pop_index(x + 1, y, 0, ny, paired) - cs if (lx == TW - 1 and x < nx - 1) else i0
                    bases = (i0, iL, iR)
                    for base, off, plane, cx, cy in offs:
                        e = bases[base] + off
                        assert 0 <= e < total, (nx, ny, x, y, plane)
                        wall_lane = (cx == 1 and x == 0) or (cx == -1 and x == nx - 1)
                        if wall_lane:
                            # clamped: stays in the cell's own tile, rows y-1..y+1
                            lo = pop_index(bx * TW, y - 1, 0, ny, paired)
                            hi = pop_index(bx * TW, y + 1, 0, ny, paired) + RS
                            assert lo <= e < hi, (nx, ny, x, y, plane)
                            assert sidewall
                        else:
                            # a true neighbour: the source cell's own plane element
                            want = pop_index(x - cx, y - cy, plane, ny, paired)
                            assert e == want, (nx, ny, x, y, plane)
                            if paired and plane < 9:  # the 32-bit word is aligned
                                assert e % 2 == 0


@pytest.mark.parametrize("paired", [False, True])
@pytest.mark.parametrize("nx", [2, 3, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 300, 383, 384])
def test_fast_loads_stay_in_the_buffer(nx, paired):
    check_width(nx, 5, paired)


@pytest.mark.parametrize("paired", [False, True])
def test_fast_loads_for_every_width_up_to_four_tiles(paired):
    for nx in range(2, 4 * TW + 2):
        check_width(nx, 3, paired)


def test_paired_layout_is_a_permutation_of_the_tile_row():
    """Both layouts place the 18 planes of a tile row's 128 cells on the same
    18 * 128 elements, each exactly once, and a (g_i, f_i) word starts on an
    even element."""
    for paired in (False, True):
        seen = sorted(plane_ofs(p, lx, paired) for p in range(PLANES) for lx in range(TW))
        assert seen == list(range(RS))
    for i in range(9):
        for lx in range(TW):
            f, g = plane_ofs(i, lx, True), plane_ofs(9 + i, lx, True)
            assert f % 2 == 0 and g == f + 1


# ---- one-buffer streaming (the push sweep): every cell must read and write
# the same locations, and no location may be written by two cells --------------
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]


def elem(x, y, plane, ny, paired):
    return pop_index(x, y, plane, ny, paired)


def push_sweep_sets(nx, ny, paired, stefan, flow):
    """Per cell, the elements the push sweep reads and writes, replaying the
    sweep's own arithmetic: pull_fast's bases and offsets and PushFast's
    targets (base by c_x, + c_y rows + c_x columns, slot opp(i)) for cells of
    warps clear of both side walls on interior rows; for the cavity's side-wall
    warps on interior rows pull_sidewall's and PushSide's (the same bases, the
    cell's own slots across the side wall), checked element by element against
    pull_any's and PushAny's per-direction targets, which serve everywhere else
    (y periodic for the Stefan problem)."""
    cs = 2 if paired else 1
    halves = (0, 9) if flow else (9,)
    offs = load_offsets(paired)
    out = {}
    for x in range(nx):
        bx, lx = divmod(x, TW)
        xw = bx * TW + (lx // 32) * 32
        fastcol = xw >= 1 and xw + 31 <= nx - 2
        for y in range(ny):
            inner = 1 <= y <= ny - 2
            reads, writes = [], []
            if fastcol and inner:
                i0 = pop_index(x, y, 0, ny, paired)
                iL = pop_index(x - 1, y, 0, ny, paired) + cs if lx == 0 else i0
                iR = pop_index(x + 1, y, 0, ny, paired) - cs if lx == TW - 1 else i0
                bases = (i0, iL, iR)
                for base, off, plane, cx, cy in offs:
                    if plane >= 9 or flow:
                        reads.append(bases[base] + off)
                for i, (cx, cy) in enumerate(C):
                    d = (iR if cx > 0 else (iL if cx < 0 else i0)) + cy * RS + cx * cs
                    for P in halves:
                        e = d + (2 * OPP[i] * TW + (1 if P else 0) if paired else (P + OPP[i]) * TW)
                        assert e == elem(x + cx, y + cy, P + OPP[i], ny, paired), (nx, x, y, i, P)
                        writes.append(e)
            else:
                side = not stefan and inner    # a cavity side-wall warp: pull_sidewall / PushSide
                i0 = pop_index(x, y, 0, ny, paired)
                iL = pop_index(x - 1, y, 0, ny, paired) + cs if (lx == 0 and x > 0) else i0
                iR = pop_index(x + 1, y, 0, ny, paired) - cs if (lx == TW - 1 and x < nx - 1) else i0

                def slot_elem(cell, slot, P):
                    return cell + (2 * slot * TW + (1 if P else 0) if paired else (P + slot) * TW)
                for i, (cx, cy) in enumerate(C):
                    sx, sy, tx, ty = x - cx, y - cy, x + cx, y + cy
                    if stefan:
                        sy, ty = sy % ny, ty % ny
                    src_in = 0 <= sx < nx and 0 <= sy < ny
                    dst_in = 0 <= tx < nx and 0 <= ty < ny
                    for P in halves:
                        r = elem(sx, sy, P + i, ny, paired) if src_in else elem(x, y, P + OPP[i], ny, paired)
                        w = elem(tx, ty, P + OPP[i], ny, paired) if dst_in else elem(x, y, P + i, ny, paired)
                        if side:
                            wall = (cx > 0 and x == 0) or (cx < 0 and x == nx - 1)
                            frm = (iL if cx > 0 else (iR if cx < 0 else i0)) - cy * RS - cx * cs
                            assert slot_elem(i0 if wall else frm, OPP[i] if wall else i, P) == r, (nx, x, y, i)
                            wall_t = (cx > 0 and x == nx - 1) or (cx < 0 and x == 0)
                            to = i0 if wall_t else (iR if cx > 0 else (iL if cx < 0 else i0)) + cy * RS + cx * cs
                            assert slot_elem(to, i if wall_t else OPP[i], P) == w, (nx, x, y, i)
                        reads.append(r)
                        writes.append(w)
            out[(x, y)] = (reads, writes)
    return out


@pytest.mark.parametrize("paired", [False, True])
@pytest.mark.parametrize("stefan,flow", [(False, True), (False, False), (True, False), (True, True)])
@pytest.mark.parametrize("nx,ny", [(2, 3), (3, 4), (33, 5), (127, 3), (128, 4), (129, 6), (256, 3), (300, 7)])
def test_push_sweep_reads_what_it_writes(nx, ny, paired, stefan, flow):
    total = ((nx + TW - 1) // TW) * ny * RS
    seen = set()
    for (x, y), (reads, writes) in push_sweep_sets(nx, ny, paired, stefan, flow).items():
        assert len(set(writes)) == len(writes) == len(reads), (x, y)
        assert set(reads) == set(writes), (nx, ny, x, y)
        for w in writes:
            assert 0 <= w < total
            assert w not in seen, (nx, ny, x, y, w)   # no location written by two cells
            seen.add(w)
