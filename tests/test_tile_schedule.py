"""The schedule of the tile-coloured Kaczmarz kernel, checked on the host.

Inside an 8x8 tile, colour step c (0..15) relaxes site (i, j) of each of the
four 4x4 quadrants k: i = c // 4 + 4 (k // 2), j = c % 4 + 4 (k % 2).  The
update of a site reads and writes r on its 3x3 window (the 9-point stencil
in rotated coordinates).  The kernel keeps the window in registers while it
slides along a quadrant row (two columns kept, one read, one written back).
That is correct when (1) the four windows of a step are disjoint, so the
step's updates commute, and (2) no other quadrant's window at step c or
c + 1 touches a cell a thread keeps from step c to c + 1."""
import itertools


def site(c, k):
    return c // 4 + 4 * (k // 2), c % 4 + 4 * (k % 2)


def window(c, k):
    i, j = site(c, k)
    return {(i + da, j + db) for da in (-1, 0, 1) for db in (-1, 0, 1)}


def test_every_tile_site_once():
    seen = [site(c, k) for c in range(16) for k in range(4)]
    assert sorted(seen) == [(i, j) for i in range(8) for j in range(8)]


def test_windows_of_a_step_are_disjoint():
    for c in range(16):
        for k1, k2 in itertools.combinations(range(4), 2):
            assert not window(c, k1) & window(c, k2), (c, k1, k2)


def test_kept_cells_are_private():
    for c in range(16):
        if c % 4 == 3:  # the row ends: the whole window is written back
            continue
        for k in range(4):
            i, j = site(c, k)
            kept = window(c, k) & window(c + 1, k)
            assert kept == {(i + da, j + db) for da in (-1, 0, 1) for db in (0, 1)}
            for other in range(4):
                if other != k:
                    assert not kept & (window(c, other) | window(c + 1, other)), (c, k, other)


def test_write_back_covers_every_updated_cell():
    """Column j - 1 of the window is written after steps 0..2 of a row and
    the whole window after step 3: every cell the row updates is stored."""
    for row in range(4):
        for k in range(4):
            touched, stored = set(), set()
            for u in range(4):
                c = 4 * row + u
                i, j = site(c, k)
                touched |= window(c, k)
                stored |= window(c, k) if u == 3 else {(i + da, j - 1) for da in (-1, 0, 1)}
            assert stored == touched, (row, k)
