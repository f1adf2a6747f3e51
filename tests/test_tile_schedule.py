"""The schedule of the tile-coloured Kaczmarz kernel, checked on the host
with the kernel's own schedule functions (csrc/wl_tile_order.h, compiled
here with the host C++ compiler).

Inside an 8x8 tile, step s (0..15) relaxes, in each of the four 4x4
quadrants k, the site of colour c = tile_step_colour(s): i = c // 4 +
4 (k // 2), j = c % 4 + 4 (k % 2).  The update of a site reads and writes r
on its 3x3 window.  A thread keeps the window in registers from one step to
the next (tile_window_src says which cell of the previous window holds each
cell), reads the cells new to the window and writes back the cells that
leave it (tile_window_leaves), all of them after the last step; one block
barrier per step orders the write-back of step s - 1 before the reads of
step s.  That is correct when (1) the windows of one step are disjoint, so
no thread reads or writes a cell another thread touches in the same step,
(2) a kept cell belongs to no other quadrant's window in either step, (3)
the source mapping names the same lattice cell, and (4) every updated cell
is written back exactly when it leaves."""
import itertools
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(HERE, "..", "paper_1308_5992_gb300", "csrc", "wl_tile_order.h")

DRIVER = r"""
#include <cstdio>
#include "wl_tile_order.h"
int main() {
  std::printf("[");
  for (int s = 0; s < 16; ++s) {
    std::printf("%s{\"colour\": %d, \"move\": %d, \"src\": [", s ? ", " : "", tile_step_colour(s),
                s ? tile_step_move(s) : 0);
    for (int d = 0; d < 9; ++d) std::printf("%s%d", d ? ", " : "", s ? tile_window_src(s, d) : -1);
    std::printf("], \"leaves\": [");
    for (int d = 0; d < 9; ++d) std::printf("%s%d", d ? ", " : "", tile_window_leaves(s, d) ? 1 : 0);
    std::printf("]}");
  }
  std::printf("]\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def sched(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("sched")
    src, exe = d / "sched.cpp", d / "sched"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-std=c++17", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)], check=True)
    return json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)


def site(sched, s, k):
    c = sched[s]["colour"]
    return c // 4 + 4 * (k // 2), c % 4 + 4 * (k % 2)


def cells(sched, s, k):
    """window cell d = 3 da + db of step s -> tile cell"""
    i, j = site(sched, s, k)
    return [(i + d // 3 - 1, j + d % 3 - 1) for d in range(9)]


def test_colours_are_the_serpentine_order(sched):
    assert [x["colour"] for x in sched] == [0, 1, 2, 3, 7, 6, 5, 4, 8, 9, 10, 11, 15, 14, 13, 12]


def test_every_tile_site_once(sched):
    seen = [site(sched, s, k) for s in range(16) for k in range(4)]
    assert sorted(seen) == [(i, j) for i in range(8) for j in range(8)]


def test_consecutive_sites_are_neighbours(sched):
    for s in range(1, 16):
        (i0, j0), (i1, j1) = site(sched, s - 1, 0), site(sched, s, 0)
        assert abs(i1 - i0) + abs(j1 - j0) == 1, s
        assert sched[s]["move"] == {(0, 1): 1, (0, -1): 2, (1, 0): 3}[(i1 - i0, j1 - j0)], s


def test_windows_of_a_step_are_disjoint(sched):
    for s in range(16):
        for k1, k2 in itertools.combinations(range(4), 2):
            assert not set(cells(sched, s, k1)) & set(cells(sched, s, k2)), (s, k1, k2)


def test_kept_cells_are_the_same_cells_and_private(sched):
    for s in range(1, 16):
        for k in range(4):
            old, new = cells(sched, s - 1, k), cells(sched, s, k)
            kept = set()
            for d, src in enumerate(sched[s]["src"]):
                if src >= 0:
                    assert new[d] == old[src], (s, k, d)  # the register holds this very cell
                    kept.add(new[d])
                else:
                    assert new[d] not in old, (s, k, d)  # a new cell is read from shared memory
            assert kept == set(old) & set(new)
            for other in range(4):
                if other != k:
                    assert not kept & (set(cells(sched, s - 1, other)) | set(cells(sched, s, other))), (s, k)


def test_write_back_covers_every_cell_once(sched):
    """A cell is written back at the end of the step after which it leaves the
    window (every cell after the last step); every cell the quadrant's thread
    ever held is written back exactly when it leaves, so the cells it wrote
    last are the ones in shared memory at the end."""
    for k in range(4):
        touched, stored = set(), []
        for s in range(16):
            win = cells(sched, s, k)
            touched |= set(win)
            leaving = {win[d] for d in range(9) if sched[s]["leaves"][d]}
            nxt = set(cells(sched, s + 1, k)) if s < 15 else set()
            assert leaving == set(win) - nxt, (s, k)
            stored += sorted(leaving)
        assert set(stored) == touched
