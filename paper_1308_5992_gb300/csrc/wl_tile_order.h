// wl_tile_order.h -- the schedule of one tile of the tile-coloured
// Kaczmarz sweep: the order of the 16 site colours inside a tile and how a
// thread's 3x3 window of r moves between consecutive steps.  Plain constexpr
// functions, compiled for the device by the kernels and for the host by the
// schedule test.
#pragma once
#ifndef __CUDACC__
#define __host__
#define __device__
#endif

// Colour of step s of a tile sweep: the 4 x 4 grid of site colours
// 4 (a mod 4) + (b mod 4) row by row, rows alternately left to right and
// right to left (serpentine), so that the sites of consecutive steps of a
// quadrant are neighbours in a row or a column.
__host__ __device__ constexpr int tile_step_colour(int s) {
  return 4 * (s >> 2) + (((s >> 2) & 1) ? 3 - (s & 3) : (s & 3));
}
// how the site of step s > 0 lies from the site of step s - 1: 1 one column
// right, 2 one column left, 3 one row down
__host__ __device__ constexpr int tile_step_move(int s) {
  return (s & 3) == 0 ? 3 : (((s >> 2) & 1) ? 2 : 1);
}
// window cell d = 3 da + db of step s - 1 that holds cell d of step s after
// the move (-1: a cell new to the window, read from shared memory)
__host__ __device__ constexpr int tile_window_src(int s, int d) {
  return tile_step_move(s) == 1 ? (d % 3 < 2 ? d + 1 : -1)
         : tile_step_move(s) == 2 ? (d % 3 > 0 ? d - 1 : -1)
                                  : (d / 3 < 2 ? d + 3 : -1);
}
// whether window cell d of step s leaves the window at the next move (all
// cells after the last step)
__host__ __device__ constexpr bool tile_window_leaves(int s, int d) {
  return s == 15 ? true
         : tile_step_move(s + 1) == 1 ? d % 3 == 0
         : tile_step_move(s + 1) == 2 ? d % 3 == 2
                                      : d / 3 == 0;
}
