// Generated by gen_grid_box_spline.py: the quadratic pieces of the grid box
// spline beta_b (see that script).  For a tap at (floor, frac) = (z, (u, v)),
// u = U / 1024, v = V / 1024, the weight of sample z + (i1, i2),
// i1 in {-1, 0, 1}, i2 in {-2, -1, 0}, is beta_b(-i1 + u, -i2 + v) * 2^23 =
// w[(i1 + 1) * 3 + (i2 + 2)] (cell c = (-i1, -i2)), with
// 8 beta_b(c + (u, v)) = k0 + k1 u + k2 v + k3 u^2 + k4 u v + k5 v^2 per triangle
// tri of the cell (0: v <= u, u + v <= 1; 1: v <= u, u + v >= 1;
// 2: v >= u, u + v >= 1; 3: v >= u, u + v <= 1).
#pragma once

__device__ __forceinline__ void grid_box_spline_weights(int tri, int U, int V, int w[9]) {
  const int UU = U * U, UV = U * V, VV = V * V;
  switch (tri) {
    case 0:
      w[0] = 2 * (1 << 20) + -4 * (U << 10) + -4 * (V << 10) + 2 * UU + 4 * UV + 2 * VV;  // cell (1, 2)
      w[1] = 2 * (1 << 20) + -4 * (U << 10) + 4 * (V << 10) + 2 * UU + -4 * UV + -2 * VV;  // cell (1, 1)
      w[2] = 0;  // cell (1, 0)
      w[3] = 2 * (1 << 20) + 4 * (U << 10) + -4 * (V << 10) + -4 * UU;  // cell (0, 2)
      w[4] = 2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * UU + -4 * VV;  // cell (0, 1)
      w[5] = 4 * VV;  // cell (0, 0)
      w[6] = 2 * UU + -4 * UV + 2 * VV;  // cell (-1, 2)
      w[7] = 2 * UU + 4 * UV + -2 * VV;  // cell (-1, 1)
      w[8] = 0;  // cell (-1, 0)
      return;
    case 1:
      w[0] = 0;  // cell (1, 2)
      w[1] = 4 * (1 << 20) + -8 * (U << 10) + 4 * UU;  // cell (1, 1)
      w[2] = 0;  // cell (1, 0)
      w[3] = 4 * (1 << 20) + -8 * (V << 10) + -2 * UU + 4 * UV + 2 * VV;  // cell (0, 2)
      w[4] = 2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * UU + -4 * VV;  // cell (0, 1)
      w[5] = -2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -2 * UU + -4 * UV + 2 * VV;  // cell (0, 0)
      w[6] = 2 * UU + -4 * UV + 2 * VV;  // cell (-1, 2)
      w[7] = -2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * VV;  // cell (-1, 1)
      w[8] = 2 * (1 << 20) + -4 * (U << 10) + -4 * (V << 10) + 2 * UU + 4 * UV + 2 * VV;  // cell (-1, 0)
      return;
    case 2:
      w[0] = 0;  // cell (1, 2)
      w[1] = 4 * (1 << 20) + -8 * (U << 10) + 2 * UU + 4 * UV + -2 * VV;  // cell (1, 1)
      w[2] = 2 * UU + -4 * UV + 2 * VV;  // cell (1, 0)
      w[3] = 4 * (1 << 20) + -8 * (V << 10) + 4 * VV;  // cell (0, 2)
      w[4] = 2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * UU + -4 * VV;  // cell (0, 1)
      w[5] = -2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * UU;  // cell (0, 0)
      w[6] = 0;  // cell (-1, 2)
      w[7] = -2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + 2 * UU + -4 * UV + -2 * VV;  // cell (-1, 1)
      w[8] = 2 * (1 << 20) + -4 * (U << 10) + -4 * (V << 10) + 2 * UU + 4 * UV + 2 * VV;  // cell (-1, 0)
      return;
    default:
      w[0] = 2 * (1 << 20) + -4 * (U << 10) + -4 * (V << 10) + 2 * UU + 4 * UV + 2 * VV;  // cell (1, 2)
      w[1] = 2 * (1 << 20) + -4 * (U << 10) + 4 * (V << 10) + -4 * VV;  // cell (1, 1)
      w[2] = 2 * UU + -4 * UV + 2 * VV;  // cell (1, 0)
      w[3] = 2 * (1 << 20) + 4 * (U << 10) + -4 * (V << 10) + -2 * UU + -4 * UV + 2 * VV;  // cell (0, 2)
      w[4] = 2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * UU + -4 * VV;  // cell (0, 1)
      w[5] = -2 * UU + 4 * UV + 2 * VV;  // cell (0, 0)
      w[6] = 0;  // cell (-1, 2)
      w[7] = 4 * UU;  // cell (-1, 1)
      w[8] = 0;  // cell (-1, 0)
      return;
  }
}
