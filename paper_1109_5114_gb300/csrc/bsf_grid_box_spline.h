// Generated by gen_grid_box_spline.py: the quadratic pieces of the grid box
// spline beta_b (see that script).  For a tap at (floor, frac) = (z, (u, v)),
// u = U / 1024, v = V / 1024, sample z + (i1, i2), i1 in {-1, 0, 1},
// i2 in {-2, -1, 0}, has the weight beta_b(-i1 + u, -i2 + v) * 2^23, with
// 8 beta_b(c + (u, v)) = k0 + k1 u + k2 v + k3 u^2 + k4 u v + k5 v^2 on
// triangle tri of the cell c (0: v <= u, u + v <= 1; 1: v <= u, u + v >= 1;
// 2: v >= u, u + v >= 1; 3: v >= u, u + v <= 1).
// grid_box_spline_tap returns sum_samples weight * S[base + i2 pitch + i1]
// modulo 2^bits of T; the weights are non-negative and below 2^23.
#pragma once

template <typename T, typename Load>
__device__ __forceinline__ T grid_box_spline_tap(int tri, int U, int V, int base, int pitch,
                                                 Load&& load) {
  const int UU = U * U, UV = U * V, VV = V * V;
  T f = (T)0;
  switch (tri) {
    case 0:
      f += (T)(unsigned)(2 * (1 << 20) + -4 * (U << 10) + -4 * (V << 10) + 2 * UU + 4 * UV + 2 * VV) * load(base - 2 * pitch - 1);  // cell (1, 2)
      f += (T)(unsigned)(2 * (1 << 20) + -4 * (U << 10) + 4 * (V << 10) + 2 * UU + -4 * UV + -2 * VV) * load(base - 1 * pitch - 1);  // cell (1, 1)
      f += (T)(unsigned)(2 * (1 << 20) + 4 * (U << 10) + -4 * (V << 10) + -4 * UU) * load(base - 2 * pitch);  // cell (0, 2)
      f += (T)(unsigned)(2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * UU + -4 * VV) * load(base - 1 * pitch);  // cell (0, 1)
      f += (T)(unsigned)(4 * VV) * load(base);  // cell (0, 0)
      f += (T)(unsigned)(2 * UU + -4 * UV + 2 * VV) * load(base - 2 * pitch + 1);  // cell (-1, 2)
      f += (T)(unsigned)(2 * UU + 4 * UV + -2 * VV) * load(base - 1 * pitch + 1);  // cell (-1, 1)
      return f;
    case 1:
      f += (T)(unsigned)(4 * (1 << 20) + -8 * (U << 10) + 4 * UU) * load(base - 1 * pitch - 1);  // cell (1, 1)
      f += (T)(unsigned)(4 * (1 << 20) + -8 * (V << 10) + -2 * UU + 4 * UV + 2 * VV) * load(base - 2 * pitch);  // cell (0, 2)
      f += (T)(unsigned)(2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * UU + -4 * VV) * load(base - 1 * pitch);  // cell (0, 1)
      f += (T)(unsigned)(-2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -2 * UU + -4 * UV + 2 * VV) * load(base);  // cell (0, 0)
      f += (T)(unsigned)(2 * UU + -4 * UV + 2 * VV) * load(base - 2 * pitch + 1);  // cell (-1, 2)
      f += (T)(unsigned)(-2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * VV) * load(base - 1 * pitch + 1);  // cell (-1, 1)
      f += (T)(unsigned)(2 * (1 << 20) + -4 * (U << 10) + -4 * (V << 10) + 2 * UU + 4 * UV + 2 * VV) * load(base + 1);  // cell (-1, 0)
      return f;
    case 2:
      f += (T)(unsigned)(4 * (1 << 20) + -8 * (U << 10) + 2 * UU + 4 * UV + -2 * VV) * load(base - 1 * pitch - 1);  // cell (1, 1)
      f += (T)(unsigned)(2 * UU + -4 * UV + 2 * VV) * load(base - 1);  // cell (1, 0)
      f += (T)(unsigned)(4 * (1 << 20) + -8 * (V << 10) + 4 * VV) * load(base - 2 * pitch);  // cell (0, 2)
      f += (T)(unsigned)(2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * UU + -4 * VV) * load(base - 1 * pitch);  // cell (0, 1)
      f += (T)(unsigned)(-2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * UU) * load(base);  // cell (0, 0)
      f += (T)(unsigned)(-2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + 2 * UU + -4 * UV + -2 * VV) * load(base - 1 * pitch + 1);  // cell (-1, 1)
      f += (T)(unsigned)(2 * (1 << 20) + -4 * (U << 10) + -4 * (V << 10) + 2 * UU + 4 * UV + 2 * VV) * load(base + 1);  // cell (-1, 0)
      return f;
    default:
      f += (T)(unsigned)(2 * (1 << 20) + -4 * (U << 10) + -4 * (V << 10) + 2 * UU + 4 * UV + 2 * VV) * load(base - 2 * pitch - 1);  // cell (1, 2)
      f += (T)(unsigned)(2 * (1 << 20) + -4 * (U << 10) + 4 * (V << 10) + -4 * VV) * load(base - 1 * pitch - 1);  // cell (1, 1)
      f += (T)(unsigned)(2 * UU + -4 * UV + 2 * VV) * load(base - 1);  // cell (1, 0)
      f += (T)(unsigned)(2 * (1 << 20) + 4 * (U << 10) + -4 * (V << 10) + -2 * UU + -4 * UV + 2 * VV) * load(base - 2 * pitch);  // cell (0, 2)
      f += (T)(unsigned)(2 * (1 << 20) + 4 * (U << 10) + 4 * (V << 10) + -4 * UU + -4 * VV) * load(base - 1 * pitch);  // cell (0, 1)
      f += (T)(unsigned)(-2 * UU + 4 * UV + 2 * VV) * load(base);  // cell (0, 0)
      f += (T)(unsigned)(4 * UU) * load(base - 1 * pitch + 1);  // cell (-1, 1)
      return f;
  }
}
