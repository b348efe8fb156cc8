// Per-pixel step solve shared by the kernels of libbsf.so:
// covariance -> minimum-kurtosis scales -> integer steps.
//
// Section 1.1 of the paper: a covariance C fixes the scale vector a of the
// four-directional box spline up to one degree of freedom; the box spline of
// minimum kurtosis is chosen (Frobenius norm of the kurtosis matrix
// kappa sum_k a_k^4 u_k u_k^T, the form the paper prints for its rotated
// box spline in Section 2.3).  For the order-n filter C = (n/12) sum_k A_k u_k u_k^T,
// A_k = a_k^2.  With u = (A2 + A4)/2 the family is
//   A1 = c1 - u, A2 = u + b, A3 = c3 - u, A4 = u - b,
//   c1 = (12/n) C11, c3 = (12/n) C22, b = (12/n) C12,  |b| <= u <= min(c1, c3),
// feasible iff |C12| <= min(C11, C22), which is the elongation bound e(phi)
// of eq. "boundE".  dF/du = 0 is a strictly increasing cubic; with u = s/4 + v
// (s = c1 + c3, d = c1 - c3) it reads v^3 + p v + q = 0,
//   p = (2.5 d^2 + 2 c1 c3 + 8 b^2) / 8,   q = s (b^2 - d^2/4) / 8.
// Newton's method from v0 = -q/p converges monotonically; two steps reach
// float32 precision and are taken.  Every operation is an explicit IEEE round-to-nearest float32
// intrinsic (no contraction into fused multiply-add), so the result, and the
// integer steps rounded from it, are reproducible bit for bit by any IEEE
// float32 implementation of the same sequence.
//
// Steps: lambda_k = sqrt(1 + A_k / |d_k|^2) (BSF_STEP_D1: L grid samples
// spaced |d_k| apart then have variance A_k/12, that of a box of width a_k),
// or lambda_k = a_k / |d_k| (BSF_STEP_D1_PAPER); L_k = the admissible integer
// nearest lambda_k (odd when n is odd), ties to the larger.
#pragma once

#include "bsf_device.cuh"

namespace bsf_solve {

constexpr float kLMax = 32767.f;

struct Solved {
  float A[4];
  int flags;  // 1 = clamped to e(phi), 2 = non-finite input
};

__device__ __forceinline__ Solved solve_scales(float C11, float C12, float C22, float B) {
  Solved r;
  r.flags = 0;
  if (!(isfinite(C11) && isfinite(C12) && isfinite(C22))) {
    r.flags |= 2;
    C11 = 0.f; C12 = 0.f; C22 = 0.f;
  }
  float c11 = fmaxf(C11, 0.f), c22 = fmaxf(C22, 0.f);
  float m = fminf(c11, c22);
  float c12 = C12;
  if (fabsf(c12) > m) { r.flags |= 1; c12 = copysignf(m, c12); }
  const float c1 = __fmul_rn(B, c11), c3 = __fmul_rn(B, c22), b = __fmul_rn(B, c12);
  const float s = __fadd_rn(c1, c3), d = __fsub_rn(c1, c3);
  const float bb = __fmul_rn(b, b), dd = __fmul_rn(d, d);
  const float p = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(2.5f, dd), __fmul_rn(2.f, __fmul_rn(c1, c3))),
                                      __fmul_rn(8.f, bb)), 0.125f);
  const float q = __fmul_rn(__fmul_rn(s, __fsub_rn(bb, __fmul_rn(0.25f, dd))), 0.125f);
  float v = (p > 0.f) ? __fdiv_rn(-q, p) : 0.f;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float v2 = __fmul_rn(v, v);
    const float h = __fadd_rn(__fmul_rn(__fadd_rn(v2, p), v), q);
    const float dh = __fadd_rn(__fmul_rn(3.f, v2), p);
    if (dh > 0.f) v = __fsub_rn(v, __fdiv_rn(h, dh));
  }
  float u = __fadd_rn(__fmul_rn(0.25f, s), v);
  u = fminf(fmaxf(u, fabsf(b)), fminf(c1, c3));
  r.A[0] = fmaxf(__fsub_rn(c1, u), 0.f);
  r.A[1] = fmaxf(__fadd_rn(u, b), 0.f);
  r.A[2] = fmaxf(__fsub_rn(c3, u), 0.f);
  r.A[3] = fmaxf(__fsub_rn(u, b), 0.f);
  return r;
}

__device__ __forceinline__ int round_step(float lam, int n) {
  lam = fminf(lam, kLMax);
  int L = (n & 1) ? 2 * __float2int_rd(__fmul_rn(0.5f, lam)) + 1 : __float2int_rd(__fadd_rn(lam, 0.5f));
  L = max(L, 1);
  return min(L, (int)kLMax);
}

// Largest |offset| of any tap: along d_k the offsets run from -n(L+1)/2 to n(L-1)/2.
__device__ __forceinline__ int tap_reach(const int L[4], int n) {
  int lo[4], hi[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) { lo[k] = -(n * (L[k] + 1)) / 2; hi[k] = (n * (L[k] - 1)) / 2; }
  const int xr = max(-(lo[0] + lo[1] - hi[3]), hi[0] + hi[1] - lo[3]);
  const int yr = max(-(lo[1] + lo[2] + lo[3]), hi[1] + hi[2] + hi[3]);
  return max(xr, yr);
}


// Integer steps of one pixel; returns false when the taps would leave the
// padding R (the steps are then reset to 1).  flags: 1 clamped, 2 non-finite.
// B = 12/n as float32 (exactly 12, 6 or 4)
__device__ __forceinline__ float scale_of_order(int n) { return n == 1 ? 12.f : (n == 2 ? 6.f : 4.f); }

__device__ __forceinline__ bool pixel_steps(float C11, float C12, float C22, int n, int rule,
                                            int R, int L[4], int& flags, int& reach) {
  Solved sv = solve_scales(C11, C12, C22, scale_of_order(n));
  flags = sv.flags;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float a = (k & 1) ? __fmul_rn(sv.A[k], 0.5f) : sv.A[k];  // A / |d_k|^2
    const float lam = (rule == BSF_STEP_D1_PAPER) ? __fsqrt_rn(a) : __fsqrt_rn(__fadd_rn(1.f, a));
    L[k] = round_step(lam, n);
  }
  reach = tap_reach(L, n);
  if (R >= 0 && reach > R) {  // keep every tap inside the workspace (R >= 3n always)
    L[0] = L[1] = L[2] = L[3] = 1;
    reach = tap_reach(L, n);
    return false;
  }
  return true;
}

}  // namespace bsf_solve
