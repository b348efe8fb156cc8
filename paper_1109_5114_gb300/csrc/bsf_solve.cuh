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

// ---------------------------------------------------------------------------
// Sampled continuous box spline (BSF_STEP_SAMPLED, order 1): lambda_k =
// a_k / |d_k| = sqrt(A_k / |d_k|^2), quantised to Lq_k = max(1, RNE(512
// lambda_k)).  The taps lie within sum lambda |d|_inf / 2 of the pixel and
// the interpolation reaches one sample left, right and up, two down:
// reach = max(ceil(Sx / 512), ceil(Sy / 512)) / 2 + 3, Sx = Lq1 + Lq2 + Lq4,
// Sy = Lq2 + Lq3 + Lq4.  Out of reach: Lq = 512 (lambda = 1), false.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int sampled_reach(const int Lq[4]) {
  const long long sx = (long long)Lq[0] + Lq[1] + Lq[3], sy = (long long)Lq[1] + Lq[2] + Lq[3];
  const long long cx = (sx + 511) >> 9, cy = (sy + 511) >> 9;
  const long long r = (cx > cy ? cx : cy) / 2 + 3;
  return r > (1 << 30) ? (1 << 30) : (int)r;
}

__device__ __forceinline__ bool pixel_steps_sampled(float C11, float C12, float C22, int R, int Lq[4],
                                                    int& flags, int& reach) {
  Solved sv = solve_scales(C11, C12, C22, 12.f);
  flags = sv.flags;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float a = (k & 1) ? __fmul_rn(sv.A[k], 0.5f) : sv.A[k];  // A / |d_k|^2
    const float lam = fminf(__fsqrt_rn(a), 4194304.f);               // keeps 512 lambda in int range
    Lq[k] = max(__float2int_rn(__fmul_rn(lam, 512.f)), 1);
  }
  reach = sampled_reach(Lq);
  if (R >= 0 && reach > R) {
    Lq[0] = Lq[1] = Lq[2] = Lq[3] = 512;
    reach = sampled_reach(Lq);
    return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// The second box spline beta'_a (Section 2.3): boxes along the grid vectors
// e_1 = (2, 1), e_2 = (1, 2), e_3 = (-1, 2), e_4 = (-2, 1), |e_k|^2 = 5, with
// covariance (n/12) sum_k A_k e_k e_k^T / 5.  With M = (12/n) C, carried
// times 3: P3 = 4 M11 - M22 = 3 (A1 + A4), Q3 = 4 M22 - M11 = 3 (A2 + A3),
// m3 = 7.5 M12 = 3 (A1 + A2 - A3 - A4); the family is
//   3A = (T, (P3 + Q3 + m3)/2 - T, (Q3 - P3 - m3)/2 + T, P3 - T),
// feasible iff P3, Q3 >= 0 and |m3| <= P3 + Q3 (beyond: clamped, flag 1).
// The kurtosis sum_k A_k^2 u_k u_k^T of Section 2.3 has, along the family,
// the stationarity cubic V^3 + p V + q = 0 with T = P3/2 + m3/4 + V,
//   p = (50 (P3^2 + Q3^2) + 32 (P3 - Q3)^2 + 43 m3^2) / 400 > 0,
//   q = m3 (P3 - Q3) (P3 + Q3) / 32,
// solved like the Cartesian one: two Newton steps from -q/p.  A holds 3A_k.
// ---------------------------------------------------------------------------
__device__ __forceinline__ Solved solve_scales_k(float C11, float C12, float C22, float B) {
  Solved r;
  r.flags = 0;
  if (!(isfinite(C11) && isfinite(C12) && isfinite(C22))) {
    r.flags |= 2;
    C11 = 0.f; C12 = 0.f; C22 = 0.f;
  }
  const float c11 = fmaxf(C11, 0.f), c22 = fmaxf(C22, 0.f);
  const float m11 = __fmul_rn(B, c11), m22 = __fmul_rn(B, c22), m12 = __fmul_rn(B, C12);
  float P3 = __fsub_rn(__fmul_rn(4.f, m11), m22);
  float Q3 = __fsub_rn(__fmul_rn(4.f, m22), m11);
  float m3 = __fmul_rn(7.5f, m12);
  if (P3 < 0.f) { P3 = 0.f; r.flags |= 1; }
  if (Q3 < 0.f) { Q3 = 0.f; r.flags |= 1; }
  const float S3 = __fadd_rn(P3, Q3);
  if (fabsf(m3) > S3) { m3 = copysignf(S3, m3); r.flags |= 1; }
  const float dPQ = __fsub_rn(P3, Q3);
  const float p = __fdiv_rn(
      __fadd_rn(__fadd_rn(__fmul_rn(50.f, __fadd_rn(__fmul_rn(P3, P3), __fmul_rn(Q3, Q3))),
                          __fmul_rn(32.f, __fmul_rn(dPQ, dPQ))),
                __fmul_rn(43.f, __fmul_rn(m3, m3))),
      400.f);
  const float q = __fmul_rn(__fmul_rn(__fmul_rn(m3, dPQ), S3), 0.03125f);
  float v = (p > 0.f) ? __fdiv_rn(-q, p) : 0.f;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float v2 = __fmul_rn(v, v);
    const float h = __fadd_rn(__fmul_rn(__fadd_rn(v2, p), v), q);
    const float dh = __fadd_rn(__fmul_rn(3.f, v2), p);
    if (dh > 0.f) v = __fsub_rn(v, __fdiv_rn(h, dh));
  }
  float T = __fadd_rn(__fadd_rn(__fmul_rn(0.5f, P3), __fmul_rn(0.25f, m3)), v);
  const float half = __fmul_rn(0.5f, __fadd_rn(S3, m3));
  T = fminf(fmaxf(T, fmaxf(__fmul_rn(0.5f, __fadd_rn(dPQ, m3)), 0.f)), fminf(P3, half));
  r.A[0] = fmaxf(T, 0.f);
  r.A[1] = fmaxf(__fsub_rn(half, T), 0.f);
  r.A[2] = fmaxf(__fadd_rn(__fmul_rn(0.5f, __fsub_rn(__fsub_rn(Q3, P3), m3)), T), 0.f);
  r.A[3] = fmaxf(__fsub_rn(P3, T), 0.f);
  return r;
}

// Largest |offset| of the taps of beta'_a: along e_k the offsets run from
// -n(L+1)/2 to n(L-1)/2 units of e_k.
__device__ __forceinline__ int tap_reach_k(const int L[4], int n) {
  int lo[4], hi[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) { lo[k] = -(n * (L[k] + 1)) / 2; hi[k] = (n * (L[k] - 1)) / 2; }
  const int xr = max(-(2 * lo[0] + lo[1] - hi[2] - 2 * hi[3]), 2 * hi[0] + hi[1] - lo[2] - 2 * lo[3]);
  const int yr = max(-(lo[0] + 2 * lo[1] + 2 * lo[2] + lo[3]), hi[0] + 2 * hi[1] + 2 * hi[2] + hi[3]);
  return max(xr, yr);
}

__device__ __forceinline__ bool pixel_steps_k(float C11, float C12, float C22, int n, int rule,
                                              int R, int L[4], int& flags, int& reach) {
  Solved sv = solve_scales_k(C11, C12, C22, scale_of_order(n));
  flags = sv.flags;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float a = __fdiv_rn(sv.A[k], 15.f);  // A / |e_k|^2 from 3A
    const float lam = (rule == BSF_STEP_D1_PAPER) ? __fsqrt_rn(a) : __fsqrt_rn(__fadd_rn(1.f, a));
    L[k] = round_step(lam, n);
  }
  reach = tap_reach_k(L, n);
  if (R >= 0 && reach > R) {
    L[0] = L[1] = L[2] = L[3] = 1;
    reach = tap_reach_k(L, n);
    return false;
  }
  return true;
}

// Sampled continuous box spline of the second set (BSF_STEP_SAMPLED with
// BSF_DIRS_SECOND / _PAIR, order 1): lambda_k = a_k / sqrt(5) = sqrt(3A_k / 15),
// quantised to Lq_k = max(1, RNE(32 lambda_k)).  The taps lie within
// Sx / 64 across and Sy / 64 down of the pixel (Sx = 2 Lq1 + Lq2 + Lq3 +
// 2 Lq4, Sy = Lq1 + 2 Lq2 + 2 Lq3 + Lq4) and the interpolation reaches two
// samples left, three right, five up: reach = max(ceil(Sx / 32),
// ceil(Sy / 32)) / 2 + 7.  Out of reach: Lq = 32 (lambda = 1), false.
__device__ __forceinline__ int sampled_reach_k(const int Lq[4]) {
  const long long sx = 2LL * Lq[0] + Lq[1] + Lq[2] + 2LL * Lq[3];
  const long long sy = (long long)Lq[0] + 2LL * Lq[1] + 2LL * Lq[2] + Lq[3];
  const long long cx = (sx + 31) >> 5, cy = (sy + 31) >> 5;
  const long long r = (cx > cy ? cx : cy) / 2 + 7;
  return r > (1 << 30) ? (1 << 30) : (int)r;
}

__device__ __forceinline__ bool pixel_steps_sampled_k(float C11, float C12, float C22, int R, int Lq[4],
                                                      int& flags, int& reach) {
  Solved sv = solve_scales_k(C11, C12, C22, 12.f);
  flags = sv.flags;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float lam = fminf(__fsqrt_rn(__fdiv_rn(sv.A[k], 15.f)), 33554432.f);  // 32 lambda in int range
    Lq[k] = max(__float2int_rn(__fmul_rn(lam, 32.f)), 1);
  }
  reach = sampled_reach_k(Lq);
  if (R >= 0 && reach > R) {
    Lq[0] = Lq[1] = Lq[2] = Lq[3] = 32;
    reach = sampled_reach_k(Lq);
    return false;
  }
  return true;
}

// Algorithm 2's sector: beta'_a where its elongation bound is the larger one,
// i.e. |C11 - C22| < 3 |C12| < 6 |C11 - C22| (|C11 - C22| rounded once to
// float64; 3|C12| and 2|C11 - C22| are exact there).
__device__ __forceinline__ bool use_second_set(float C11, float C12, float C22) {
  const double d = fabs(__dsub_rn((double)C11, (double)C22));
  const double a = fabs((double)C12);
  return d < 3.0 * a && a < 2.0 * d;
}

// Direction sets of the integer-step filter (BSF_DIRS_*): steps of one pixel
// for the set the context uses; `second` says which set the pixel takes.
__device__ __forceinline__ bool pixel_steps_set(int dirset, float C11, float C12, float C22, int n,
                                                int rule, int R, int L[4], int& flags, int& reach,
                                                bool& second) {
  second = dirset == BSF_DIRS_SECOND || (dirset == BSF_DIRS_PAIR && use_second_set(C11, C12, C22));
  return second ? pixel_steps_k(C11, C12, C22, n, rule, R, L, flags, reach)
                : pixel_steps(C11, C12, C22, n, rule, R, L, flags, reach);
}

// ---------------------------------------------------------------------------
// Float32 elementary functions for the log-parameter fields, written out as
// fixed sequences of IEEE round-to-nearest operations (no contraction), so
// that any IEEE float32 implementation of the same steps gives the same bits.
//   exp: Cody-Waite reduction x = k ln2 + r, |r| <= ln2/2, with ln2 split into
//        a 16-bit head (k ln2_hi exact) and a tail; e^r by its Taylor
//        polynomial of degree 7 (Horner); times 2^k from the exponent bits.
//        Input clamped to [-87, 88].  Within 1.2 ulp of the exact value.
//   sin, cos: Cody-Waite reduction x = j pi/2 + r, |r| <= pi/4, with pi/2
//        split into two 12-bit heads and a tail (exact products for
//        |j| < 2^12, i.e. |x| below about 6400); Taylor polynomials of degree
//        9 (sin) and 10 (cos); the quadrant j mod 4 selects and signs them.
//        Within 1.5 x 2^-24 absolute on [-20, 20].
// (Cody and Waite, Software Manual for the Elementary Functions, 1980.)
// ---------------------------------------------------------------------------
constexpr float kLn2Hi = 0.693145751953125f, kLn2Lo = 1.428606765330187e-06f;
constexpr float kLog2e = 1.4426950216293335f;
constexpr float kPio2A = 1.57080078125f, kPio2B = -4.453584551811218e-06f,
                kPio2C = -8.705516307827565e-10f, k2OverPi = 0.6366197466850281f;
// 1/k! rounded to float32
constexpr float kF2 = 0.5f, kF3 = 0.1666666716337204f, kF4 = 0.0416666679084301f,
                kF5 = 0.008333333767950535f, kF6 = 0.0013888889225199819f,
                kF7 = 0.00019841270113829523f, kF8 = 2.4801587642286904e-05f,
                kF9 = 2.7557318844628753e-06f, kF10 = 2.755731998149713e-07f;

__device__ __forceinline__ float exp_cw(float x) {
  x = fminf(fmaxf(x, -87.f), 88.f);
  const float kf = rintf(__fmul_rn(x, kLog2e));
  const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(kf, kLn2Hi)), __fmul_rn(kf, kLn2Lo));
  float p = kF7;
  p = __fadd_rn(__fmul_rn(p, r), kF6);
  p = __fadd_rn(__fmul_rn(p, r), kF5);
  p = __fadd_rn(__fmul_rn(p, r), kF4);
  p = __fadd_rn(__fmul_rn(p, r), kF3);
  p = __fadd_rn(__fmul_rn(p, r), kF2);
  p = __fadd_rn(__fmul_rn(p, r), 1.f);
  p = __fadd_rn(__fmul_rn(p, r), 1.f);
  return __fmul_rn(p, __int_as_float(((int)kf + 127) << 23));
}

__device__ __forceinline__ void sincos_cw(float x, float& sn, float& cs) {
  const float jf = rintf(__fmul_rn(x, k2OverPi));
  float r = __fsub_rn(x, __fmul_rn(jf, kPio2A));
  r = __fsub_rn(r, __fmul_rn(jf, kPio2B));
  r = __fsub_rn(r, __fmul_rn(jf, kPio2C));
  const float r2 = __fmul_rn(r, r);
  float sp = kF9;
  sp = __fsub_rn(__fmul_rn(sp, r2), kF7);
  sp = __fadd_rn(__fmul_rn(sp, r2), kF5);
  sp = __fsub_rn(__fmul_rn(sp, r2), kF3);
  sp = __fadd_rn(__fmul_rn(__fmul_rn(sp, r2), r), r);
  float cp = -kF10;
  cp = __fadd_rn(__fmul_rn(cp, r2), kF8);
  cp = __fsub_rn(__fmul_rn(cp, r2), kF6);
  cp = __fadd_rn(__fmul_rn(cp, r2), kF4);
  cp = __fsub_rn(__fmul_rn(cp, r2), kF2);
  cp = __fadd_rn(__fmul_rn(cp, r2), 1.f);
  switch ((int)jf & 3) {
    case 0: sn = sp; cs = cp; break;
    case 1: sn = cp; cs = -sp; break;
    case 2: sn = -sp; cs = -cp; break;
    default: sn = -cp; cs = sp; break;
  }
}

// ---------------------------------------------------------------------------
// Covariance of one pixel from a field of kind BSF_COV_C (planes C11, C12,
// C22) or BSF_COV_LOGSIG_THETA_LOGRHO (planes log sigma, theta, log rho), in
// float32 with the functions above, in this fixed order:
//   s2 = exp(2 ls), rho = exp(lr), k = (2 s2) / (1 + rho),
//   C11 = k (rho c^2 + s^2), C22 = k (rho s^2 + c^2), C12 = k ((rho - 1) (s c))
// (trace 2 sigma^2, eigenvalue ratio rho, major axis at theta).
// ---------------------------------------------------------------------------
struct LogCov {  // intermediates kept for the chain rule
  float k, rho, c, s, C11, C12, C22;
};

__device__ __forceinline__ LogCov cov_of_log_params(float ls, float th, float lr) {
  LogCov r;
  const float s2 = exp_cw(__fmul_rn(2.f, ls));
  r.rho = exp_cw(lr);
  r.k = __fdiv_rn(__fmul_rn(2.f, s2), __fadd_rn(1.f, r.rho));
  sincos_cw(th, r.s, r.c);
  const float cc = __fmul_rn(r.c, r.c), ss = __fmul_rn(r.s, r.s), sc = __fmul_rn(r.s, r.c);
  r.C11 = __fmul_rn(r.k, __fadd_rn(__fmul_rn(r.rho, cc), ss));
  r.C22 = __fmul_rn(r.k, __fadd_rn(__fmul_rn(r.rho, ss), cc));
  r.C12 = __fmul_rn(r.k, __fmul_rn(__fsub_rn(r.rho, 1.f), sc));
  return r;
}

__device__ __forceinline__ void load_cov(const float* __restrict__ cov, int kind, long long HW,
                                         long long i, float& C11, float& C12, float& C22) {
  const float a = cov[i], b = cov[HW + i], c = cov[2 * HW + i];
  if (kind == BSF_COV_LOGSIG_THETA_LOGRHO) {
    const LogCov r = cov_of_log_params(a, b, c);
    C11 = r.C11; C12 = r.C12; C22 = r.C22;
  } else {
    C11 = a; C12 = b; C22 = c;
  }
}

// ---------------------------------------------------------------------------
// Continuous steps (BSF_STEP_D2).  lambda_k = sqrt(1 + A_k / |d_k|^2) is
// quantised to 2^-9 of a grid step: Hq_k = RNE(512 lambda_k), so that every
// interpolation fraction of the taps is a multiple of 2^-10.
// ---------------------------------------------------------------------------
constexpr int kHalf = 512;              // 2^(QW-1), QW = 10 fraction bits
constexpr int kHMax = 512 * 32767;

// Along d_k the samples lie at offsets a0, a0 + 1 (tap t = 0) and their
// mirror images (t = n), plus -1 for the middle tap of n = 2:
//   n = 2: a0 = (2 Hq - 1024) >> 10, offsets -a0-3 .. a0+1
//   n = 1: a0 = (Hq - 512) >> 10,    offsets -a0-2 .. a0+1
__device__ __forceinline__ int d2_a0(int Hq, int n) {
  return n == 2 ? (2 * Hq - 1024) >> 10 : (Hq - 512) >> 10;
}
__device__ __forceinline__ int d2_reach(const int Hq[4], int n) {
  int lo[4], hi[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int a0 = d2_a0(Hq[k], n);
    lo[k] = -a0 - (n == 2 ? 3 : 2);
    hi[k] = a0 + 1;
  }
  const int xr = max(-(lo[0] + lo[1] - hi[3]), hi[0] + hi[1] - lo[3]);
  const int yr = max(-(lo[1] + lo[2] + lo[3]), hi[1] + hi[2] + hi[3]);
  return max(xr, yr);
}
// Exact mass (times 2^10) of one direction's 1-D kernel and its right
// derivative with respect to lambda (times 2^10, times 2 for n = 1):
//   n = 2: sum_j max(0, 2 Hq - 1024 |j|) = 2 Hq (2m + 1) - 1024 m (m + 1),
//          m = (2 Hq - 1) >> 10;  derivative 1024 (2 floor(lambda~) + 1)
//   n = 1: 2 Hq (box of width lambda~);  derivative 2 * 1024
__device__ __forceinline__ unsigned long long d2_mass(int Hq, int n) {
  if (n == 1) return 2ull * (unsigned)Hq;
  const unsigned long long m = (unsigned long long)((2 * Hq - 1) >> 10);
  return 2ull * (unsigned)Hq * (2ull * m + 1ull) - 1024ull * m * (m + 1ull);
}
__device__ __forceinline__ unsigned long long d2_dmass(int Hq, int n) {
  if (n == 1) return 2048ull;
  return 1024ull * (2ull * (unsigned long long)(Hq >> 9) + 1ull);
}

// Steps of one pixel for the continuous path; false (identity steps,
// Hq = 512) when a sample would leave the padding R.
__device__ __forceinline__ bool pixel_steps_d2(float C11, float C12, float C22, int n, int R,
                                               int Hq[4], float lam[4], int& flags, int& reach) {
  const Solved sv = solve_scales(C11, C12, C22, scale_of_order(n));
  flags = sv.flags;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float a = (k & 1) ? __fmul_rn(sv.A[k], 0.5f) : sv.A[k];
    lam[k] = __fsqrt_rn(__fadd_rn(1.f, a));
    Hq[k] = min(__float2int_rn(__fmul_rn(lam[k], (float)kHalf)), kHMax);
  }
  reach = d2_reach(Hq, n);
  if (R >= 0 && reach > R) {
    Hq[0] = Hq[1] = Hq[2] = Hq[3] = kHalf;
    reach = d2_reach(Hq, n);
    return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Adjoint of the scale solve: given gA_k = d out / d A_k, the derivative with
// respect to (C11, C12, C22).  The forward steps are repeated; the Newton root
// v of v^3 + p v + q = 0 is differentiated implicitly,
//   dv = -(v dp + dq) / (3 v^2 + p),
// with p = (2.5 d^2 + 2 c1 c3 + 8 b^2)/8, q = s (b^2 - d^2/4)/8; where u is
// clamped, it follows the active bound; the C12 clamp and the floors at zero
// route the derivative the same way.  float32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void solve_scales_vjp(float C11, float C12, float C22, float B,
                                                 const float gA[4], float gC[3]) {
  gC[0] = gC[1] = gC[2] = 0.f;
  if (!(isfinite(C11) && isfinite(C12) && isfinite(C22))) return;
  const float c11 = fmaxf(C11, 0.f), c22 = fmaxf(C22, 0.f);
  const float m = fminf(c11, c22);
  const bool clamp12 = fabsf(C12) > m;
  const float c12 = clamp12 ? copysignf(m, C12) : C12;
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
  const float u0 = __fadd_rn(__fmul_rn(0.25f, s), v);
  const float lo = fabsf(b), hi = fminf(c1, c3);
  // A1 = c1 - u, A2 = u + b, A3 = c3 - u, A4 = u - b
  const float gu = gA[1] + gA[3] - gA[0] - gA[2];
  float gc1 = gA[0], gc3 = gA[2], gb = gA[1] - gA[3];
  if (u0 < lo) {  // u = |b|
    gb += b < 0.f ? -gu : gu;
  } else if (u0 > hi) {
    if (c1 <= c3) gc1 += gu; else gc3 += gu;
  } else {
    const float den = 3.f * v * v + p;
    if (den > 0.f) {
      const float gq = -gu / den;
      const float gp = gq * v;
      const float w = bb - 0.25f * dd;
      gc1 += 0.25f * gu + gp * (0.125f * (5.f * d + 2.f * c3)) + gq * (0.125f * (w - 0.5f * s * d));
      gc3 += 0.25f * gu + gp * (0.125f * (2.f * c1 - 5.f * d)) + gq * (0.125f * (w + 0.5f * s * d));
      gb += gp * (2.f * b) + gq * (0.25f * s * b);
    } else {
      gc1 += 0.25f * gu;
      gc3 += 0.25f * gu;
    }
  }
  float g11 = B * gc1, g22 = B * gc3, g12 = B * gb;
  if (clamp12) {  // c12 = sign(C12) min(c11, c22)
    const float gm = C12 < 0.f ? -g12 : g12;
    g12 = 0.f;
    if (c11 <= c22) g11 += gm; else g22 += gm;
  }
  gC[0] = C11 > 0.f ? g11 : 0.f;
  gC[1] = g12;
  gC[2] = C22 > 0.f ? g22 : 0.f;
}

// Chain from (C11, C12, C22) to (log sigma, theta, log rho) (float32):
//   dC/dls = 2 C,  dC/dtheta = (-2 C12, C11 - C22, 2 C12),
//   dC/dlr = rho (k (c^2, s c, s^2) - C / (1 + rho)).
__device__ __forceinline__ void log_params_vjp(const LogCov& r, const float gC[3], float gP[3]) {
  const float g11 = gC[0], g12 = gC[1], g22 = gC[2];
  const float inv = 1.f / (1.f + r.rho);
  gP[0] = 2.f * (r.C11 * g11 + r.C12 * g12 + r.C22 * g22);
  gP[1] = 2.f * r.C12 * (g22 - g11) + (r.C11 - r.C22) * g12;
  gP[2] = r.rho * ((r.k * r.c * r.c - r.C11 * inv) * g11 + (r.k * r.s * r.c - r.C12 * inv) * g12 +
                   (r.k * r.s * r.s - r.C22 * inv) * g22);
}

}  // namespace bsf_solve
