// Continuous-step filter: the running sums sampled at off-grid taps by linear
// interpolation (Section 2.3, eq. "interpolation", read for the Cartesian
// mesh), and the exact derivative sums behind its Jacobian with respect to
// the covariance field.
//
// Per direction d_k the quantised step Hq (lambda~ = Hq / 512) fixes the
// first tap q_0 = c = n (lambda~ - 1)/2 = a0 + th / 1024 (th in 0..1023);
// the last tap is its mirror image and, for n = 2, the middle tap sits at -1:
//   n = 2: offsets  a0, a0+1, -1, -a0-3, -a0-2
//          weights  1024-th, th, -2048, th, 1024-th
//          d/dlambda 1024 * (-1, 1, 0, 1, -1)
//   n = 1: offsets  a0, a0+1, -a0-2, -a0-1
//          weights  1024-th, th, -th, th-1024
//          2 d/dlambda 1024 * (-1, 1, -1, 1)
// (the mirror tap is bracketed from above, so every derivative is the right
// derivative in lambda).  Each direction applies the weights as
//   V(X) = 1024 Base + th E,  DV(X) = 1024 E,
// with Base and E fixed +-1/-2 combinations of its samples X, so the
// 5^4 = 625 (n = 2) weighted samples of one pixel reduce to nested sums with
// one small multiplication per interpolation node, and the four derivative
// sums come out of the same pass.  All of it is exact modulo 2^b.
#pragma once

#include "bsf_solve.cuh"

namespace bsf_d2 {

using namespace bsf_solve;

// e * t modulo 2^128 for 0 <= t < 2^32, from 32 x 32 -> 64-bit partial products
__device__ __forceinline__ u128 mul_small(u128 e, unsigned t) {
  const unsigned long long lo = (unsigned long long)e, hi = (unsigned long long)(e >> 64);
  const unsigned long long p0 = (unsigned long long)(unsigned)lo * t;
  const unsigned long long p1 = (unsigned long long)(unsigned)(lo >> 32) * t;
  const unsigned long long r_lo = p0 + (p1 << 32);
  const unsigned long long carry = (r_lo < p0) ? 1ull : 0ull;
  const unsigned long long r_hi = hi * (unsigned long long)t + (p1 >> 32) + carry;
  return ((u128)r_hi << 64) | (u128)r_lo;
}
__device__ __forceinline__ uint64_t mul_small(uint64_t e, unsigned t) { return e * (uint64_t)t; }

template <typename T> __device__ __forceinline__ void addc(T& a, const T& x, int c) {
  if (c == 1) a += x;
  else if (c == -1) a -= x;
  else if (c == -2) a -= x + x;
}

// Sample i of one direction: offset (in grid steps along d_k) and the
// coefficients of the sample in Base and E.
template <int NF> struct Pattern;
template <> struct Pattern<2> {
  static constexpr int NP = 5;
  __device__ static constexpr int base(int i) { return (i == 0 || i == 4) ? 1 : (i == 2 ? -2 : 0); }
  __device__ static constexpr int diff(int i) { return (i == 1 || i == 3) ? 1 : (i == 2 ? 0 : -1); }
  // a0, a0 + 1, -1, -a0 - 3, -a0 - 2
  __device__ static int pos(int a0, int i) {
    return i == 0 ? a0 : i == 1 ? a0 + 1 : i == 2 ? -1 : i == 3 ? -a0 - 3 : -a0 - 2;
  }
};
template <> struct Pattern<1> {
  static constexpr int NP = 4;
  __device__ static constexpr int base(int i) { return i == 0 ? 1 : (i == 3 ? -1 : 0); }
  __device__ static constexpr int diff(int i) { return (i == 1 || i == 3) ? 1 : -1; }
  // a0, a0 + 1, -a0 - 2, -a0 - 1
  __device__ static int pos(int a0, int i) {
    return i == 0 ? a0 : i == 1 ? a0 + 1 : i == 2 ? -a0 - 2 : -a0 - 1;
  }
};

struct DirTaps {
  int a0;       // first interpolation bracket along d_k
  int e;        // element stride of d_k
  unsigned th;  // interpolation fraction, units of 2^-10
};

// Directions K >= kUnrolled are unrolled (the inner 25 samples for n = 2);
// the outer ones are loops, which keeps the kernel body small enough for the
// instruction cache.
constexpr int kUnrolled = 2;

// Weighted sums over the samples of directions K..3 for the sample set
// anchored at element idx.  out[0] is the value; with DER, out[1 + (j - K)]
// is the derivative sum with respect to lambda_j, j = K..3.
template <typename T, int NF, int K, bool DER>
__device__ __forceinline__ void interp_level(const T* __restrict__ S, int idx, const DirTaps* dt,
                                             T* out) {
  using P = Pattern<NF>;
  constexpr int NCI = (K == 3 || !DER) ? 1 : 4 - K;
  T base[NCI], e[NCI];
#pragma unroll
  for (int c = 0; c < NCI; ++c) { base[c] = 0; e[c] = 0; }
  const DirTaps d = dt[K];
  if constexpr (K >= kUnrolled) {
#pragma unroll
    for (int i = 0; i < P::NP; ++i) {
      T in[NCI];
      const int at = idx + P::pos(d.a0, i) * d.e;
      if constexpr (K == 3) {
        in[0] = bsf_load(S + at);
      } else {
        interp_level<T, NF, K + 1, DER>(S, at, dt, in);
      }
#pragma unroll
      for (int c = 0; c < NCI; ++c) {
        addc(base[c], in[c], P::base(i));
        addc(e[c], in[c], P::diff(i));
      }
    }
  } else {
#pragma unroll 1
    for (int i = 0; i < P::NP; ++i) {
      T in[NCI];
      interp_level<T, NF, K + 1, DER>(S, idx + P::pos(d.a0, i) * d.e, dt, in);
      const int cb = P::base(i), ce = P::diff(i);
#pragma unroll
      for (int c = 0; c < NCI; ++c) {
        addc(base[c], in[c], cb);
        addc(e[c], in[c], ce);
      }
    }
  }
  out[0] = (base[0] << 10) + mul_small(e[0], d.th);
  if constexpr (DER) {
    out[1] = e[0] << 10;
#pragma unroll
    for (int c = 1; c < NCI; ++c) out[1 + c] = (base[c] << 10) + mul_small(e[c], d.th);
  }
}

__device__ __forceinline__ double to_f64(uint64_t a) { return __ll2double_rn((long long)a); }
__device__ __forceinline__ double to_f64(u128 a) { return bsf_rn64((i128)a); }
__device__ __forceinline__ float to_f32(uint64_t a) { return bsf_rn32_i64((long long)a); }
__device__ __forceinline__ float to_f32(u128 a) { return bsf_rn32((i128)a); }

enum { kOut = 0, kOutJac = 1, kVjp = 2 };

// Resident blocks of 128 threads per SM asked of the register allocator.
// 128-bit sums: the forward at four (128 registers); with the derivative
// sums at five (96 registers, a few hundred bytes spilled to L1), measured
// 0.74-0.79 against 0.79-0.85 ms per 1024^2 image at four; the forward at
// five or six is slower.
template <typename T, int NF, int MODE> struct D2Occ {
  static constexpr int value = sizeof(T) == 8 ? (MODE == kOut ? 6 : 4) : (MODE == kOut ? 4 : 5);
};

template <typename T, int NF, typename Out, int MODE>
__global__ void __launch_bounds__(128, (D2Occ<T, NF, MODE>::value))
k_stencil_d2(const T* __restrict__ S, long long pitch, int R, const float* __restrict__ cov,
             int kind, int H, int W, int row0, int rows, float scale_f, double scale_d,
             Out* __restrict__ out, long long ldo, float* __restrict__ jac, long long ldj,
             long long jac_plane, const float* __restrict__ gout, long long ldg,
             DevStatus* st) {
  constexpr bool DER = MODE != kOut;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= rows) return;
  const long long HW = (long long)H * W, i = (long long)(row0 + y) * W + x;
  float C11, C12, C22;
  LogCov lc;
  if (kind == BSF_COV_LOGSIG_THETA_LOGRHO) {
    lc = cov_of_log_params(cov[i], cov[HW + i], cov[2 * HW + i]);
    C11 = lc.C11; C12 = lc.C12; C22 = lc.C22;
  } else {
    C11 = cov[i]; C12 = cov[HW + i]; C22 = cov[2 * HW + i];
  }
  int Hq[4], flags, reach;
  float lam[4];
  const bool in_reach = pixel_steps_d2(C11, C12, C22, NF, R, Hq, lam, flags, reach);
  {  // rare-event counters, aggregated per warp
    const unsigned act = __activemask();
    const unsigned mc = __ballot_sync(act, flags & 1), mb = __ballot_sync(act, flags & 2),
                   mr = __ballot_sync(act, !in_reach);
    if ((mc | mb | mr) && (threadIdx.x & 31) == __ffs(act) - 1) {
      if (mc) atomicAdd(&st->clamp_count, (unsigned)__popc(mc));
      if (mb) { atomicAdd(&st->bad_count, (unsigned)__popc(mb)); bsf_set_error(st, BSF_ECOV); }
      if (mr) { atomicAdd(&st->range_count, (unsigned)__popc(mr)); bsf_set_error(st, BSF_ERANGE); }
    }
  }
  const int p32 = (int)pitch;
  const int estep[4] = {1, p32 + 1, p32, p32 - 1};
  DirTaps dt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int Q0 = NF == 2 ? 2 * Hq[k] - 1024 : Hq[k] - 512;
    dt[k].a0 = Q0 >> 10;
    dt[k].th = (unsigned)(Q0 & 1023);
    dt[k].e = estep[k];
  }
  T res[DER ? 5 : 1];
  interp_level<T, NF, 0, DER>(S, (y + R) * p32 + (x + R), dt, res);

  // exact mass prod_k M_k (each M_k < 2^40) and the overflow bound
  unsigned long long Mk[4];
  u128 D = 1;
  float Df = 1.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    Mk[k] = d2_mass(Hq[k], NF);
    D *= (u128)Mk[k];
    Df *= (float)Mk[k];
  }
  const float maxq = __uint_as_float(st->max_absq_bits) + 1.f;
  const float lim = bsf_pow2_f32(ElemBits<T>::value - 1);
  if (maxq * Df * (DER ? 4.0001f : 1.0001f) >= lim) {
    atomicAdd(&st->overflow_count, 1u);
    bsf_set_error(st, BSF_EOVERFLOW);
  }
  if constexpr (MODE != kVjp) {
    if constexpr (sizeof(Out) == 4) {
      out[(long long)y * ldo + x] = __fdiv_rn(__fmul_rn(to_f32(res[0]), scale_f), bsf_rn32_u(D));
    } else {
      out[(long long)y * ldo + x] = __ddiv_rn(__dmul_rn(to_f64(res[0]), scale_d), bsf_rn64_u(D));
    }
  }
  if constexpr (DER) {
    // d out / d lambda_k = 2^-q (dacc_k M_k - acc dM_k) / (dscale M_k prod M).
    // The difference cancels most of its terms: it is formed in float64 with
    // one fused multiply-add (each operand within 2^-53 of its exact value);
    // everything after it is float32.
    const double a = to_f64(res[0]);
    const float inv = 1.f / (bsf_rn32_u(D) * (NF == 1 ? 2.f : 1.f));
    float gA[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double t = __fma_rn(to_f64(res[1 + k]), (double)Mk[k],
                                -__dmul_rn(a, (double)d2_dmass(Hq[k], NF)));
      const float jl = (float)(t * scale_d) * inv / (float)Mk[k];  // t 2^-q < 2^99 |J|
      // lambda = sqrt(1 + A / |d|^2):  d lambda / d A = 1 / (2 lambda |d|^2)
      gA[k] = in_reach ? jl / ((k & 1 ? 4.f : 2.f) * lam[k]) : 0.f;
    }
    float gC[3], gP[3];
    solve_scales_vjp(C11, C12, C22, scale_of_order(NF), gA, gC);
    if (kind == BSF_COV_LOGSIG_THETA_LOGRHO) {
      log_params_vjp(lc, gC, gP);
    } else {
      gP[0] = gC[0]; gP[1] = gC[1]; gP[2] = gC[2];
    }
    if constexpr (MODE == kOutJac) {
#pragma unroll
      for (int c = 0; c < 3; ++c) jac[c * jac_plane + (long long)y * ldj + x] = gP[c];
    } else {
      const float g = gout[(long long)(row0 + y) * ldg + x];
#pragma unroll
      for (int c = 0; c < 3; ++c) jac[c * jac_plane + (long long)y * ldj + x] = g * gP[c];
    }
  }
}

}  // namespace bsf_d2
