// Per-pixel finite differences on the running sums (Section 1.1: the 16-tap
// finite-difference mesh of the BoxFilter algorithm, generalised to order n,
// whose mesh grows to (n+1)^4 taps -- Section 2.1 counts 2^N points per
// order, two per box distribution).
//
// For pixel p with integer steps L_k and centring c_k = n (L_k - 1)/2:
//   acc = sum_{t in {0..n}^4} prod_k (-1)^t_k C(n, t_k) S(p + sum_k (c_k - t_k L_k) d_k)
// evaluated exactly modulo 2^b as the nested order-n backward differences
// along d1, d2, d3, d4 (innermost first), then
//   out = RN32(RN32(acc) 2^-q) / RN32(D)  or  RN64(RN64(acc) 2^-q) / RN64(D),
//   D = prod_k L_k^n.
// One thread per output pixel; a warp covers 32 consecutive pixels of a row,
// so each tap is a coalesced row segment of S whenever neighbouring pixels
// share their steps (the covariance field is smooth).  The second direction
// set of Section 2.3 (Table 1's mesh of Algorithm 3) is the same stencil
// along e1 = (2,1), e2 = (1,2), e3 = (-1,2), e4 = (-2,1).
//
// Shared by the kernels of bsf_stencil.cu (first direction set, batches) and
// bsf_stencil_second.cu (second set, and the pair of Algorithm 2).
#pragma once

#include <type_traits>

#include "bsf_solve.cuh"

namespace {

// Order 2 in exact modular arithmetic, summed by coefficient: the tap
// t = (t1..t4) in {0,1,2}^4 carries prod_k (1, -2, 1)[t_k] = (-2)^j, j the
// number of t_k equal to 1, so the 81 taps go into five sums G_j (16, 32,
// 24, 8 and 1 taps) and acc = G0 - 2 (G1 - 2 (G2 - 2 (G3 - 2 G4))): 80 + 8
// additions against the nested form's 120, with the same result modulo 2^b.
// SH: 0 = global memory through the read-only path, 1 = shared memory,
// 2 = global memory by plain loads (data written earlier in the same launch).
template <typename T, int SH>
__device__ __forceinline__ T tap_load(const T* __restrict__ S, int i) {
  if constexpr (SH == 1) return S[i];
  else if constexpr (SH == 2) return bsf_load_weak(S + i);
  else return bsf_load(S + i);
}

template <typename T, int SH>
__device__ __forceinline__ T comb2_by_coefficient(const T* __restrict__ S, int idx, const int* s) {
  T G[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) G[j] = 0;
#pragma unroll
  for (int t4 = 0; t4 < 3; ++t4)
#pragma unroll
    for (int t3 = 0; t3 < 3; ++t3)
#pragma unroll
      for (int t2 = 0; t2 < 3; ++t2)
#pragma unroll
        for (int t1 = 0; t1 < 3; ++t1) {
          const int i = idx - t1 * s[0] - t2 * s[1] - t3 * s[2] - t4 * s[3];
          G[(t1 == 1) + (t2 == 1) + (t3 == 1) + (t4 == 1)] += tap_load<T, SH>(S, i);
        }
  T a = G[4];
#pragma unroll
  for (int j = 3; j >= 0; --j) a = G[j] - (a + a);
  return a;
}

// Nested order-n differences.  Taps are addressed by 32-bit element indices
// into S (the padded domain holds fewer than 2^31 elements); level LVL applies
// the difference along direction LVL-1 (stride s[LVL-1] elements) to level
// LVL-1, and level 0 loads one element.  Order 2 on the integer element
// types takes the grouped form above.
// SH: where S lies and how it is loaded (tap_load).
template <typename T, int NF, int LVL, int SH = 0>
__device__ __forceinline__ T comb(const T* __restrict__ S, int idx, const int* s) {
  if constexpr (LVL == 4 && NF == 2 && IsFixed<T>::value) {
    return comb2_by_coefficient<T, SH>(S, idx, s);
  } else if constexpr (LVL == 0) {
    return tap_load<T, SH>(S, idx);
  } else {
    const int sk = s[LVL - 1];
    const T v0 = comb<T, NF, LVL - 1, SH>(S, idx, s);
    const T v1 = comb<T, NF, LVL - 1, SH>(S, idx - sk, s);
    if constexpr (NF == 1) {
      return v0 - v1;
    } else if constexpr (NF == 2) {
      const T v2 = comb<T, NF, LVL - 1, SH>(S, idx - 2 * sk, s);
      return (v0 + v2) - (v1 + v1);
    } else {
      const T v2 = comb<T, NF, LVL - 1, SH>(S, idx - 2 * sk, s);
      const T v3 = comb<T, NF, LVL - 1, SH>(S, idx - 3 * sk, s);
      const T a = v1 - v2;
      return (v0 - v3) - (a + a + a);
    }
  }
}

template <typename T> __device__ __forceinline__ float to_f32(T acc, T D);
template <> __device__ __forceinline__ float to_f32<uint32_t>(uint32_t acc, uint32_t D) {
  (void)D;
  return __int2float_rn((int)acc);
}
template <> __device__ __forceinline__ float to_f32<uint64_t>(uint64_t acc, uint64_t D) {
  (void)D;
  return bsf_rn32_i64((long long)acc);
}
template <> __device__ __forceinline__ float to_f32<u128>(u128 acc, u128 D) {
  (void)D;
  return bsf_rn32((i128)acc);
}
template <typename T> __device__ __forceinline__ double to_f64(T acc);
template <> __device__ __forceinline__ double to_f64<uint32_t>(uint32_t acc) { return (double)(int)acc; }
template <> __device__ __forceinline__ double to_f64<uint64_t>(uint64_t acc) {
  return __ll2double_rn((long long)acc);
}
template <> __device__ __forceinline__ double to_f64<u128>(u128 acc) { return bsf_rn64((i128)acc); }

template <typename T> __device__ __forceinline__ float mass_f32(T D);
template <> __device__ __forceinline__ float mass_f32<uint32_t>(uint32_t D) { return __uint2float_rn(D); }
template <> __device__ __forceinline__ float mass_f32<uint64_t>(uint64_t D) { return bsf_rn32_u64(D); }
template <> __device__ __forceinline__ float mass_f32<u128>(u128 D) { return bsf_rn32_u(D); }
template <typename T> __device__ __forceinline__ double mass_f64(T D);
template <> __device__ __forceinline__ double mass_f64<uint32_t>(uint32_t D) { return (double)D; }
template <> __device__ __forceinline__ double mass_f64<uint64_t>(uint64_t D) { return __ull2double_rn(D); }
template <> __device__ __forceinline__ double mass_f64<u128>(u128 D) { return bsf_rn64_u(D); }

// Resident blocks per SM requested from the register allocator: enough warps
// to cover the latency of the (n+1)^4 gathers.
template <typename T, int NF> struct StencilOcc {
  static constexpr int value = sizeof(T) <= 8 ? (NF == 1 ? 6 : NF == 2 ? 4 : 1) : (NF == 1 ? 4 : NF == 2 ? 2 : 1);
};

// Rare-event counters of the step solve (clamped, non-finite, out of
// reach), aggregated over the active lanes of the warp.
__device__ __forceinline__ void count_pixel_flags(int flags, bool in_reach, DevStatus* st) {
  const unsigned act = __activemask();
  const unsigned mc = __ballot_sync(act, flags & 1), mb = __ballot_sync(act, flags & 2),
                 mr = __ballot_sync(act, !in_reach);
  if ((mc | mb | mr) && (threadIdx.x & 31) == __ffs(act) - 1) {
    if (mc) atomicAdd(&st->clamp_count, (unsigned)__popc(mc));
    if (mb) { atomicAdd(&st->bad_count, (unsigned)__popc(mb)); bsf_set_error(st, BSF_ECOV); }
    if (mr) { atomicAdd(&st->range_count, (unsigned)__popc(mr)); bsf_set_error(st, BSF_ERANGE); }
  }
}

// The output rule of one pixel from its exact accumulator: D = prod_k L_k^n
// and out = RN(RN(acc) 2^-q) / RN(D) (fixed point), or acc / D (floating-
// point variants).  maxq bounds max|Q| + 1 over the kernel's support: the
// bound max|Q| * D < 2^(b-1), which makes the modular accumulator equal the
// true one, is checked in float32 with a margin far above its rounding
// (|acc| <= D max|Q|).
template <typename T, int NF, typename Out>
__device__ __forceinline__ void finish_pixel(T acc, const int* L, float maxq, float scale_f, double scale_d,
                                             Out* __restrict__ o, DevStatus* st) {
  const int L1 = L[0], L2 = L[1], L3 = L[2], L4w = L[3];
  if constexpr (IsFixed<T>::value) {
    T D = 1;
    const T D1 = (T)(unsigned)(L1 * L2) * (T)(unsigned)(L3 * L4w);
    const float Df1 = (float)(L1 * L2) * (float)(L3 * L4w);
    float Df = Df1;
#pragma unroll
    for (int j = 0; j < NF; ++j) D *= D1;
#pragma unroll
    for (int j = 1; j < NF; ++j) Df *= Df1;
    const float lim = bsf_pow2_f32(ElemBits<T>::value - 1);
    if (maxq * Df * 1.0001f >= lim) {
      atomicAdd(&st->overflow_count, 1u);
      bsf_set_error(st, BSF_EOVERFLOW);
    }
    if constexpr (sizeof(Out) == 4) {
      const float xa = __fmul_rn(to_f32<T>(acc, D), scale_f);
      *o = __fdiv_rn(xa, mass_f32<T>(D));
    } else {
      const double xa = __dmul_rn(to_f64<T>(acc), scale_d);
      *o = __ddiv_rn(xa, mass_f64<T>(D));
    }
  } else {
    // floating-point precision variants: acc / prod L^n
    double Dd = 1.0;
    const double D1 = (double)(L1 * L2) * (double)(L3 * L4w);
#pragma unroll
    for (int j = 0; j < NF; ++j) Dd *= D1;
    double a;
    if constexpr (std::is_same<T, double>::value) a = acc;
    else a = (double)acc.hi + (double)acc.lo;
    const double v = a / Dd;
    if constexpr (sizeof(Out) == 4) *o = __double2float_rn(v);
    else *o = v;
  }
}

// The step solve of bsf_solve.cuh runs here, per pixel, so its arithmetic
// overlaps the gathers of other warps and no step field goes through HBM.
// DS (BSF_DIRS_*): the direction set.  BSF_DIRS_CARTESIAN takes the taps
// from S along d1..d4; BSF_DIRS_SECOND from S along e1 = (2,1), e2 = (1,2),
// e3 = (-1,2), e4 = (-2,1); BSF_DIRS_PAIR chooses per pixel between S
// (Cartesian running sums) and S2 (running sums of the second set), which
// share one pitch.
// LD: the load mode of the taps (tap_load); (tx, ty) the thread's place in a
// block of 32 x bdy pixels (default: the launch's thread indices).
template <typename T, int NF, typename Out, int DS = BSF_DIRS_CARTESIAN, int LD = 0>
__device__ __forceinline__ void stencil_d1_body(const T* __restrict__ S, const T* __restrict__ S2,
                                                long long pitch, int R,
                                                const float* __restrict__ cov, int kind, int rule, int H,
                                                int W, int row0, int rows, float scale_f,
                                                double scale_d, Out* __restrict__ out,
                                                long long ldo, DevStatus* st, int bx, int by,
                                                int tx = -1, int ty = 0, int bdy = 0) {
  // pixel (x, row0 + y) of an H x W image; rows [row0, row0 + rows) are
  // filtered from running sums whose padded row 0 is image row row0 - R
  if (tx < 0) {
    tx = threadIdx.x;
    ty = threadIdx.y;
    bdy = blockDim.y;
  }
  const int x = bx * 32 + tx;
  const int y = by * bdy + ty;
  if (x >= W || y >= rows) return;
  const long long HW = (long long)H * W, i = (long long)(row0 + y) * W + x;
  int L[4], flags, reach;
  float C11, C12, C22;
  bsf_solve::load_cov(cov, kind, HW, i, C11, C12, C22);
  bool second = false;
  bool in_reach;
  if constexpr (DS == BSF_DIRS_CARTESIAN)
    in_reach = bsf_solve::pixel_steps(C11, C12, C22, NF, rule, R, L, flags, reach);
  else
    in_reach = bsf_solve::pixel_steps_set(DS, C11, C12, C22, NF, rule, R, L, flags, reach, second);
  count_pixel_flags(flags, in_reach, st);
  // the step solve above reads only the field; the running sums may still be
  // in the making when this kernel was launched as a programmatic dependent
  bsf_grid_dep_wait();
  const int L1 = L[0], L2 = L[1], L3 = L[2], L4w = L[3];
  // element strides of d1 = (1,0), d2 = (1,1), d3 = (0,1), d4 = (-1,1), or
  // of e1 = (2,1), e2 = (1,2), e3 = (-1,2), e4 = (-2,1)
  const int p32 = (int)pitch;
  int e1 = 1, e2 = p32 + 1, e3 = p32, e4 = p32 - 1;
  const T* Sp = S;
  if constexpr (DS != BSF_DIRS_CARTESIAN) {
    if (second) {
      e1 = p32 + 2; e2 = 2 * p32 + 1; e3 = 2 * p32 - 1; e4 = p32 - 2;
      if constexpr (DS == BSF_DIRS_PAIR) Sp = S2;
    }
  }
  const int c1 = NF * (L1 - 1) / 2, c2 = NF * (L2 - 1) / 2, c3 = NF * (L3 - 1) / 2,
            c4 = NF * (L4w - 1) / 2;
  const int base = (y + R) * p32 + (x + R) + c1 * e1 + c2 * e2 + c3 * e3 + c4 * e4;
  const int s[4] = {L1 * e1, L2 * e2, L3 * e3, L4w * e4};
  const T acc = comb<T, NF, 4, LD>(Sp, base, s);
  finish_pixel<T, NF, Out>(acc, L, __uint_as_float(st->max_absq_bits) + 1.f, scale_f, scale_d,
                           out + (long long)(y) * ldo + x, st);
}

}  // namespace
