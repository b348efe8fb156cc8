// The sampled continuous box spline (BSF_STEP_SAMPLED, order 1): the taps of
// the 16-point mesh at continuous offsets (1/2 - t_k) lambda_k d_k, the
// running sums interpolated there by the grid box spline beta_b of unit steps
// (Section 2.3, eq. "interpolation", for the Cartesian set), then the
// order-1 differences:
//   out(p) = (1 / prod lambda) sum_t (-1)^|t| sum_m S(m) beta_b(p + o_t - m),
// which is sum_m f(m) beta_a(p + tau - m), the continuous box spline beta_a
// (boxes of lambda_k steps along d_k) sampled at the grid.
//
// lambda_k = a_k / |d_k| from the minimum-kurtosis scales (the continuous
// beta_a has covariance C exactly), quantised to Lq_k = max(1, RNE(512
// lambda_k)).  Every tap then lies on the grid of 2^-10; the nine samples
// around it get integer weights beta_b * 2^23 (bsf_grid_box_spline.h), so
//   acc = sum_t (-1)^|t| sum_samples w S   (exact, modulo 2^b),
//   out = RN(RN(acc) 2^(13 - q)) / RN(prod Lq)
// since prod lambda = prod Lq / 2^36.  |acc| <= 2^23 prod lambda max|Q|,
// the bound the mass prod Lq 2^-13 enters.
//
// The second set (Algorithm 3 as printed: beta'_a, the running sums along
// e1 = (2,1), e2 = (1,2), e3 = (-1,2), e4 = (-2,1) interpolated by beta'_b):
// lambda_k = a_k / sqrt(5) quantised to Lq = max(1, RNE(32 lambda)), the taps
// on the grid of 2^-6, the samples of a 6 x 6 block per tap weighted by
// beta'_b * 491520 (bsf_knight_box_spline.h), out = RN(RN(acc) 2^(5 - q)) /
// RN(15 prod Lq).  The pair chooses per pixel by sector.
#include "bsf_grid_box_spline.h"
#include "bsf_knight_box_spline.h"
#include "bsf_stencil.cuh"

namespace {

// Cartesian set: the 16 taps on the 2^-10 grid, nine samples each.
template <typename T>
__device__ __forceinline__ T sampled_acc(const T* __restrict__ S, int p32, int x, int y, int R, const int Lq[4]) {
  const int X0 = (x + R) << 10, Y0 = (y + R) << 10;  // the pixel in units of 2^-10 of the padded frame
  T acc = (T)0;
#pragma unroll 2
  for (int t = 0; t < 16; ++t) {
    // offsets (1 - 2 t_k) Lq_k d_k (units of 2^-10) of d1 = (1,0),
    // d2 = (1,1), d3 = (0,1), d4 = (-1,1)
    const int o1 = (t & 1) ? -Lq[0] : Lq[0], o2 = (t & 2) ? -Lq[1] : Lq[1];
    const int o3 = (t & 4) ? -Lq[2] : Lq[2], o4 = (t & 8) ? -Lq[3] : Lq[3];
    const int Zx = X0 + o1 + o2 - o4, Zy = Y0 + o2 + o3 + o4;
    const int U = Zx & 1023, V = Zy & 1023;
    const int tri = V <= U ? (U + V <= 1024 ? 0 : 1) : (U + V >= 1024 ? 2 : 3);
    int w[9];
    grid_box_spline_weights(tri, U, V, w);
    // samples (zx + i1, zy + i2), i1 in {-1, 0, 1}, i2 in {-2, -1, 0}
    const int base = (Zy >> 10) * p32 + (Zx >> 10);
    T f = (T)0;
#pragma unroll
    for (int i1 = -1; i1 <= 1; ++i1)
#pragma unroll
      for (int i2 = -2; i2 <= 0; ++i2)
        f += (T)(unsigned)w[(i1 + 1) * 3 + (i2 + 2)] * bsf_load(S + base + i2 * p32 + i1);
    acc = (__popc(t) & 1) ? acc - f : acc + f;
  }
  return acc;
}

// Second set: the 16 taps on the 2^-6 grid, the samples of a 6 x 6 block
// around each (beta'_b lies within [-3, 3] x [0, 6] of a sample), weighted
// by the table of beta'_b * 491520 folded by its symmetries.
template <typename T>
__device__ __forceinline__ T sampled_acc_k(const T* __restrict__ S, int p32, int x, int y, int R, const int Lq[4]) {
  const int X0 = (x + R) << 6, Y0 = (y + R) << 6;  // units of 2^-6
  T acc = (T)0;
#pragma unroll 1
  for (int t = 0; t < 16; ++t) {
    // offsets (1 - 2 t_k) Lq_k e_k (units of 2^-6) of e1 = (2,1), e2 = (1,2),
    // e3 = (-1,2), e4 = (-2,1)
    const int o1 = (t & 1) ? -Lq[0] : Lq[0], o2 = (t & 2) ? -Lq[1] : Lq[1];
    const int o3 = (t & 4) ? -Lq[2] : Lq[2], o4 = (t & 8) ? -Lq[3] : Lq[3];
    const int Zx = X0 + 2 * o1 + o2 - o3 - 2 * o4, Zy = Y0 + o1 + 2 * o2 + 2 * o3 + o4;
    const int U = Zx & 63, V = Zy & 63;
    const int base = (Zy >> 6) * p32 + (Zx >> 6);
    T f = (T)0;
    // sample (zx + i1, zy + i2): offset from beta'_b's centre (0, 3), units
    // of 2^-6: (U - 64 i1, V - 64 i2 - 192)
#pragma unroll
    for (int i2 = -5; i2 <= 0; ++i2) {
      const int b2 = V - 64 * i2 - 192;
#pragma unroll
      for (int i1 = -2; i1 <= 3; ++i1) {
        const int b1 = U - 64 * i1;
        const int ax = b1 < 0 ? -b1 : b1, ay = b2 < 0 ? -b2 : b2;
        const int a = ax > ay ? ax : ay, b = ax > ay ? ay : ax;
        if (a <= 192) {
          const int w = __ldg(&kKnightBoxSpline[a * (a + 1) / 2 + b]);
          if (w) f += (T)(unsigned)w * bsf_load(S + base + i2 * p32 + i1);
        }
      }
    }
    acc = (__popc(t) & 1) ? acc - f : acc + f;
  }
  return acc;
}

// DS (BSF_DIRS_*): the Cartesian set on S, the second set on S, or the pair
// (S Cartesian, S2 the second set's sums), chosen per pixel by sector.
template <typename T, typename Out, int DS>
__global__ void __launch_bounds__(256, 2)
k_stencil_sampled(const T* __restrict__ S, const T* __restrict__ S2, long long pitch, int R,
                  const float* __restrict__ cov, int kind, int H, int W, int row0, int rows, int q,
                  Out* __restrict__ out, long long ldo, DevStatus* st) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= rows) return;
  const long long HW = (long long)H * W, i = (long long)(row0 + y) * W + x;
  float C11, C12, C22;
  bsf_solve::load_cov(cov, kind, HW, i, C11, C12, C22);
  const bool second = DS == BSF_DIRS_SECOND ||
                      (DS == BSF_DIRS_PAIR && bsf_solve::use_second_set(C11, C12, C22));
  int Lq[4], flags, reach;
  const bool in_reach = second ? bsf_solve::pixel_steps_sampled_k(C11, C12, C22, R, Lq, flags, reach)
                               : bsf_solve::pixel_steps_sampled(C11, C12, C22, R, Lq, flags, reach);
  count_pixel_flags(flags, in_reach, st);
  const int p32 = (int)pitch;
  T acc;
  int e;       // out = RN(RN(acc) 2^(e - q)) / RN(M)
  u128 M;      // Cartesian: prod Lq, e = 13; second set: 15 prod Lq, e = 5
  if (DS == BSF_DIRS_CARTESIAN || !second) {
    acc = sampled_acc<T>(S, p32, x, y, R, Lq);
    e = 13;
    M = 1;
  } else {
    acc = sampled_acc_k<T>(DS == BSF_DIRS_PAIR ? S2 : S, p32, x, y, R, Lq);
    e = 5;
    M = 15;
  }
  M *= (u128)(unsigned)Lq[0] * (unsigned)Lq[1] * (u128)((unsigned long long)(unsigned)Lq[2] * (unsigned)Lq[3]);
  // the bound |acc| <= M 2^-e max|Q| (the weights' sum times prod lambda)
  const float Mf = bsf_rn32_u(M) * bsf_pow2_f32(-e);
  const float maxq = __uint_as_float(st->max_absq_bits) + 1.f;
  if (maxq * Mf * 1.0001f >= bsf_pow2_f32(ElemBits<T>::value - 1)) {
    atomicAdd(&st->overflow_count, 1u);
    bsf_set_error(st, BSF_EOVERFLOW);
  }
  Out* o = out + (long long)y * ldo + x;
  if constexpr (sizeof(Out) == 4) {
    const float xa = __fmul_rn(to_f32<T>(acc, acc), bsf_pow2_f32(e - q));  // q <= 100: normal
    *o = __fdiv_rn(xa, bsf_rn32_u(M));
  } else {
    const double xa = __dmul_rn(to_f64<T>(acc), ldexp(1.0, e - q));
    *o = __ddiv_rn(xa, bsf_rn64_u(M));
  }
}

template <typename T, int DS>
cudaError_t launch_sampled_t(const T* S, const T* S2, long long pitch, int R, const float* cov, int kind, int H,
                             int W, int row0, int rows, int q, void* out, int out_dtype, long long ldo,
                             DevStatus* st, cudaStream_t s) {
  dim3 block(32, 8);
  dim3 grid((W + 31) / 32, (rows + 7) / 8);
  if (out_dtype == BSF_F32)
    k_stencil_sampled<T, float, DS><<<grid, block, 0, s>>>(S, S2, pitch, R, cov, kind, H, W, row0, rows, q,
                                                           (float*)out, ldo, st);
  else if (out_dtype == BSF_F64)
    k_stencil_sampled<T, double, DS><<<grid, block, 0, s>>>(S, S2, pitch, R, cov, kind, H, W, row0, rows, q,
                                                            (double*)out, ldo, st);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sampled_d(int dirset, const void* S, const void* S2, long long pitch, int R, const float* cov,
                             int kind, int H, int W, int row0, int rows, int q, void* out, int out_dtype,
                             long long ldo, DevStatus* st, cudaStream_t s) {
  const T* a = (const T*)S;
  const T* b = (const T*)S2;
  switch (dirset) {
    case BSF_DIRS_CARTESIAN:
      return launch_sampled_t<T, BSF_DIRS_CARTESIAN>(a, b, pitch, R, cov, kind, H, W, row0, rows, q, out, out_dtype,
                                                     ldo, st, s);
    case BSF_DIRS_SECOND:
      return launch_sampled_t<T, BSF_DIRS_SECOND>(a, b, pitch, R, cov, kind, H, W, row0, rows, q, out, out_dtype,
                                                  ldo, st, s);
    case BSF_DIRS_PAIR:
      if (!S2) return cudaErrorInvalidValue;
      return launch_sampled_t<T, BSF_DIRS_PAIR>(a, b, pitch, R, cov, kind, H, W, row0, rows, q, out, out_dtype, ldo,
                                                st, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t bsf_launch_stencil_sampled(int prec, int dirset, const void* S, const void* S2, long long pitch, int R,
                                       const float* cov, int cov_kind, int H, int W, int row0, int rows, int q,
                                       void* out, int out_dtype, long long ldo, DevStatus* st, cudaStream_t s) {
  if (prec == BSF_FIX64)
    return launch_sampled_d<uint64_t>(dirset, S, S2, pitch, R, cov, cov_kind, H, W, row0, rows, q, out, out_dtype,
                                      ldo, st, s);
  if (prec == BSF_FIX128)
    return launch_sampled_d<u128>(dirset, S, S2, pitch, R, cov, cov_kind, H, W, row0, rows, q, out, out_dtype, ldo,
                                  st, s);
  return cudaErrorInvalidValue;
}
