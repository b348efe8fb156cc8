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
#include "bsf_grid_box_spline.h"
#include "bsf_stencil.cuh"

namespace {

template <typename T, typename Out>
__global__ void __launch_bounds__(256, 2)
k_stencil_sampled(const T* __restrict__ S, long long pitch, int R, const float* __restrict__ cov, int kind,
                  int H, int W, int row0, int rows, float scale_f, double scale_d, Out* __restrict__ out,
                  long long ldo, DevStatus* st) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= rows) return;
  const long long HW = (long long)H * W, i = (long long)(row0 + y) * W + x;
  float C11, C12, C22;
  bsf_solve::load_cov(cov, kind, HW, i, C11, C12, C22);
  int Lq[4], flags, reach;
  const bool in_reach = bsf_solve::pixel_steps_sampled(C11, C12, C22, R, Lq, flags, reach);
  count_pixel_flags(flags, in_reach, st);

  const int p32 = (int)pitch;
  // the pixel in units of 2^-10 of the padded frame
  const int X0 = (x + R) << 10, Y0 = (y + R) << 10;
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
    const int par = __popc(t) & 1;
    acc = par ? acc - f : acc + f;
  }

  // mass prod Lq (exact in 128 bits) and the bound |acc| <= 2^-13 prod Lq max|Q|
  const u128 M = (u128)(unsigned)Lq[0] * (unsigned)Lq[1] * (u128)((unsigned long long)(unsigned)Lq[2] * (unsigned)Lq[3]);
  const float Mf = (float)Lq[0] * (float)Lq[1] * (float)Lq[2] * (float)Lq[3] * 0x1p-13f;
  const float maxq = __uint_as_float(st->max_absq_bits) + 1.f;
  if (maxq * Mf * 1.0001f >= bsf_pow2_f32(ElemBits<T>::value - 1)) {
    atomicAdd(&st->overflow_count, 1u);
    bsf_set_error(st, BSF_EOVERFLOW);
  }
  Out* o = out + (long long)y * ldo + x;
  if constexpr (sizeof(Out) == 4) {
    const float xa = __fmul_rn(to_f32<T>(acc, acc), scale_f);
    *o = __fdiv_rn(xa, bsf_rn32_u(M));
  } else {
    const double xa = __dmul_rn(to_f64<T>(acc), scale_d);
    *o = __ddiv_rn(xa, bsf_rn64_u(M));
  }
}

template <typename T>
cudaError_t launch_sampled_t(const T* S, long long pitch, int R, const float* cov, int kind, int H, int W,
                             int row0, int rows, int q, void* out, int out_dtype, long long ldo, DevStatus* st,
                             cudaStream_t s) {
  dim3 block(32, 8);
  dim3 grid((W + 31) / 32, (rows + 7) / 8);
  // 2^(13 - q) with q <= 100: normal in float32
  const float sf = ldexpf(1.f, 13 - q);
  const double sd = ldexp(1.0, 13 - q);
  if (out_dtype == BSF_F32)
    k_stencil_sampled<T, float><<<grid, block, 0, s>>>(S, pitch, R, cov, kind, H, W, row0, rows, sf, sd,
                                                       (float*)out, ldo, st);
  else if (out_dtype == BSF_F64)
    k_stencil_sampled<T, double><<<grid, block, 0, s>>>(S, pitch, R, cov, kind, H, W, row0, rows, sf, sd,
                                                        (double*)out, ldo, st);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace

cudaError_t bsf_launch_stencil_sampled(int prec, const void* S, long long pitch, int R, const float* cov,
                                       int cov_kind, int H, int W, int row0, int rows, int q, void* out,
                                       int out_dtype, long long ldo, DevStatus* st, cudaStream_t s) {
  if (prec == BSF_FIX64)
    return launch_sampled_t<uint64_t>((const uint64_t*)S, pitch, R, cov, cov_kind, H, W, row0, rows, q, out,
                                      out_dtype, ldo, st, s);
  if (prec == BSF_FIX128)
    return launch_sampled_t<u128>((const u128*)S, pitch, R, cov, cov_kind, H, W, row0, rows, q, out, out_dtype,
                                  ldo, st, s);
  return cudaErrorInvalidValue;
}
