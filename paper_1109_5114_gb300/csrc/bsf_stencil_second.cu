// Stencil kernels of the second direction set (BSF_DIRS_SECOND: Algorithm 3's
// beta'_a with integer steps) and of the pair switched per pixel by sector
// (BSF_DIRS_PAIR: Algorithm 2).  Fixed point only (32, 64 and 128 bits).
#include "bsf_stencil.cuh"

namespace {

template <typename T, int NF, typename Out, int DS>
__global__ void __launch_bounds__(256, (StencilOcc<T, NF>::value))
k_stencil_sets(const T* __restrict__ S, const T* __restrict__ S2, long long pitch, int R,
               const float* __restrict__ cov, int kind, int rule, int H, int W, int row0, int rows,
               float scale_f, double scale_d, Out* __restrict__ out, long long ldo, DevStatus* st) {
  stencil_d1_body<T, NF, Out, DS>(S, S2, pitch, R, cov, kind, rule, H, W, row0, rows, scale_f, scale_d,
                                  out, ldo, st, blockIdx.x, blockIdx.y);
}

template <typename T, int NF, int DS>
cudaError_t launch_sets(const T* S, const T* S2, long long pitch, int R, const float* cov, int kind,
                        int rule, int H, int W, int row0, int rows, int q, void* out, int out_dtype,
                        long long ldo, DevStatus* st, cudaStream_t s) {
  dim3 block(32, 8);
  dim3 grid((W + 31) / 32, (rows + 7) / 8);
  const float sf = ldexpf(1.f, -q);
  const double sd = ldexp(1.0, -q);
  if (out_dtype == BSF_F32)
    k_stencil_sets<T, NF, float, DS><<<grid, block, 0, s>>>(S, S2, pitch, R, cov, kind, rule, H, W, row0,
                                                            rows, sf, sd, (float*)out, ldo, st);
  else if (out_dtype == BSF_F64)
    k_stencil_sets<T, NF, double, DS><<<grid, block, 0, s>>>(S, S2, pitch, R, cov, kind, rule, H, W, row0,
                                                             rows, sf, sd, (double*)out, ldo, st);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T, int DS>
cudaError_t launch_sets_n(int n, const void* S, const void* S2, long long pitch, int R, const float* cov,
                          int kind, int rule, int H, int W, int row0, int rows, int q, void* out,
                          int out_dtype, long long ldo, DevStatus* st, cudaStream_t s) {
  const T* a = (const T*)S;
  const T* b = (const T*)S2;
  switch (n) {
    case 1: return launch_sets<T, 1, DS>(a, b, pitch, R, cov, kind, rule, H, W, row0, rows, q, out, out_dtype, ldo, st, s);
    case 2: return launch_sets<T, 2, DS>(a, b, pitch, R, cov, kind, rule, H, W, row0, rows, q, out, out_dtype, ldo, st, s);
    case 3: return launch_sets<T, 3, DS>(a, b, pitch, R, cov, kind, rule, H, W, row0, rows, q, out, out_dtype, ldo, st, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t bsf_launch_stencil_sets(int prec, int n, int dirset, const void* S, const void* S2,
                                    long long pitch, int R, const float* cov, int cov_kind, int rule,
                                    int H, int W, int row0, int rows, int q, void* out, int out_dtype,
                                    long long ldo, DevStatus* st, cudaStream_t s) {
  if (dirset == BSF_DIRS_PAIR && !S2) return cudaErrorInvalidValue;
  if (prec == BSF_FIX32) {
    if (dirset == BSF_DIRS_SECOND)
      return launch_sets_n<uint32_t, BSF_DIRS_SECOND>(n, S, S2, pitch, R, cov, cov_kind, rule, H, W, row0, rows, q, out, out_dtype, ldo, st, s);
    if (dirset == BSF_DIRS_PAIR)
      return launch_sets_n<uint32_t, BSF_DIRS_PAIR>(n, S, S2, pitch, R, cov, cov_kind, rule, H, W, row0, rows, q, out, out_dtype, ldo, st, s);
  } else if (prec == BSF_FIX64) {
    if (dirset == BSF_DIRS_SECOND)
      return launch_sets_n<uint64_t, BSF_DIRS_SECOND>(n, S, S2, pitch, R, cov, cov_kind, rule, H, W, row0, rows, q, out, out_dtype, ldo, st, s);
    if (dirset == BSF_DIRS_PAIR)
      return launch_sets_n<uint64_t, BSF_DIRS_PAIR>(n, S, S2, pitch, R, cov, cov_kind, rule, H, W, row0, rows, q, out, out_dtype, ldo, st, s);
  } else if (prec == BSF_FIX128) {
    if (dirset == BSF_DIRS_SECOND)
      return launch_sets_n<u128, BSF_DIRS_SECOND>(n, S, S2, pitch, R, cov, cov_kind, rule, H, W, row0, rows, q, out, out_dtype, ldo, st, s);
    if (dirset == BSF_DIRS_PAIR)
      return launch_sets_n<u128, BSF_DIRS_PAIR>(n, S, S2, pitch, R, cov, cov_kind, rule, H, W, row0, rows, q, out, out_dtype, ldo, st, s);
  }
  return cudaErrorInvalidValue;
}
