// Continuous-step stencil instances for one element type of the running sums
// (split from the dispatcher so the instances compile in parallel).
#include "bsf_continuous.cuh"

namespace {

using namespace bsf_d2;

template <typename T, int NF, int MODE>
cudaError_t launch_d2(const T* S, long long pitch, int R, const float* cov, int kind, int H, int W,
                      int row0, int rows, int q, void* out, int out_dtype, long long ldo,
                      float* jac, long long ldj, long long jac_plane, const float* gout,
                      long long ldg, DevStatus* st, cudaStream_t s) {
  const dim3 block(32, 4);
  const dim3 grid((W + 31) / 32, (rows + 3) / 4);
  const float sf = ldexpf(1.f, -q);
  const double sd = ldexp(1.0, -q);
  if (out_dtype == BSF_F64) {  // float64 output: forward only
    if constexpr (MODE == kOut)
      k_stencil_d2<T, NF, double, MODE><<<grid, block, 0, s>>>(S, pitch, R, cov, kind, H, W, row0,
                                                              rows, sf, sd, (double*)out, ldo, jac,
                                                              ldj, jac_plane, gout, ldg, st);
    else
      return cudaErrorInvalidValue;
  } else
    k_stencil_d2<T, NF, float, MODE><<<grid, block, 0, s>>>(S, pitch, R, cov, kind, H, W, row0, rows,
                                                           sf, sd, (float*)out, ldo, jac, ldj,
                                                           jac_plane, gout, ldg, st);
  return cudaGetLastError();
}

template <typename T, int NF>
cudaError_t launch_mode(int mode, const void* S, long long pitch, int R, const float* cov, int kind,
                        int H, int W, int row0, int rows, int q, void* out, int out_dtype,
                        long long ldo, float* jac, long long ldj, long long jac_plane,
                        const float* gout, long long ldg, DevStatus* st, cudaStream_t s) {
  const T* St = (const T*)S;
  if (mode == kOut)
    return launch_d2<T, NF, kOut>(St, pitch, R, cov, kind, H, W, row0, rows, q, out, out_dtype, ldo,
                                  jac, ldj, jac_plane, gout, ldg, st, s);
  if (mode == kOutJac)
    return launch_d2<T, NF, kOutJac>(St, pitch, R, cov, kind, H, W, row0, rows, q, out, out_dtype,
                                     ldo, jac, ldj, jac_plane, gout, ldg, st, s);
  return launch_d2<T, NF, kVjp>(St, pitch, R, cov, kind, H, W, row0, rows, q, out, BSF_F32, ldo,
                                jac, ldj, jac_plane, gout, ldg, st, s);
}

}  // namespace

cudaError_t bsf_launch_stencil_d2_u128(int n, int mode, const void* S, long long pitch, int R, const float* cov,
                  int cov_kind, int H, int W, int row0, int rows, int q, void* out, int out_dtype,
                  long long ldo, float* jac, long long ldj, long long jac_plane, const float* gout,
                  long long ldg, DevStatus* st, cudaStream_t s) {
  if (n == 1)
    return launch_mode<u128, 1>(mode, S, pitch, R, cov, cov_kind, H, W, row0, rows, q, out,
                                out_dtype, ldo, jac, ldj, jac_plane, gout, ldg, st, s);
  if (n == 2)
    return launch_mode<u128, 2>(mode, S, pitch, R, cov, cov_kind, H, W, row0, rows, q, out,
                                out_dtype, ldo, jac, ldj, jac_plane, gout, ldg, st, s);
  return cudaErrorInvalidValue;
}
