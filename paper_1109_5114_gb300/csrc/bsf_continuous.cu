// Dispatch of the continuous-step stencil by element type, and the
// vector-Jacobian product kernel.  The stencil itself is in bsf_continuous.cuh.
#include "bsf_continuous.cuh"

cudaError_t bsf_launch_stencil_d2_u64(int n, int mode, const void* S, long long pitch, int R,
                                      const float* cov, int cov_kind, int H, int W, int row0,
                                      int rows, int q, void* out, int out_dtype, long long ldo,
                                      float* jac, long long ldj, long long jac_plane,
                                      const float* gout, long long ldg, DevStatus* st,
                                      cudaStream_t s);
cudaError_t bsf_launch_stencil_d2_u128(int n, int mode, const void* S, long long pitch, int R,
                                       const float* cov, int cov_kind, int H, int W, int row0,
                                       int rows, int q, void* out, int out_dtype, long long ldo,
                                       float* jac, long long ldj, long long jac_plane,
                                       const float* gout, long long ldg, DevStatus* st,
                                       cudaStream_t s);

namespace {

__global__ void k_jacobian_vjp(const float* __restrict__ gout, long long ldg,
                               const float* __restrict__ jac, long long ldj, float* __restrict__ gcov,
                               int H, int W) {
  const long long HW = (long long)H * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
       i += (long long)gridDim.x * blockDim.x) {
    const long long y = i / W, x = i - y * W;
    const float g = gout[y * ldg + x];
    const long long jp = (long long)H * ldj;
#pragma unroll
    for (int c = 0; c < 3; ++c) gcov[c * HW + i] = g * jac[c * jp + y * ldj + x];
  }
}

}  // namespace

cudaError_t bsf_launch_stencil_d2(int prec, int n, int mode, const void* S, long long pitch, int R,
                                  const float* cov, int cov_kind, int H, int W, int row0, int rows,
                                  int q, void* out, int out_dtype, long long ldo, float* jac,
                                  long long ldj, long long jac_plane, const float* gout,
                                  long long ldg, DevStatus* st, cudaStream_t s) {
  if (mode < bsf_d2::kOut || mode > bsf_d2::kVjp) return cudaErrorInvalidValue;
  if (out_dtype != BSF_F32 && out_dtype != BSF_F64) return cudaErrorInvalidValue;
  if (prec == BSF_FIX64)
    return bsf_launch_stencil_d2_u64(n, mode, S, pitch, R, cov, cov_kind, H, W, row0, rows, q, out,
                                     out_dtype, ldo, jac, ldj, jac_plane, gout, ldg, st, s);
  if (prec == BSF_FIX128)
    return bsf_launch_stencil_d2_u128(n, mode, S, pitch, R, cov, cov_kind, H, W, row0, rows, q, out,
                                      out_dtype, ldo, jac, ldj, jac_plane, gout, ldg, st, s);
  return cudaErrorInvalidValue;
}

cudaError_t bsf_launch_jacobian_vjp(const float* gout, long long ldg, const float* jac,
                                    long long ldj, float* gcov, int H, int W, cudaStream_t s) {
  const int threads = 256;
  long long blocks = ((long long)H * W + threads - 1) / threads;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  k_jacobian_vjp<<<(int)blocks, threads, 0, s>>>(gout, ldg, jac, ldj, gcov, H, W);
  return cudaGetLastError();
}
