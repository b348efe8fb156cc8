// Kernels of the integer-step filter with the Cartesian direction set: one
// image (k_stencil_d1) and batches (k_batch_stencil).  The stencil itself is
// in bsf_stencil.cuh.
#include "bsf_stencil.cuh"

namespace {

template <typename T, int NF, typename Out>
__global__ void __launch_bounds__(256, (StencilOcc<T, NF>::value))
k_stencil_d1(const T* __restrict__ S, long long pitch, int R, const float* __restrict__ cov,
             int kind, int rule, int H, int W, int row0, int rows, float scale_f, double scale_d,
             Out* __restrict__ out, long long ldo, DevStatus* st) {
  stencil_d1_body<T, NF, Out>(S, nullptr, pitch, R, cov, kind, rule, H, W, row0, rows, scale_f, scale_d,
                              out, ldo, st, blockIdx.x, blockIdx.y);
}

template <typename T, int NF>
cudaError_t launch_t(const T* S, long long pitch, int R, const float* cov, int kind, int rule, int H, int W,
                     int row0, int rows, int q, void* out, int out_dtype, long long ldo,
                     DevStatus* st, cudaStream_t s, bool pdl) {
  // 32 x 4 pixels per block (0.2167 against 0.2188 ms per 2048^2 step with
  // 32 x 8; 32 x 2 0.2171)
  dim3 block(32, 4);
  dim3 grid((W + 31) / 32, (rows + 3) / 4);
  const float sf = ldexpf(1.f, -q);
  const double sd = ldexp(1.0, -q);
  // pdl: launched as a programmatic dependent of the last running-sum kernel,
  // the kernel just before on the stream: its blocks solve their steps while
  // that kernel finishes, then wait for it before the gathers
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (out_dtype == BSF_F32)
    return cudaLaunchKernelEx(&cfg, k_stencil_d1<T, NF, float>, S, pitch, R, cov, kind, rule, H, W, row0, rows,
                              sf, sd, (float*)out, ldo, st);
  if (out_dtype == BSF_F64)
    return cudaLaunchKernelEx(&cfg, k_stencil_d1<T, NF, double>, S, pitch, R, cov, kind, rule, H, W, row0, rows,
                              sf, sd, (double*)out, ldo, st);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t bsf_launch_stencil_d1_ex(int prec, int n, const void* S, long long pitch, int R,
                                     const float* cov, int cov_kind, int rule, int H, int W, int row0, int rows,
                                     int q, void* out, int out_dtype, long long ldo, DevStatus* st,
                                     cudaStream_t s, bool after_scans) {
#define BSF_ST(T, NF)                                                                          \
  return launch_t<T, NF>((const T*)S, pitch, R, cov, cov_kind, rule, H, W, row0, rows, q, out, out_dtype, \
                         ldo, st, s, after_scans)
  switch (prec * 10 + n) {
    case 51: BSF_ST(uint32_t, 1);
    case 52: BSF_ST(uint32_t, 2);
    case 53: BSF_ST(uint32_t, 3);
    case 11: BSF_ST(uint64_t, 1);
    case 12: BSF_ST(uint64_t, 2);
    case 13: BSF_ST(uint64_t, 3);
    case 21: BSF_ST(u128, 1);
    case 22: BSF_ST(u128, 2);
    case 23: BSF_ST(u128, 3);
    case 31: BSF_ST(double, 1);
    case 32: BSF_ST(double, 2);
    case 33: BSF_ST(double, 3);
    case 41: BSF_ST(f32x2, 1);
    case 42: BSF_ST(f32x2, 2);
    case 43: BSF_ST(f32x2, 3);
    default: break;
  }
#undef BSF_ST
  return cudaErrorInvalidValue;
}

cudaError_t bsf_launch_stencil_d1(int prec, int n, const void* S, long long pitch, int R,
                                  const float* cov, int cov_kind, int rule, int H, int W, int row0, int rows,
                                  int q, void* out, int out_dtype, long long ldo, DevStatus* st,
                                  cudaStream_t s) {
  return bsf_launch_stencil_d1_ex(prec, n, S, pitch, R, cov, cov_kind, rule, H, W, row0, rows, q, out, out_dtype,
                                  ldo, st, s, false);
}

namespace {

__device__ __forceinline__ int batch_find_st(const int* __restrict__ starts, int B, int blk) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int NF, typename Out>
__global__ void __launch_bounds__(256, (StencilOcc<uint64_t, NF>::value))
k_batch_stencil(const BatchImage* __restrict__ imgs, const int* __restrict__ starts, int B, int rule,
                float scale_f, double scale_d, DevStatus* st) {
  const int i = batch_find_st(starts, B, blockIdx.x);
  const BatchImage& im = imgs[i];
  const int local = blockIdx.x - starts[i];
  const int gx = (im.W + 31) / 32;
  stencil_d1_body<uint64_t, NF, Out>((const uint64_t*)im.S, nullptr, im.pitch, im.R, im.cov, BSF_COV_C,
                                     rule, im.H, im.W, 0, im.H, scale_f, scale_d, (Out*)im.out, im.ldo,
                                     st, local % gx, local / gx);
}

}  // namespace

cudaError_t bsf_launch_batch_stencil(int n, int out_dtype, const BatchImage* imgs, const int* starts,
                                     int B, int total, int rule, int q, DevStatus* st,
                                     cudaStream_t s) {
  const dim3 block(32, 8);
  const float sf = ldexpf(1.f, -q);
  const double sd = ldexp(1.0, -q);
#define BSF_BS(NF, O) k_batch_stencil<NF, O><<<total, block, 0, s>>>(imgs, starts, B, rule, sf, sd, st)
  if (out_dtype == BSF_F32) {
    if (n == 1) BSF_BS(1, float); else if (n == 2) BSF_BS(2, float); else BSF_BS(3, float);
  } else if (out_dtype == BSF_F64) {
    if (n == 1) BSF_BS(1, double); else if (n == 2) BSF_BS(2, double); else BSF_BS(3, double);
  } else {
    return cudaErrorInvalidValue;
  }
#undef BSF_BS
  return cudaGetLastError();
}
