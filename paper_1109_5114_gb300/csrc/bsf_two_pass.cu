// Algorithm 1 of the paper: split each covariance C = sigma^2 I + Delta C
// (eq. "SigmaIso"), filter with the isotropic sigma^2 I, then with the
// space-variant residual Delta C.  sigma^2 is a fraction (one half in the
// paper) of the smallest eq. "condition2" bound over the field, which keeps
// every residual within the elongation bound e(phi) of eq. "boundE".
//
// The bound is evaluated without trigonometry, in one fixed float64 order:
//   root = sqrt((C11 - C22)^2 + 4 C12^2),
//   tan(phi) = ((C22 - C11) + root) / (2 C12)   if C22 >= C11,
//            = 2 C12 / ((C11 - C22) + root)     otherwise,
//   t = |tan(phi) - 1/tan(phi)| / 2,
//   (e + 1)/(e - 1) = (1 + t)/sqrt(1 + t^2) = (1 + 1/t)/sqrt(1 + 1/t^2),
//   bound = (C11 + C22 - (e + 1)/(e - 1) root) / 2   (factor 1 when C12 = 0).
#include "bsf_reduce.cuh"
#include "bsf_solve.cuh"

namespace {

__device__ __forceinline__ double cond2_bound(double c11, double c12, double c22) {
  const double d = __dsub_rn(c11, c22);
  const double root = __dsqrt_rn(__dadd_rn(__dmul_rn(d, d), __dmul_rn(4.0, __dmul_rn(c12, c12))));
  double ratio = 1.0;
  if (c12 != 0.0) {
    const double tn = c22 >= c11 ? __ddiv_rn(__dadd_rn(__dsub_rn(c22, c11), root), __dmul_rn(2.0, c12))
                                 : __ddiv_rn(__dmul_rn(2.0, c12), __dadd_rn(__dsub_rn(c11, c22), root));
    const double t = __ddiv_rn(fabs(__dsub_rn(tn, __ddiv_rn(1.0, tn))), 2.0);
    if (t > 1.0) {
      const double u = __ddiv_rn(1.0, t);
      ratio = __ddiv_rn(__dadd_rn(1.0, u), __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(u, u))));
    } else {
      ratio = __ddiv_rn(__dadd_rn(1.0, t), __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(t, t))));
    }
  }
  return __ddiv_rn(__dsub_rn(__dadd_rn(c11, c22), __dmul_rn(ratio, root)), 2.0);
}

// The same bound in float32 with an error margin.  Every step is one
// correctly rounded operation; the ratio (a function of t with slope at most
// 1 on either branch) is off by a few units of 2^-24, the tangent by a few
// relative units, so |bound_f32 - bound| stays near 2^-23 (|C11| + |C22| +
// root); the margin 2^-16 (|C11| + |C22| + root) gives an interval [lo, hi]
// that holds the float64 bound.  A value that overflows float32 gives a NaN
// or infinite end, which both passes below treat as "no information".
__device__ __forceinline__ void cond2_interval(float c11, float c12, float c22, float& lo, float& hi) {
  const float d = __fsub_rn(c11, c22);
  const float root = __fsqrt_rn(__fadd_rn(__fmul_rn(d, d), __fmul_rn(4.f, __fmul_rn(c12, c12))));
  float ratio = 1.f;
  if (c12 != 0.f) {
    const float tn = c22 >= c11 ? __fdiv_rn(__fadd_rn(__fsub_rn(c22, c11), root), __fmul_rn(2.f, c12))
                                : __fdiv_rn(__fmul_rn(2.f, c12), __fadd_rn(__fsub_rn(c11, c22), root));
    const float t = __fmul_rn(fabsf(__fsub_rn(tn, __fdiv_rn(1.f, tn))), 0.5f);
    const float u = t > 1.f ? __fdiv_rn(1.f, t) : t;
    ratio = __fdiv_rn(__fadd_rn(1.f, u), __fsqrt_rn(__fadd_rn(1.f, __fmul_rn(u, u))));
  }
  const float b = __fmul_rn(__fsub_rn(__fadd_rn(c11, c22), __fmul_rn(ratio, root)), 0.5f);
  const float e = __fadd_rn(__fmul_rn(__fadd_rn(__fadd_rn(fabsf(c11), fabsf(c22)), root), 0x1p-16f),
                            0x1p-126f);
  lo = __fsub_rn(b, e);
  hi = __fadd_rn(b, e);
}

// Pass 1: an upper limit of min over pixels of max(bound, 0) (float bits;
// non-negative floats order like their bits).
__global__ void k_cond2_upper(const float* __restrict__ cov, int kind, long long HW,
                              unsigned int* __restrict__ upper_bits) {
  float m = __int_as_float(0x7f800000);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
       i += (long long)gridDim.x * blockDim.x) {
    float C11, C12, C22, lo, hi;
    bsf_solve::load_cov(cov, kind, HW, i, C11, C12, C22);
    cond2_interval(C11, C12, C22, lo, hi);
    m = fminf(m, hi == hi ? fmaxf(hi, 0.f) : __int_as_float(0x7f800000));
  }
  m = bsf_block_reduce(m, [](float a, float b) { return fminf(a, b); });
  if (threadIdx.x == 0) atomicMin(upper_bits, __float_as_uint(m));
}

// Pass 2: the float64 bound of the pixels whose interval reaches below that
// limit (the only ones that can hold the minimum); min of max(bound, 0) as
// the bits of a non-negative double.
__global__ void k_cond2_min(const float* __restrict__ cov, int kind, long long HW,
                            const unsigned int* __restrict__ upper_bits,
                            unsigned long long* __restrict__ min_bits) {
  const float U = __uint_as_float(*upper_bits);
  double m = 1.0 / 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
       i += (long long)gridDim.x * blockDim.x) {
    float C11, C12, C22, lo, hi;
    bsf_solve::load_cov(cov, kind, HW, i, C11, C12, C22);
    cond2_interval(C11, C12, C22, lo, hi);
    if (!(fmaxf(lo, 0.f) > U)) m = fmin(m, fmax(cond2_bound(C11, C12, C22), 0.0));
  }
  m = bsf_block_reduce(m, [](double a, double b) { return fmin(a, b); });
  if (threadIdx.x == 0) atomicMin(min_bits, (unsigned long long)__double_as_longlong(m));
}

// iso = (s2, 0, s2), res = (C11 - s2, C12, C22 - s2) in float32,
// s2 = RN32(frac * min bound)
__global__ void k_cov_split(const float* __restrict__ cov, int kind, long long HW,
                            const unsigned long long* __restrict__ min_bits, double frac,
                            float* __restrict__ iso, float* __restrict__ res) {
  const float s2 = __double2float_rn(__dmul_rn(frac, __longlong_as_double((long long)*min_bits)));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
       i += (long long)gridDim.x * blockDim.x) {
    float C11, C12, C22;
    bsf_solve::load_cov(cov, kind, HW, i, C11, C12, C22);
    iso[i] = s2;
    iso[HW + i] = 0.f;
    iso[2 * HW + i] = s2;
    res[i] = __fsub_rn(C11, s2);
    res[HW + i] = C12;
    res[2 * HW + i] = __fsub_rn(C22, s2);
  }
}

int grid_for2(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  const long long cap = 152LL * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t bsf_launch_cov_split(const float* cov, int cov_kind, int H, int W, double frac,
                                 unsigned long long* min_bits, float* iso, float* res,
                                 cudaStream_t s) {
  const long long HW = (long long)H * W;
  // all-ones: above the bits of every non-negative double (min_bits[0]) and
  // float (the low word of min_bits[1])
  cudaError_t e = cudaMemsetAsync(min_bits, 0xff, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  unsigned int* upper = reinterpret_cast<unsigned int*>(min_bits + 1);
  k_cond2_upper<<<grid_for2(HW, 256), 256, 0, s>>>(cov, cov_kind, HW, upper);
  k_cond2_min<<<grid_for2(HW, 256), 256, 0, s>>>(cov, cov_kind, HW, upper, min_bits);
  k_cov_split<<<grid_for2(HW, 256), 256, 0, s>>>(cov, cov_kind, HW, min_bits, frac, iso, res);
  return cudaGetLastError();
}
