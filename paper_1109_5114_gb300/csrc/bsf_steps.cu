// Per-pixel step solve: covariance -> minimum-kurtosis scales -> integer steps.
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
// Newton's method from v0 = -q/p converges monotonically; four steps are
// taken.  Every operation is an explicit IEEE round-to-nearest float32
// intrinsic (no contraction into fused multiply-add), so the result, and the
// integer steps rounded from it, are reproducible bit for bit by any IEEE
// float32 implementation of the same sequence.
//
// Steps: lambda_k = sqrt(1 + A_k / |d_k|^2) (BSF_STEP_D1: L grid samples
// spaced |d_k| apart then have variance A_k/12, that of a box of width a_k),
// or lambda_k = a_k / |d_k| (BSF_STEP_D1_PAPER); L_k = the admissible integer
// nearest lambda_k (odd when n is odd), ties to the larger.
#include "bsf_device.cuh"

namespace {

constexpr float kLMax = 32767.f;

struct Solved {
  float A[4];
  int flags;  // 1 = clamped to e(phi), 2 = non-finite input
};

__device__ __forceinline__ Solved solve_scales(float C11, float C12, float C22, int n) {
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
  const float B = __fdiv_rn(12.f, (float)n);
  const float c1 = __fmul_rn(B, c11), c3 = __fmul_rn(B, c22), b = __fmul_rn(B, c12);
  const float s = __fadd_rn(c1, c3), d = __fsub_rn(c1, c3);
  const float bb = __fmul_rn(b, b), dd = __fmul_rn(d, d);
  const float p = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(2.5f, dd), __fmul_rn(2.f, __fmul_rn(c1, c3))),
                                      __fmul_rn(8.f, bb)), 0.125f);
  const float q = __fmul_rn(__fmul_rn(s, __fsub_rn(bb, __fmul_rn(0.25f, dd))), 0.125f);
  float v = (p > 0.f) ? __fdiv_rn(-q, p) : 0.f;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
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
  float L = (n & 1) ? __fadd_rn(__fmul_rn(2.f, floorf(__fmul_rn(0.5f, lam))), 1.f)
                    : floorf(__fadd_rn(lam, 0.5f));
  L = fminf(fmaxf(L, 1.f), kLMax);
  return (int)L;
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

__global__ void k_steps(const float* __restrict__ cov, int H, int W, int n, int rule, int R,
                        ushort4* __restrict__ Lf, DevStatus* st) {
  const long long HW = (long long)H * W;
  int my_reach = 0;
  float my_mass = 1.f;
  unsigned my_clamp = 0, my_bad = 0, my_range = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
       i += (long long)gridDim.x * blockDim.x) {
    Solved sv = solve_scales(cov[i], cov[HW + i], cov[2 * HW + i], n);
    int L[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float a = (k & 1) ? __fmul_rn(sv.A[k], 0.5f) : sv.A[k];  // A / |d_k|^2
      const float lam = (rule == BSF_STEP_D1_PAPER) ? __fsqrt_rn(a) : __fsqrt_rn(__fadd_rn(1.f, a));
      L[k] = round_step(lam, n);
    }
    int reach = tap_reach(L, n);
    if (R >= 0 && reach > R) {  // keep every tap inside the workspace (R >= 3n always)
      L[0] = L[1] = L[2] = L[3] = 1;
      reach = tap_reach(L, n);
      ++my_range;
    }
    // prod L^n in float32 (a bound for the choice of q; the stencil checks exactly)
    const float m1 = (float)(L[0] * L[1]) * (float)(L[2] * L[3]);
    float mass = m1;
    for (int j = 1; j < n; ++j) mass *= m1;
    my_reach = max(my_reach, reach);
    my_mass = fmaxf(my_mass, mass);
    my_clamp += (sv.flags & 1) ? 1u : 0u;
    my_bad += (sv.flags & 2) ? 1u : 0u;
    Lf[i] = make_ushort4((unsigned short)L[0], (unsigned short)L[1], (unsigned short)L[2],
                         (unsigned short)L[3]);
  }
  // block reduction, then one atomic per block
  __shared__ int s_reach[32];
  __shared__ float s_mass[32];
  __shared__ unsigned s_cnt[3][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    my_reach = max(my_reach, __shfl_xor_sync(0xffffffffu, my_reach, o));
    my_mass = fmaxf(my_mass, __shfl_xor_sync(0xffffffffu, my_mass, o));
    my_clamp += __shfl_xor_sync(0xffffffffu, my_clamp, o);
    my_bad += __shfl_xor_sync(0xffffffffu, my_bad, o);
    my_range += __shfl_xor_sync(0xffffffffu, my_range, o);
  }
  if (lane == 0) {
    s_reach[wid] = my_reach; s_mass[wid] = my_mass;
    s_cnt[0][wid] = my_clamp; s_cnt[1][wid] = my_bad; s_cnt[2][wid] = my_range;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    int r = 0; float m = 1.f; unsigned c0 = 0, c1 = 0, c2 = 0;
    for (int w = 0; w < nw; ++w) {
      r = max(r, s_reach[w]); m = fmaxf(m, s_mass[w]);
      c0 += s_cnt[0][w]; c1 += s_cnt[1][w]; c2 += s_cnt[2][w];
    }
    atomicMax(&st->max_reach, r);
    bsf_atomic_max_pos_float(&st->max_mass_bits, m);
    if (c0) atomicAdd(&st->clamp_count, c0);
    if (c1) { atomicAdd(&st->bad_count, c1); bsf_set_error(st, BSF_ECOV); }
    if (c2) { atomicAdd(&st->range_count, c2); bsf_set_error(st, BSF_ERANGE); }
  }
}

template <typename In>
__global__ void k_absmax(const In* __restrict__ img, long long ld, int H, int W, DevStatus* st) {
  double m = 0.0;
  const long long HW = (long long)H * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
       i += (long long)gridDim.x * blockDim.x) {
    const long long y = i / W, x = i - y * W;
    const double v = fabs((double)img[y * ld + x]);
    m = (v > m || v != v) ? v : m;  // NaN propagates (fails the later bound)
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) bsf_atomic_max_pos_double(&st->max_absf_bits, m);
}

int grid_for(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  const long long cap = 152LL * 16;  // 16 resident 256-thread blocks per SM
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t bsf_launch_steps(const float* cov, int cov_kind, int H, int W, int n, int rule,
                             int R, ushort4* Lf, DevStatus* st, cudaStream_t s) {
  if (cov_kind != BSF_COV_C) return cudaErrorInvalidValue;
  const int threads = 256;
  k_steps<<<grid_for((long long)H * W, threads), threads, 0, s>>>(cov, H, W, n, rule, R, Lf, st);
  return cudaGetLastError();
}

cudaError_t bsf_launch_absmax(const void* img, int dtype, long long ld, int H, int W,
                              DevStatus* st, cudaStream_t s) {
  const int threads = 256;
  const int g = grid_for((long long)H * W, threads);
  switch (dtype) {
    case BSF_U8: k_absmax<<<g, threads, 0, s>>>((const uint8_t*)img, ld, H, W, st); break;
    case BSF_F32: k_absmax<<<g, threads, 0, s>>>((const float*)img, ld, H, W, st); break;
    case BSF_F64: k_absmax<<<g, threads, 0, s>>>((const double*)img, ld, H, W, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
