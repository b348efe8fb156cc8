// Step-field kernel (plan and diagnostics) and the value reduction used by
// automatic q.  The per-pixel solve itself is in bsf_solve.cuh.
#include "bsf_reduce.cuh"
#include "bsf_solve.cuh"

namespace {

using namespace bsf_solve;

// rule BSF_STEP_D2: Lf holds floor(lambda~) (capped at 65535) and the mass is
// that of the interpolated kernels (prod_k M_k, times 2^40).
// dirset (BSF_DIRS_*): the direction set of the integer-step rules; with
// BSF_DIRS_PAIR bit 15 of L1 marks the pixels that take the second set.
__global__ void k_steps(const float* __restrict__ cov, int kind, int H, int W, int n, int rule,
                        int dirset, int R, ushort4* __restrict__ Lf, DevStatus* st) {
  const long long HW = (long long)H * W;
  int my_reach = 0;
  float my_mass = 1.f;
  unsigned my_clamp = 0, my_bad = 0, my_range = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
       i += (long long)gridDim.x * blockDim.x) {
    int L[4], flags, reach;
    float C11, C12, C22, mass;
    load_cov(cov, kind, HW, i, C11, C12, C22);
    if (rule == BSF_STEP_D2) {
      int Hq[4];
      float lam[4];
      if (!pixel_steps_d2(C11, C12, C22, n, R, Hq, lam, flags, reach)) ++my_range;
      mass = 1.f;
      for (int k = 0; k < 4; ++k) {
        mass *= (float)d2_mass(Hq[k], n);
        L[k] = min(Hq[k] >> 9, 65535);
      }
    } else if (rule == BSF_STEP_SAMPLED) {
      const bool second = dirset == BSF_DIRS_SECOND || (dirset == BSF_DIRS_PAIR && use_second_set(C11, C12, C22));
      const bool ok = second ? pixel_steps_sampled_k(C11, C12, C22, R, L, flags, reach)
                             : pixel_steps_sampled(C11, C12, C22, R, L, flags, reach);
      if (!ok) ++my_range;
      // the bound of |acc|: prod Lq 2^-13 (Cartesian) or 15 prod Lq 2^-5 (second set), times max|Q|
      mass = (float)L[0] * (float)L[1] * (float)L[2] * (float)L[3] * (second ? 15.f * 0x1p-5f : 0x1p-13f);
      const int sh = second ? 5 : 9;
      for (int k = 0; k < 4; ++k) L[k] = min(L[k] >> sh, 65535);  // floor(lambda)
      if (dirset == BSF_DIRS_PAIR && second) L[0] |= 0x8000;
    } else {
      bool second;
      if (!pixel_steps_set(dirset, C11, C12, C22, n, rule, R, L, flags, reach, second)) ++my_range;
      // prod L^n in float32 (a bound for the choice of q; the stencil checks exactly)
      const float m1 = (float)(L[0] * L[1]) * (float)(L[2] * L[3]);
      mass = m1;
      for (int j = 1; j < n; ++j) mass *= m1;
      if (dirset == BSF_DIRS_PAIR && second) L[0] |= 0x8000;
    }
    my_reach = max(my_reach, reach);
    my_mass = fmaxf(my_mass, mass);
    my_clamp += (flags & 1) ? 1u : 0u;
    my_bad += (flags & 2) ? 1u : 0u;
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
  // NaN propagates through the block (fmax would drop it)
  m = bsf_block_reduce(m, [](double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); });
  if (threadIdx.x == 0) bsf_atomic_max_pos_double(&st->max_absf_bits, m);
}

int grid_for(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  const long long cap = 152LL * 16;  // 16 resident 256-thread blocks per SM
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t bsf_launch_steps(const float* cov, int cov_kind, int H, int W, int n, int rule,
                             int dirset, int R, ushort4* Lf, DevStatus* st, cudaStream_t s) {
  if (cov_kind != BSF_COV_C && cov_kind != BSF_COV_LOGSIG_THETA_LOGRHO) return cudaErrorInvalidValue;
  if (rule == BSF_STEP_D2 && (n > 2 || dirset != BSF_DIRS_CARTESIAN)) return cudaErrorInvalidValue;
  if (rule == BSF_STEP_SAMPLED && n != 1) return cudaErrorInvalidValue;
  if (dirset < BSF_DIRS_CARTESIAN || dirset > BSF_DIRS_PAIR) return cudaErrorInvalidValue;
  const int threads = 256;
  k_steps<<<grid_for((long long)H * W, threads), threads, 0, s>>>(cov, cov_kind, H, W, n, rule,
                                                                  dirset, R, Lf, st);
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
