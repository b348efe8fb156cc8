// Backward pass of the D1 filter with respect to the image: the transpose of
// the forward pipeline (Section 1.1's BoxFilter: extension, running sums,
// finite differences), read backwards.
//
//   forward:   out(p) = sum_t w_t S(tap_t(p)) / D_p,  S = C4^n C2^n C3^n C1^n E f
//   backward:  G = sum_p (gout(p)/D_p) sum_t w_t delta_{tap_t(p)}     (scatter)
//              G <- (C1^T)^n (C3^T)^n (C2^T)^n (C4^T)^n G                (suffix sums)
//              gimg = E^T G                                           (extension fold)
//
// Fixed point: each weight gout(p)/D_p is quantised once,
//   g(p) = RNE(RN32(RN32(gout(p) 2^qg) / RN32(D_p))),  qg = 54 - ceil(log2 max|gout|)
// (clamped to [0, 100]; the max is reduced on the device and every thread
// derives the same qg), the scatter adds w_t g(p) with 64-bit integer
// reductions (exact and order-independent, hence deterministic), the suffix
// sums wrap modulo 2^64, and gimg = RN32(acc) 2^-qg.  Contexts with uint128
// running sums (large kernels, masses up to 2^100) take the same pipeline in
// 128 bits: qg = 118 - ceil(log2 max|gout|) in [0, 126], 128-bit additions
// built from two 64-bit atomics (the low word's old value gives the carry),
// sums modulo 2^128.
#include <cstring>

#include "bsf_reduce.cuh"
#include "bsf_solve.cuh"

namespace {

__global__ void k_gabsmax(const float* __restrict__ g, long long ld, int H, int W, DevStatus* st) {
  bsf_grid_dep_launch();  // the scatter may solve its steps meanwhile (it waits for this grid)
  float m = 0.f;
  const long long HW = (long long)H * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
       i += (long long)gridDim.x * blockDim.x) {
    const long long y = i / W, x = i - y * W;
    m = fmaxf(m, fabsf(g[y * ld + x]));  // NaN is ignored here; the weights check it
  }
  m = bsf_block_reduce(m, [](float a, float b) { return fmaxf(a, b); });
  if (threadIdx.x == 0) bsf_atomic_max_pos_float(&st->max_absg_bits, m);
}

// qg from the float32 bits of max|gout|: 54 - ceil(log2 m), clamped to [0, 100]
__device__ __forceinline__ int grad_q(unsigned mbits) {
  const unsigned E = (mbits >> 23) & 0xffu, M = mbits & 0x7fffffu;
  int c;
  if (E == 0 || E == 0xffu) c = E == 0 && M != 0 ? -126 : 0;  // subnormal / zero / non-finite
  else c = (int)E - 127 + (M != 0 ? 1 : 0);
  const int q = 54 - c;
  return q < 0 ? 0 : (q > 100 ? 100 : q);
}

// (-1)^t C(n, t) as a two's-complement weight of the element type
template <int NF, typename T = uint64_t> __device__ __forceinline__ T tap_w(int t) {
  const unsigned long long c = NF == 1 ? 1 : (NF == 2 ? (t == 1 ? 2 : 1) : (t == 1 || t == 2 ? 3 : 1));
  return (t & 1) ? (T)0 - (T)c : (T)c;
}

// qg of the 128-bit adjoint: 118 - ceil(log2 max|gout|), clamped to [0, 126]
__device__ __forceinline__ int grad_q_wide(unsigned mbits) {
  const unsigned E = (mbits >> 23) & 0xffu, M = mbits & 0x7fffffu;
  int c;
  if (E == 0 || E == 0xffu) c = E == 0 && M != 0 ? -126 : 0;
  else c = (int)E - 127 + (M != 0 ? 1 : 0);
  const int q = 118 - c;
  return q < 0 ? 0 : (q > 126 ? 126 : q);
}

__device__ __forceinline__ void red_add(uint64_t* p, uint64_t v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}
// exact 128-bit addition modulo 2^128 from two 64-bit atomics: the low word's
// old value tells whether this addition carried into the high word
__device__ __forceinline__ void red_add(u128* p, u128 v) {
  unsigned long long* q = reinterpret_cast<unsigned long long*>(p);
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  const unsigned long long old = atomicAdd(q, lo);
  const unsigned long long h = hi + ((old + lo < old) ? 1ull : 0ull);
  if (h) atomicAdd(q + 1, h);
}

// Transposed taps: pixel p adds w_t g(p) at each of its (n+1)^4 taps.  A warp
// is 32 consecutive pixels of one row; along d1 the taps of lanes L1 apart
// fall on each other (lane x + t L1's tap t is lane x's tap 0) whenever the
// two pixels have the same steps, so lane x adds its partners' tap values to
// its own tap 0 through shuffles and issues one reduction for all of them;
// a tap whose lane x - t L1 took it is not issued again.  Sums are modulo
// 2^64, so the grouping changes nothing but the number of reductions.
template <int NF, typename T = uint64_t>
__global__ void __launch_bounds__(256)
k_scatter_d1(T* __restrict__ G, long long pitch, int R,
             const float* __restrict__ cov, int kind, int rule, const float* __restrict__ gout,
             long long ldg, int H, int W, int row0, int rows, int qg_given, DevStatus* st) {
  constexpr bool kWide = sizeof(T) == 16;
  // pixel (x, row0 + y) of the band; G holds the band's padded rows
  // (row 0 = image row row0 - R).  blockDim.x == 32: one warp per row segment.
  const int lane = threadIdx.x;
  const int x = blockIdx.x * 32 + lane;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (y >= rows) return;  // uniform across the warp
  const bool in = x < W;
  int L[4] = {1, 1, 1, 1};
  T g = 0;
  if (in) {
    const long long HW = (long long)H * W, i = (long long)(row0 + y) * W + x;
    int flags, reach;
    float C11, C12, C22;
    bsf_solve::load_cov(cov, kind, HW, i, C11, C12, C22);
    bsf_solve::pixel_steps(C11, C12, C22, NF, rule, R, L, flags, reach);
  }
  // the steps read only the field; max |gout| comes from the kernel before
  // this one when it was launched as its programmatic dependent
  bsf_grid_dep_wait();
  if (in) {
    const int qg = qg_given >= 0 ? qg_given : (kWide ? grad_q_wide(st->max_absg_bits) : grad_q(st->max_absg_bits));
    T D = (T)(unsigned)(L[0] * L[1]) * (T)(unsigned)(L[2] * L[3]);
    const T D1 = D;
#pragma unroll
    for (int j = 1; j < NF; ++j) D *= D1;
    const float xg = __fmul_rn(gout[(long long)(row0 + y) * ldg + x], bsf_pow2_f32(qg));  // exact scaling
    bool ok;
    float Df;
    if constexpr (kWide) Df = bsf_rn32_u(D);
    else Df = bsf_rn32_u64(D);
    g = bsf_quantize_f32<T>(__fdiv_rn(xg, Df), 0, ok);
    if (!ok) bsf_set_error(st, BSF_EOVERFLOW);
  }
  // lanes with equal steps share tap positions; L < 2^15, so the pair packs
  const unsigned sa = in ? (unsigned)L[0] | ((unsigned)L[1] << 16) : 0xffffffffu;
  const unsigned sb = in ? (unsigned)L[2] | ((unsigned)L[3] << 16) : 0xffffffffu;
  const int L1 = L[0];
  bool up[NF + 1], dn[NF + 1];
  int src[NF + 1];
#pragma unroll
  for (int t = 1; t <= NF; ++t) {
    const int u = lane + t * L1, d = lane - t * L1;
    src[t] = u < 32 ? u : lane;
    const unsigned ua = __shfl_sync(0xffffffffu, sa, src[t]), ub = __shfl_sync(0xffffffffu, sb, src[t]);
    const unsigned da = __shfl_sync(0xffffffffu, sa, d >= 0 ? d : lane),
                   db = __shfl_sync(0xffffffffu, sb, d >= 0 ? d : lane);
    up[t] = in && u < 32 && ua == sa && ub == sb;
    dn[t] = in && d >= 0 && da == sa && db == sb;
  }
  const long long e1 = 1, e2 = pitch + 1, e3 = pitch, e4 = pitch - 1;
  const long long c1 = NF * (L[0] - 1) / 2, c2 = NF * (L[1] - 1) / 2, c3 = NF * (L[2] - 1) / 2,
                  c4 = NF * (L[3] - 1) / 2;
  T* base = G + (long long)(y + R) * pitch + (x + R) + c1 * e1 + c2 * e2 + c3 * e3 + c4 * e4;
  const long long s2 = L[1] * e2, s3 = L[2] * e3, s4 = L[3] * e4;
#pragma unroll 1
  for (int t4 = 0; t4 <= NF; ++t4) {
#pragma unroll
    for (int t3 = 0; t3 <= NF; ++t3) {
#pragma unroll
      for (int t2 = 0; t2 <= NF; ++t2) {
        const T w = g * tap_w<NF, T>(t2) * tap_w<NF, T>(t3) * tap_w<NF, T>(t4);
        T* p = base - t2 * s2 - t3 * s3 - t4 * s4;
        T tot = w;  // tap 0 (weight 1)
        T v[NF + 1];
#pragma unroll
        for (int t = 1; t <= NF; ++t) {
          v[t] = w * tap_w<NF, T>(t);
          const T pv = bsf_shfl_idx<T>(v[t], src[t]);
          if (up[t]) tot += pv;
        }
        if (in && tot != 0) red_add(p, tot);
#pragma unroll
        for (int t = 1; t <= NF; ++t)
          if (in && !dn[t] && v[t] != 0) red_add(p - t * L1, v[t]);
      }
    }
  }
}

// Padded coordinates z in [-R, N + R) whose extension maps onto image
// coordinate i, visited as padded indices z + R.
template <typename F>
__device__ __forceinline__ void for_preimages(int i, int N, int R, int boundary, F&& f) {
  if (boundary == BSF_ZERO) {
    f(i + R);
  } else if (boundary == BSF_REPLICATE) {
    const int lo = i == 0 ? -R : i, hi = i == N - 1 ? N - 1 + R : i;
    for (int z = lo; z <= hi; ++z) f(z + R);
  } else {  // half-sample symmetric: z = i + 2kN or z = 2kN - 1 - i
    const int P = 2 * N;
    for (int fam = 0; fam < 2; ++fam) {
      const int b = fam == 0 ? i : P - 1 - i;  // representative in [0, 2N)
      // smallest z >= -R with z = b (mod 2N)
      int z = b - ((b + R + P - 1) / P) * P;
      if (z < -R) z += P;
      for (; z < N + R; z += P) f(z + R);
    }
  }
}

template <typename T>
__global__ void k_fold_x(const T* __restrict__ G, long long pitch, int Hp, int W,
                         int R, int boundary, T* __restrict__ Gx) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int yr = blockIdx.y;
  if (x >= W || yr >= Hp) return;
  const T* row = G + (long long)yr * pitch;
  T acc = 0;
  for_preimages(x, W, R, boundary, [&](int xp) { acc += row[xp]; });
  Gx[(long long)yr * W + x] = acc;
}

// Both folds at once: pixel (x, y) sums G over the padded positions that
// extend onto it in each dimension (interior pixels: one), then rounds.
__global__ void k_fold_xy_out(const unsigned long long* __restrict__ G, long long pitch, int H, int W,
                              int R, int boundary, float* __restrict__ gimg, long long ldo,
                              const DevStatus* st) {
  bsf_grid_dep_wait();  // a programmatic dependent of the last suffix sums
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= W || y >= H) return;
  unsigned long long acc = 0;
  if (x >= R && x < W - R && y >= R && y < H - R) {  // no preimage but itself
    acc = G[(long long)(y + R) * pitch + (x + R)];
  } else {
    for_preimages(y, H, R, boundary, [&](int yp) {
      const unsigned long long* row = G + (long long)yp * pitch;
      for_preimages(x, W, R, boundary, [&](int xp) { acc += row[xp]; });
    });
  }
  const int qg = grad_q(st->max_absg_bits);
  gimg[(long long)y * ldo + x] = __fmul_rn(bsf_rn32_i64((long long)acc), bsf_pow2_f32(-qg));
}

// Band form of the row fold: image rows a0 .. a1 - 1 receive the band's
// padded rows (row r = extended row row0 - R + r, r < Hb) that extend onto
// them; the exact integer sums are written (no rounding).
template <typename T>
__global__ void k_fold_y_band(const T* __restrict__ Gx, int Hb, int H, int W, int R,
                              int row0, int boundary, int a0, int a1,
                              T* __restrict__ acc_out, long long lda) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = a0 + (int)blockIdx.y;
  if (x >= W || y >= a1) return;
  T acc = 0;
  for_preimages(y, H, R, boundary, [&](int zp) {
    const int r = zp - row0;  // zp = z + R, r = z - (row0 - R)
    if (r >= 0 && r < Hb) acc += Gx[(long long)r * W + x];
  });
  acc_out[(long long)(y - a0) * lda + x] = acc;
}

__device__ __forceinline__ float rn32_signed(uint64_t v) { return bsf_rn32_i64((long long)v); }
__device__ __forceinline__ float rn32_signed(u128 v) { return bsf_rn32((i128)v); }

template <typename T>
__global__ void k_grad_finalize(const T* __restrict__ acc, long long lda, int rows, int W,
                                int qg, float* __restrict__ gimg, long long ldo) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= W || y >= rows) return;
  gimg[(long long)y * ldo + x] = __fmul_rn(rn32_signed(acc[(long long)y * lda + x]), bsf_pow2_f32(-qg));
}

// acc[r][x] += halo[r][x] modulo 2^64 or 2^128 (the neighbours' share of a
// band's adjoint sums)
template <typename T>
__global__ void k_add_rows(T* __restrict__ acc, long long lda, const T* __restrict__ halo,
                           long long ldh, int rows, int W) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= W || y >= rows) return;
  acc[(long long)y * lda + x] += halo[(long long)y * ldh + x];
}

int grid_for(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  const long long cap = 152LL * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

int bsf_grad_q_host(double m) {
  // the rule of grad_q on the float32 value of m
  const float f = (float)m;
  unsigned b;
  std::memcpy(&b, &f, sizeof b);
  const unsigned E = (b >> 23) & 0xffu, M = b & 0x7fffffu;
  int c;
  if (E == 0 || E == 0xffu) c = E == 0 && M != 0 ? -126 : 0;
  else c = (int)E - 127 + (M != 0 ? 1 : 0);
  const int q = 54 - c;
  return q < 0 ? 0 : (q > 100 ? 100 : q);
}

int bsf_grad_q_host_wide(double m) {
  // the rule of grad_q_wide on the float32 value of m
  const float f = (float)m;
  unsigned b;
  std::memcpy(&b, &f, sizeof b);
  const unsigned E = (b >> 23) & 0xffu, M = b & 0x7fffffu;
  int c;
  if (E == 0 || E == 0xffu) c = E == 0 && M != 0 ? -126 : 0;
  else c = (int)E - 127 + (M != 0 ? 1 : 0);
  const int q = 118 - c;
  return q < 0 ? 0 : (q > 126 ? 126 : q);
}

cudaError_t bsf_launch_gabsmax(const float* gout, long long ldg, int H, int W, DevStatus* st,
                               cudaStream_t s) {
  k_gabsmax<<<grid_for((long long)H * W, 256), 256, 0, s>>>(gout, ldg, H, W, st);
  return cudaGetLastError();
}

cudaError_t bsf_launch_scatter_d1(int n, int elem_bytes, void* G, long long pitch, int R, const float* cov,
                                  int cov_kind, int rule, const float* gout, long long ldg, int H,
                                  int W, int row0, int rows, int qg, DevStatus* st, cudaStream_t s,
                                  bool after_absmax) {
  const int k = cov_kind;
  // after_absmax: a programmatic dependent of the max |gout| reduction just
  // before on the stream (the steps are solved while it finishes)
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = after_absmax ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((W + 31) / 32, (rows + 7) / 8);
  cfg.blockDim = dim3(32, 8);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
#define BSF_SC(NF, T) \
  return cudaLaunchKernelEx(&cfg, k_scatter_d1<NF, T>, (T*)G, pitch, R, cov, k, rule, gout, ldg, H, W, row0, rows, \
                            qg, st)
  if (elem_bytes == 8) {
    if (n == 1) BSF_SC(1, uint64_t); else if (n == 2) BSF_SC(2, uint64_t); else if (n == 3) BSF_SC(3, uint64_t);
    else return cudaErrorInvalidValue;
  } else if (elem_bytes == 16) {
    if (n == 1) BSF_SC(1, u128); else if (n == 2) BSF_SC(2, u128); else if (n == 3) BSF_SC(3, u128);
    else return cudaErrorInvalidValue;
  } else {
    return cudaErrorInvalidValue;
  }
#undef BSF_SC
  return cudaGetLastError();
}

cudaError_t bsf_launch_fold_band(int elem_bytes, const void* G, long long pitch, int Hb, int H, int W, int R,
                                 int row0, int boundary, void* Gx, int a0, int a1, void* acc,
                                 long long lda, cudaStream_t s) {
  dim3 blk(128);
#define BSF_FB(T)                                                                                  \
  k_fold_x<T><<<dim3((W + 127) / 128, Hb), blk, 0, s>>>((const T*)G, pitch, Hb, W, R, boundary, (T*)Gx); \
  k_fold_y_band<T><<<dim3((W + 127) / 128, a1 - a0), blk, 0, s>>>((const T*)Gx, Hb, H, W, R, row0,   \
                                                                  boundary, a0, a1, (T*)acc, lda)
  if (elem_bytes == 8) {
    BSF_FB(uint64_t);
  } else if (elem_bytes == 16) {
    BSF_FB(u128);
  } else {
    return cudaErrorInvalidValue;
  }
#undef BSF_FB
  return cudaGetLastError();
}

cudaError_t bsf_launch_add_rows(int elem_bytes, void* acc, long long lda, const void* halo, long long ldh,
                                int rows, int W, cudaStream_t s) {
  const dim3 grid((W + 127) / 128, rows);
  if (elem_bytes == 8)
    k_add_rows<uint64_t><<<grid, 128, 0, s>>>((uint64_t*)acc, lda, (const uint64_t*)halo, ldh, rows, W);
  else if (elem_bytes == 16)
    k_add_rows<u128><<<grid, 128, 0, s>>>((u128*)acc, lda, (const u128*)halo, ldh, rows, W);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t bsf_launch_grad_finalize(int elem_bytes, const void* acc, long long lda, int rows, int W, int qg,
                                     float* gimg, long long ldo, cudaStream_t s) {
  const dim3 grid((W + 127) / 128, rows);
  if (elem_bytes == 8)
    k_grad_finalize<uint64_t><<<grid, 128, 0, s>>>((const uint64_t*)acc, lda, rows, W, qg, gimg, ldo);
  else if (elem_bytes == 16)
    k_grad_finalize<u128><<<grid, 128, 0, s>>>((const u128*)acc, lda, rows, W, qg, gimg, ldo);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t bsf_launch_fold(const void* G, long long pitch, int Hp, int H, int W, int R,
                            int boundary, void* Gx, float* gimg, long long ldo, const DevStatus* st,
                            cudaStream_t s) {
  (void)Hp;
  (void)Gx;
  dim3 blk(128);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((W + 127) / 128, H);
  cfg.blockDim = blk;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fold_xy_out, (const unsigned long long*)G, pitch, H, W, R, boundary, gimg,
                            ldo, st);
}
