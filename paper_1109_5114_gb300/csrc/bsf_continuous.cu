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

using namespace bsf_d2;

// qg for the continuous-step adjoint: 118 - ceil(log2 max|gout|) in [0, 126]
// (exact modulo 2^128 with 2^8 of headroom; 2^126 is still a float32).
__device__ __forceinline__ int grad_q128(unsigned mbits) {
  const unsigned E = (mbits >> 23) & 0xffu, M = mbits & 0x7fffffu;
  int c;
  if (E == 0 || E == 0xffu) c = E == 0 && M != 0 ? -126 : 0;
  else c = (int)E - 127 + (M != 0 ? 1 : 0);
  const int q = 118 - c;
  return q < 0 ? 0 : (q > 126 ? 126 : q);
}

// 128-bit atomic add from two 64-bit ones: the low word's old value tells
// this thread whether its addition carried, and the high word receives the
// high part plus that carry.  The low word then holds the low 64 bits of the
// sum and the high word every carry out of it, so the pair is the exact sum
// modulo 2^128 whatever the order of the additions.
__device__ __forceinline__ void atomic_add_u128(u128* p, u128 v) {
  unsigned long long* q = reinterpret_cast<unsigned long long*>(p);
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  const unsigned long long old = atomicAdd(q, lo);
  const unsigned long long h = hi + ((old + lo < old) ? 1ull : 0ull);
  if (h) atomicAdd(q + 1, h);
}

__device__ __forceinline__ u128 mul_signed(u128 x, int v) {
  return v >= 0 ? mul_small(x, (unsigned)v) : (u128)0 - mul_small(x, (unsigned)(-v));
}

// Interpolation weights of one direction (see the stencil): n = 2:
// 1024 - th, th, -2048, th, 1024 - th; n = 1: 1024 - th, th, -th, th - 1024.
template <int NF> __device__ __forceinline__ int tap_weight(unsigned th, int i) {
  const int t = (int)th;
  if (NF == 2) return i == 0 || i == 4 ? 1024 - t : (i == 2 ? -2048 : t);
  return i == 0 ? 1024 - t : (i == 1 ? t : (i == 2 ? -t : t - 1024));
}

// Adjoint of the continuous-step taps: each pixel adds g(p) times the
// product of its four interpolation weights at each of its samples, g(p) =
// RNE(RN32(RN32(gout 2^qg) / RN32(M))) the quantised normalised weight.
// A warp is 32 consecutive pixels of one row (blockDim.x == 32).  Along d1
// the second sample of a bracket pair of lane x falls on the first sample of
// lane x + 1 when both pixels have the same brackets a0 in every direction,
// so lane x + 1 adds it to its own through a shuffle and one 128-bit add
// serves both (n = 2: samples 0/1 and 3/4 pair up, n = 1: 0/1 and 2/3).  The
// low-word atomics of a group are all issued before their high-word adds.
// Pixels of image rows [row0, row0 + rows) scatter into G, whose padded row
// 0 is image row row0 - R (the whole image: row0 = 0, rows = H); qg_given >=
// 0 fixes the fraction bits of the weights, -1 takes them from the device
// maximum of |gout|.
// Six resident blocks per SM asked of the register allocator (80 registers):
// the scatter waits on its atomics' returns, and more warps in flight hide
// that latency (1.51 against 1.88 ms per 1024^2 image with the default 126).
template <int NF>
__global__ void __launch_bounds__(128, 6)
k_scatter_d2(u128* __restrict__ G, long long pitch, int R, const float* __restrict__ cov, int kind,
             const float* __restrict__ gout, long long ldg, int H, int W, int row0, int rows, int qg_given,
             DevStatus* st) {
  using P = Pattern<NF>;
  constexpr int NP = P::NP;
  // the pairs along d1: (first, second) sample indices
  constexpr int PA0 = 0, PA1 = 1, PB0 = NF == 2 ? 3 : 2, PB1 = NF == 2 ? 4 : 3;
  const int lane = threadIdx.x;
  const int x = blockIdx.x * 32 + lane;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (y >= rows) return;  // uniform across the warp
  const bool in = x < W;
  int Hq[4] = {kHalf, kHalf, kHalf, kHalf};
  u128 g = 0;
  if (in) {
    const long long HW = (long long)H * W, i = (long long)(row0 + y) * W + x;
    float C11, C12, C22;
    load_cov(cov, kind, HW, i, C11, C12, C22);
    int flags, reach;
    float lam[4];
    pixel_steps_d2(C11, C12, C22, NF, R, Hq, lam, flags, reach);
    u128 M = 1;
    for (int k = 0; k < 4; ++k) M *= (u128)d2_mass(Hq[k], NF);
    const int qg = qg_given >= 0 ? qg_given : grad_q128(st->max_absg_bits);
    const float xg = __fmul_rn(gout[(long long)(row0 + y) * ldg + x], bsf_pow2_f32(qg));  // exact scaling
    bool ok;
    g = bsf_quantize_f32<u128>(__fdiv_rn(xg, bsf_rn32_u(M)), 0, ok);
    if (!ok) bsf_set_error(st, BSF_EOVERFLOW);
  }
  const int p32 = (int)pitch;
  const int estep[4] = {1, p32 + 1, p32, p32 - 1};
  int a0[4];
  unsigned th[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int Q0 = NF == 2 ? 2 * Hq[k] - 1024 : Hq[k] - 512;
    a0[k] = Q0 >> 10;
    th[k] = (unsigned)(Q0 & 1023);
  }
  // lanes whose brackets agree in every direction share sample positions
  const unsigned sa = in ? (unsigned)a0[0] | ((unsigned)a0[1] << 16) : 0xffffffffu;
  const unsigned sb = in ? (unsigned)a0[2] | ((unsigned)a0[3] << 16) : 0xffffffffu;
  const unsigned la = __shfl_up_sync(0xffffffffu, sa, 1), lb = __shfl_up_sync(0xffffffffu, sb, 1);
  const unsigned ra = __shfl_down_sync(0xffffffffu, sa, 1), rb = __shfl_down_sync(0xffffffffu, sb, 1);
  const bool from_left = in && lane > 0 && la == sa && lb == sb;     // take lane - 1's seconds
  const bool to_right = in && lane < 31 && ra == sa && rb == sb;     // lane + 1 takes mine
  const int base = (y + R) * p32 + (x + R);
  // weights of the first direction's samples, and their positions
  int w1[NP], off1[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    w1[i] = tap_weight<NF>(th[0], i);
    off1[i] = P::pos(a0[0], i);
  }
#pragma unroll 1
  for (int i4 = 0; i4 < NP; ++i4) {
    const int w4 = tap_weight<NF>(th[3], i4);
    const u128 c4 = mul_signed(g, w4);
    const int b4 = base + P::pos(a0[3], i4) * estep[3];
#pragma unroll 1
    for (int i3 = 0; i3 < NP; ++i3) {
      const int w3 = tap_weight<NF>(th[2], i3);
      const u128 c3 = mul_signed(c4, w3);
      const int b3 = b4 + P::pos(a0[2], i3) * estep[2];
#pragma unroll
      for (int i2 = 0; i2 < NP; ++i2) {
        const int w2 = tap_weight<NF>(th[1], i2);
        const u128 c2 = mul_signed(c3, w2);
        const int b2 = b3 + P::pos(a0[1], i2) * estep[1];
        u128 v[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) v[i] = mul_signed(c2, w1[i]);
        // merge the left neighbour's second samples into my first ones
        const u128 sA = bsf_shfl_up(v[PA1], 1), sB = bsf_shfl_up(v[PB1], 1);
        if (from_left) {
          v[PA0] += sA;
          v[PB0] += sB;
        }
        if (to_right) {
          v[PA1] = 0;
          v[PB1] = 0;
        }
        // 128-bit adds: every low word first, then the high words with carries
        unsigned long long old[NP], lo[NP], hi[NP];
        unsigned long long* q[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          q[i] = reinterpret_cast<unsigned long long*>(G + b2 + off1[i]);
          lo[i] = (unsigned long long)v[i];
          hi[i] = (unsigned long long)(v[i] >> 64);
          old[i] = (in && v[i] != 0) ? atomicAdd(q[i], lo[i]) : 0ull;
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          if (!in || v[i] == 0) continue;
          const unsigned long long h = hi[i] + ((old[i] + lo[i] < old[i]) ? 1ull : 0ull);
          if (h) atomicAdd(q[i] + 1, h);
        }
      }
    }
  }
}

// Extension fold of the 128-bit adjoint sums: columns, then rows with the
// final rounding RN32(acc) 2^-qg.
template <typename F>
__device__ __forceinline__ void for_preimages128(int i, int N, int R, int boundary, F&& f) {
  if (boundary == BSF_ZERO) {
    f(i + R);
  } else if (boundary == BSF_REPLICATE) {
    const int lo = i == 0 ? -R : i, hi = i == N - 1 ? N - 1 + R : i;
    for (int z = lo; z <= hi; ++z) f(z + R);
  } else {
    const int P2 = 2 * N;
    for (int fam = 0; fam < 2; ++fam) {
      const int b = fam == 0 ? i : P2 - 1 - i;
      int z = b - ((b + R + P2 - 1) / P2) * P2;
      if (z < -R) z += P2;
      for (; z < N + R; z += P2) f(z + R);
    }
  }
}

// Both folds at once (see the 64-bit form): interior pixels read one element.
__global__ void k_fold_xy_out128(const u128* __restrict__ G, long long pitch, int H, int W, int R,
                                 int boundary, float* __restrict__ gimg, long long ldo,
                                 const DevStatus* st) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= W || y >= H) return;
  u128 acc = 0;
  if (x >= R && x < W - R && y >= R && y < H - R) {
    acc = bsf_load(G + (long long)(y + R) * pitch + (x + R));
  } else {
    for_preimages128(y, H, R, boundary, [&](int yp) {
      const u128* row = G + (long long)yp * pitch;
      for_preimages128(x, W, R, boundary, [&](int xp) { acc += bsf_load(row + xp); });
    });
  }
  const int qg = grad_q128(st->max_absg_bits);
  gimg[(long long)y * ldo + x] = __fmul_rn(bsf_rn32((i128)acc), bsf_pow2_f32(-qg));
}

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

cudaError_t bsf_launch_scatter_d2(int n, void* G, long long pitch, int R, const float* cov,
                                  int cov_kind, const float* gout, long long ldg, int H, int W,
                                  int row0, int rows, int qg, DevStatus* st, cudaStream_t s) {
  const dim3 block(32, 4), grid((W + 31) / 32, (rows + 3) / 4);
  if (n == 1)
    k_scatter_d2<1><<<grid, block, 0, s>>>((u128*)G, pitch, R, cov, cov_kind, gout, ldg, H, W, row0, rows, qg,
                                           st);
  else if (n == 2)
    k_scatter_d2<2><<<grid, block, 0, s>>>((u128*)G, pitch, R, cov, cov_kind, gout, ldg, H, W, row0, rows, qg,
                                           st);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t bsf_launch_fold128(const void* G, long long pitch, int Hp, int H, int W, int R,
                               int boundary, void* Gx, float* gimg, long long ldo, const DevStatus* st,
                               cudaStream_t s) {
  (void)Hp;
  (void)Gx;
  dim3 blk(128);
  k_fold_xy_out128<<<dim3((W + 127) / 128, H), blk, 0, s>>>((const u128*)G, pitch, H, W, R, boundary,
                                                             gimg, ldo, st);
  return cudaGetLastError();
}
