// Dispatch of the continuous-step stencil by element type, and the
// vector-Jacobian product kernel.  The stencil itself is in bsf_continuous.cuh.
#include <climits>

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

// Adjoint of the continuous-step taps: each pixel adds g(p) times the
// product of its four interpolation weights at each of its samples, g(p) =
// RNE(RN32(RN32(gout 2^qg) / RN32(M))) the quantised normalised weight.
// Pixels of image rows [row0, row0 + rows) scatter into G, whose padded row
// 0 is image row row0 - R (the whole image: row0 = 0, rows = H); qg_given >=
// 0 fixes the fraction bits of the weights, -1 takes them from the device
// maximum of |gout|.

// One pixel's weight g and its interpolation brackets a0 / fractions th per
// direction (identity steps for pixels outside the image or the band).
template <int NF>
__device__ __forceinline__ u128 scatter_pixel(const float* __restrict__ cov, int kind,
                                              const float* __restrict__ gout, long long ldg, int H, int W,
                                              int R, int row0, int x, int y, bool in, int qg_given,
                                              DevStatus* st, int a0[4], unsigned th[4]) {
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
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int Q0 = NF == 2 ? 2 * Hq[k] - 1024 : Hq[k] - 512;
    a0[k] = Q0 >> 10;
    th[k] = (unsigned)(Q0 & 1023);
  }
  return g;
}

// The block's pixels (a tile of kWinTX x kWinTY) first sum their samples in
// a window of G held in shared memory, then add the window to G: neighbouring
// pixels' samples fall on the same cells (the fields are smooth, and the 625
// samples of a pixel sweep a box a few steps wide), so each global 128-bit
// add carries the sum of many samples.  The window is the bounding box of
// the tile's samples; a box taller than the window's capacity is covered in
// row bands, one pass each, every pixel adding only its samples that fall in
// the band.  A box that would need more than kWinMaxPasses bands falls back
// to the direct global adds.  Shared words: low and high 64-bit planes of
// 128-bit cells, the low add returning the old word for the carry.
constexpr int kWinTX = 32, kWinTY = 8;
constexpr int kWinCells = 4096;     // 64 KB: three blocks per SM (measured best of 2,048-12,288 cells)
constexpr int kWinMaxPasses = 8;

// Sample offsets along one direction: [lo, hi] (a0 >= -1).
template <int NF> __device__ __forceinline__ int pos_lo(int a0) { return NF == 2 ? -a0 - 3 : -a0 - 2; }
__device__ __forceinline__ int pos_hi(int a0) { return a0 + 1; }

// Sample i of one direction's adjoint for coefficient c, from u = 1024 c
// and t = th c: n = 2 weights 1024 - th, th, -2048, th, 1024 - th; n = 1
// 1024 - th, th, -th, th - 1024 (all modulo 2^128).
template <int NF> __device__ __forceinline__ u128 dir_value(u128 u, u128 t, int i) {
  if (NF == 2) return i == 1 || i == 3 ? t : (i == 2 ? (u128)0 - (u << 1) : u - t);
  return i == 0 ? u - t : (i == 1 ? t : (i == 2 ? (u128)0 - t : t - u));
}

// One pixel's samples whose rows fall in [0, nr) of a target laid out in
// rows of `stride` 64-bit word pairs: the shared window (low and high words
// in two planes, `hi_off` words apart) or G itself (interleaved 128-bit
// cells: stride 2 pitch, hi_off 1, every row in range).  Row and column of
// the pixel relative to the target origin: ry, rx.  The low-word add returns
// the old word, whose carry goes into the high word's add.
template <int NF>
__device__ __forceinline__ void deposit_samples(unsigned long long* __restrict__ tgt, int stride, int cellw,
                                                int hi_off, int nr, int ry, int rx, u128 u4, u128 t4,
                                                const int a0[4], const unsigned th[4]) {
  using P = Pattern<NF>;
  constexpr int NP = P::NP;
  int off1[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) off1[i] = P::pos(a0[0], i) * cellw;
  const int d2lo = pos_lo<NF>(a0[1]), d2hi = pos_hi(a0[1]);
#pragma unroll 1
  for (int i4 = 0; i4 < NP; ++i4) {
    const int p4 = P::pos(a0[3], i4);
    const u128 c4 = dir_value<NF>(u4, t4, i4);
    const u128 u3 = c4 << 10, t3 = mul_small(c4, th[2]);
#pragma unroll 1
    for (int i3 = 0; i3 < NP; ++i3) {
      const int r3 = ry + p4 + P::pos(a0[2], i3);
      if (r3 + d2hi < 0 || r3 + d2lo >= nr) continue;  // no d2 sample of the group in range
      const u128 c3 = dir_value<NF>(u3, t3, i3);
      const u128 u2 = c3 << 10, t2 = mul_small(c3, th[1]);
#pragma unroll
      for (int i2 = 0; i2 < NP; ++i2) {
        const int p2 = P::pos(a0[1], i2);
        const int r = r3 + p2;
        if ((unsigned)r >= (unsigned)nr) continue;
        const u128 c2 = dir_value<NF>(u2, t2, i2);
        const u128 u1 = c2 << 10, t1 = mul_small(c2, th[0]);
        unsigned long long* q = tgt + (long long)r * stride + (rx + p2 - p4) * cellw;
        // the samples' words are recomputed for the high adds (fewer live registers)
        unsigned long long old[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) old[i] = atomicAdd(q + off1[i], (unsigned long long)dir_value<NF>(u1, t1, i));
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          const u128 v = dir_value<NF>(u1, t1, i);
          const unsigned long long lo = (unsigned long long)v;
          const unsigned long long h = (unsigned long long)(v >> 64) + ((old[i] + lo < old[i]) ? 1ull : 0ull);
          if (h) atomicAdd(q + off1[i] + hi_off, h);
        }
      }
    }
  }
}

template <int NF>
__global__ void __launch_bounds__(kWinTX * kWinTY, 3)
k_scatter_d2(u128* __restrict__ G, long long pitch, int R, const float* __restrict__ cov, int kind,
             const float* __restrict__ gout, long long ldg, int H, int W, int row0, int rows, int qg_given,
             DevStatus* st) {
  using P = Pattern<NF>;
  constexpr int NP = P::NP;
  constexpr int NT = kWinTX * kWinTY;
  extern __shared__ unsigned long long win_lo[];  // [kWinCells] low words, then [kWinCells] high words
  unsigned long long* win_hi = win_lo + kWinCells;
  __shared__ int box[4];                          // x0, -x1, y0, -y1
  const int lane = threadIdx.x, tid = threadIdx.y * kWinTX + lane;
  const int x = blockIdx.x * kWinTX + lane;
  const int y = blockIdx.y * kWinTY + threadIdx.y;
  const bool in = x < W && y < rows;
  int a0[4];
  unsigned th[4];
  const u128 g = scatter_pixel<NF>(cov, kind, gout, ldg, H, W, R, row0, x, y, in, qg_given, st, a0, th);
  const int p32 = (int)pitch;
  const int cx = x + R, cy = y + R;  // the pixel in padded coordinates
  // bounding box of the samples of the block's pixels: d1 = (1, 0),
  // d2 = (1, 1), d3 = (0, 1), d4 = (-1, 1)
  if (tid == 0) box[0] = box[1] = box[2] = box[3] = INT_MAX;
  __syncthreads();
  int bx0 = INT_MAX, bx1 = INT_MAX, by0 = INT_MAX, by1 = INT_MAX;  // x0, -x1, y0, -y1
  if (in) {
    bx0 = cx + pos_lo<NF>(a0[0]) + pos_lo<NF>(a0[1]) - pos_hi(a0[3]);
    bx1 = -(cx + pos_hi(a0[0]) + pos_hi(a0[1]) - pos_lo<NF>(a0[3]));
    by0 = cy + pos_lo<NF>(a0[1]) + pos_lo<NF>(a0[2]) + pos_lo<NF>(a0[3]);
    by1 = -(cy + pos_hi(a0[1]) + pos_hi(a0[2]) + pos_hi(a0[3]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bx0 = min(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
    bx1 = min(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
    by0 = min(by0, __shfl_xor_sync(0xffffffffu, by0, o));
    by1 = min(by1, __shfl_xor_sync(0xffffffffu, by1, o));
  }
  if (lane == 0 && bx0 != INT_MAX) {
    atomicMin(&box[0], bx0);
    atomicMin(&box[1], bx1);
    atomicMin(&box[2], by0);
    atomicMin(&box[3], by1);
  }
  __syncthreads();
  if (box[0] == INT_MAX) return;  // no pixel of the block in the image (uniform)
  const int X0 = box[0], X1 = -box[1], Y0 = box[2], Y1 = -box[3];
  const int Ww = X1 - X0 + 1, band = kWinCells / Ww;
  // each direction's weights are 1024 base_i + th diff_i: per coefficient c
  // one product t = th c and the shift u = 1024 c give all of its samples
  const u128 u4 = g << 10, t4 = mul_small(g, th[3]);
  const bool live = in && g != 0;
  if (band < 1 || (Y1 - Y0 + band) / band > kWinMaxPasses) {  // direct adds into G
    if (live)
      deposit_samples<NF>(reinterpret_cast<unsigned long long*>(G), 2 * p32, 2, 1, INT_MAX / 2, cy, cx,
                          u4, t4, a0, th);
    return;
  }
  for (int Yb = Y0; Yb <= Y1; Yb += band) {
    const int nr = min(band, Y1 - Yb + 1), ncell = nr * Ww;
    for (int c = tid; c < ncell; c += NT) {
      win_lo[c] = 0ull;
      win_hi[c] = 0ull;
    }
    __syncthreads();
    if (live) deposit_samples<NF>(win_lo, Ww, 1, kWinCells, nr, cy - Yb, cx - X0, u4, t4, a0, th);
    __syncthreads();
    // the band into G: low words first, then the high words with carries
    constexpr int KF = 4;
    for (int c0 = tid; c0 < ncell; c0 += KF * NT) {
      unsigned long long old[KF], lo[KF], hi[KF];
      unsigned long long* q[KF];
#pragma unroll
      for (int k = 0; k < KF; ++k) {
        const int c = c0 + k * NT;
        lo[k] = hi[k] = 0ull;
        q[k] = nullptr;
        if (c < ncell) {
          lo[k] = win_lo[c];
          hi[k] = win_hi[c];
          const int r = c / Ww;
          q[k] = reinterpret_cast<unsigned long long*>(G + (long long)(Yb + r) * pitch + X0 + (c - r * Ww));
        }
        old[k] = lo[k] ? atomicAdd(q[k], lo[k]) : 0ull;
      }
#pragma unroll
      for (int k = 0; k < KF; ++k) {
        const unsigned long long h = hi[k] + ((old[k] + lo[k] < old[k]) ? 1ull : 0ull);
        if (h) atomicAdd(q[k] + 1, h);
      }
    }
    __syncthreads();
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
  bsf_grid_dep_wait();  // a programmatic dependent of the last suffix sums
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
  const dim3 block(kWinTX, kWinTY), grid((W + kWinTX - 1) / kWinTX, (rows + kWinTY - 1) / kWinTY);
  const size_t smem = 2 * kWinCells * sizeof(unsigned long long);
  static bool attr_set[2] = {false, false};
  if (n != 1 && n != 2) return cudaErrorInvalidValue;
  if (!attr_set[n - 1]) {
    const cudaError_t e = n == 1
        ? cudaFuncSetAttribute(k_scatter_d2<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
        : cudaFuncSetAttribute(k_scatter_d2<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set[n - 1] = true;
  }
  if (n == 1)
    k_scatter_d2<1><<<grid, block, smem, s>>>((u128*)G, pitch, R, cov, cov_kind, gout, ldg, H, W, row0, rows,
                                              qg, st);
  else
    k_scatter_d2<2><<<grid, block, smem, s>>>((u128*)G, pitch, R, cov, cov_kind, gout, ldg, H, W, row0, rows,
                                              qg, st);
  return cudaGetLastError();
}

cudaError_t bsf_launch_fold128(const void* G, long long pitch, int Hp, int H, int W, int R,
                               int boundary, void* Gx, float* gimg, long long ldo, const DevStatus* st,
                               cudaStream_t s) {
  (void)Hp;
  (void)Gx;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((W + 127) / 128, H);
  cfg.blockDim = dim3(128);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fold_xy_out128, (const u128*)G, pitch, H, W, R, boundary, gimg, ldo, st);
}
