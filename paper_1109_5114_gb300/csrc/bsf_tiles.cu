// Tile-restarted pre-integration fused with the finite differences: the
// whole integer-step filter of one output tile in one thread block.
//
// The pipeline of Section 1.1 is exact on any domain that holds every tap:
// running sums that start from zero at the domain's edge and the order-n
// differences of their samples give the window sums of the kernel whatever
// lies outside.  So each block takes its own domain: the T x T output tile
// plus the reach R on every side, P = T + 2R.  It loads the extended,
// quantised image window into shared memory, runs the n-fold running sums
// along d1, d3, d2, d4 there (one thread per row, column or diagonal line,
// the n folds in registers), and evaluates the (n+1)^4 taps of every output
// pixel from shared memory.  No running sums go through HBM: the block reads
// the image window, the covariance of its tile, and writes its outputs.  The
// windows of neighbouring tiles overlap by 2R, so the scans do P^2/T^2 times
// the work of one global pass, in shared memory.
//
// The sums of a window are bounded by the window, not the image, so the
// floating-point variants (float64 sums, compensated float32 sums) keep far
// more of their accuracy on large images;
// the fixed-point bound max|Q| prod L^n < 2^(b-1) is checked against the
// window's own max|Q|.
#include "bsf_quantize.cuh"
#include "bsf_stencil.cuh"

namespace {

template <typename T>
__device__ __forceinline__ T load_quantized(const void* img, int dtype, long long idx, int q, float scale_f,
                                            bool& ok, float& ax) {
  if (dtype == BSF_U8) return quantize_one<T, uint8_t>(static_cast<const uint8_t*>(img)[idx], q, scale_f, ok, ax);
  if (dtype == BSF_F32) return quantize_one<T, float>(static_cast<const float*>(img)[idx], q, scale_f, ok, ax);
  return quantize_one<T, double>(static_cast<const double*>(img)[idx], q, scale_f, ok, ax);
}

// One walk along a line of the window: the n-fold running sum of the
// elements at S[i0], S[i0 + step], ... (m of them), in place.
template <typename T, int NF>
__device__ __forceinline__ void walk(T* S, int i0, int step, int m) {
  T a[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) a[f] = (T)0;
  int i = i0;
#pragma unroll 4
  for (int j = 0; j < m; ++j, i += step) {
    a[0] += S[i];
#pragma unroll
    for (int f = 1; f < NF; ++f) a[f] += a[f - 1];
    S[i] = a[NF - 1];
  }
}

// The n-fold running sums of the second direction set over the window:
// along e = (ex, ey), ey in {1, 2}, every line starts at a point whose
// predecessor (x - ex, y - ey) lies outside the window: the first ey rows,
// and the |ex| columns at the side the line comes from.
template <typename T, int NF>
__device__ __forceinline__ void walks_second(T* S, int P, int pitch, int ex, int ey, int tid, int nthr) {
  const int ax = ex < 0 ? -ex : ex;
  const int side = (P - ey) * ax;  // starts on the side columns below the first ey rows
  for (int i = tid; i < ey * P + side; i += nthr) {
    int x0, y0;
    if (i < ey * P) {
      y0 = i / P;
      x0 = i - y0 * P;
    } else {
      const int j = i - ey * P;
      y0 = ey + j / ax;
      const int c = j - (j / ax) * ax;
      x0 = ex > 0 ? c : P - 1 - c;
    }
    const int my = (P - 1 - y0) / ey + 1;
    const int mx = ex > 0 ? (P - 1 - x0) / ex + 1 : x0 / ax + 1;
    walk<T, NF>(S, y0 * pitch + x0, ey * pitch + ex, my < mx ? my : mx);
  }
}

template <typename T, int NF, int DS> struct TileOcc {
  static constexpr int value = (sizeof(T) <= 8 && NF <= 2 && DS != BSF_DIRS_PAIR) ? 2 : 1;
};

// DS (BSF_DIRS_*): the Cartesian set on S; the second set on S; or the pair,
// the Cartesian sums on S and the second set's on S2 = S + P pitch (both
// windows in shared memory), chosen per pixel by sector.
template <typename T, int NF, typename Out, int DS>
__global__ void __launch_bounds__(512, (TileOcc<T, NF, DS>::value))
k_tile_filter(const void* __restrict__ img, int dtype, long long ld, int H, int W, int R, int boundary,
              int row0, int rows, int TT, int q, float qscale, float scale_f, double scale_d,
              const float* __restrict__ cov, int kind, int rule, Out* __restrict__ out, long long ldo,
              DevStatus* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);
  __shared__ float s_max[16];
  const int P = TT + 2 * R;
  const int pitch = P | 1;  // odd: the column and diagonal walks hit distinct banks
  T* S2 = DS == BSF_DIRS_PAIR ? S + (size_t)P * pitch : S;
  const int x0 = blockIdx.x * TT, y0 = row0 + blockIdx.y * TT;
  const int tid = threadIdx.x, nthr = blockDim.x;

  // 1. the extended, quantised window: image rows y0 - R .. y0 + TT + R - 1
  float amax = 0.f;
  bool ok = true;
  for (int i = tid; i < P * P; i += nthr) {
    const int py = i / P, px = i - py * P;
    bool vy, vx;
    const int ys = bsf_map_index(y0 - R + py, H, boundary, vy);
    const int xs = bsf_map_index(x0 - R + px, W, boundary, vx);
    T v = (T)0;
    if (vy && vx) {
      bool ok1;
      float ax;
      v = load_quantized<T>(img, dtype, (long long)ys * ld + xs, q, qscale, ok1, ax);
      ok &= ok1;
      amax = fmaxf(amax, ax);
    }
    S[py * pitch + px] = v;
    if constexpr (DS == BSF_DIRS_PAIR) S2[py * pitch + px] = v;
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((tid & 31) == 0) s_max[tid >> 5] = amax;
  const int any_bad = __syncthreads_or(!ok);
  float wmax = s_max[0];
  for (int w = 1; w < (nthr >> 5); ++w) wmax = fmaxf(wmax, s_max[w]);
  if (tid == 0) {
    if (wmax > 0.f) bsf_atomic_max_pos_float(&st->max_absq_bits, wmax);
    if (any_bad) bsf_set_error(st, BSF_EOVERFLOW);
  }

  // 2. running sums of the window: d1 along rows, d3 down columns, d2 and
  // d4 down the diagonals (lines x - y and x + y); the second set along
  // e1 = (2,1), e2 = (1,2), e3 = (-1,2), e4 = (-2,1)
  if constexpr (DS != BSF_DIRS_SECOND) {
    for (int r = tid; r < P; r += nthr) walk<T, NF>(S, r * pitch, 1, P);
    __syncthreads();
    for (int c = tid; c < P; c += nthr) walk<T, NF>(S, c, pitch, P);
    __syncthreads();
    for (int i = tid; i < 2 * P - 1; i += nthr) {
      const int u = i - (P - 1);  // x - y
      const int ya = u < 0 ? -u : 0, yb = u > 0 ? P - 1 - u : P - 1;
      walk<T, NF>(S, ya * pitch + (u + ya), pitch + 1, yb - ya + 1);
    }
    __syncthreads();
    for (int u = tid; u < 2 * P - 1; u += nthr) {  // x + y
      const int ya = u > P - 1 ? u - (P - 1) : 0, yb = u < P - 1 ? u : P - 1;
      walk<T, NF>(S, ya * pitch + (u - ya), pitch - 1, yb - ya + 1);
    }
    __syncthreads();
  }
  if constexpr (DS != BSF_DIRS_CARTESIAN) {
    walks_second<T, NF>(S2, P, pitch, 2, 1, tid, nthr);
    __syncthreads();
    walks_second<T, NF>(S2, P, pitch, 1, 2, tid, nthr);
    __syncthreads();
    walks_second<T, NF>(S2, P, pitch, -1, 2, tid, nthr);
    __syncthreads();
    walks_second<T, NF>(S2, P, pitch, -2, 1, tid, nthr);
    __syncthreads();
  }

  // 3. the taps of every output pixel of the tile, from shared memory
  const float maxq = wmax + 1.f;
  const long long HW = (long long)H * W;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  for (int ty = warp; ty < TT; ty += nw) {
    const int y = y0 + ty;
    if (y >= row0 + rows) break;
    for (int tx = lane; tx < TT; tx += 32) {
      const int x = x0 + tx;
      if (x >= W) break;
      int L[4], flags, reach;
      float C11, C12, C22;
      bsf_solve::load_cov(cov, kind, HW, (long long)y * W + x, C11, C12, C22);
      bool second = false, in_reach;
      if constexpr (DS == BSF_DIRS_CARTESIAN)
        in_reach = bsf_solve::pixel_steps(C11, C12, C22, NF, rule, R, L, flags, reach);
      else
        in_reach = bsf_solve::pixel_steps_set(DS, C11, C12, C22, NF, rule, R, L, flags, reach, second);
      count_pixel_flags(flags, in_reach, st);
      const int c1 = NF * (L[0] - 1) / 2, c2 = NF * (L[1] - 1) / 2, c3 = NF * (L[2] - 1) / 2,
                c4 = NF * (L[3] - 1) / 2;
      int e1 = 1, e2 = pitch + 1, e3 = pitch, e4 = pitch - 1;
      const T* Sp = S;
      if constexpr (DS != BSF_DIRS_CARTESIAN) {
        if (second) {
          e1 = pitch + 2; e2 = 2 * pitch + 1; e3 = 2 * pitch - 1; e4 = pitch - 2;
          Sp = S2;
        }
      }
      const int base = (ty + R) * pitch + (tx + R) + c1 * e1 + c2 * e2 + c3 * e3 + c4 * e4;
      const int s[4] = {L[0] * e1, L[1] * e2, L[2] * e3, L[3] * e4};
      const T acc = comb<T, NF, 4, true>(Sp, base, s);
      finish_pixel<T, NF, Out>(acc, L, maxq, scale_f, scale_d, out + (long long)(y - row0) * ldo + x, st);
    }
  }
}

size_t tile_bytes(int TT, int R, int elem) {
  const size_t P = (size_t)TT + 2 * (size_t)R;
  return P * (P | 1) * (size_t)elem;
}

template <typename T, int NF, typename Out, int DS>
cudaError_t launch_tiles_t(const void* img, int dtype, long long ld, int H, int W, int R, int boundary,
                           int row0, int rows, int TT, int q, const float* cov, int kind, int rule, void* out,
                           long long ldo, DevStatus* st, cudaStream_t s) {
  const size_t smem = tile_bytes(TT, R, sizeof(T)) * (DS == BSF_DIRS_PAIR ? 2 : 1);
  cudaError_t e = cudaFuncSetAttribute(k_tile_filter<T, NF, Out, DS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((W + TT - 1) / TT, (rows + TT - 1) / TT);
  // q <= 100: 2^q and 2^-q are normal float32
  k_tile_filter<T, NF, Out, DS><<<grid, 512, smem, s>>>(img, dtype, ld, H, W, R, boundary, row0, rows, TT, q,
                                                    ldexpf(1.f, q), ldexpf(1.f, -q), ldexp(1.0, -q), cov, kind,
                                                    rule, (Out*)out, ldo, st);
  return cudaGetLastError();
}

template <typename T, int NF, int DS>
cudaError_t launch_tiles_o(int out_dtype, const void* img, int dtype, long long ld, int H, int W, int R,
                           int boundary, int row0, int rows, int TT, int q, const float* cov, int kind, int rule,
                           void* out, long long ldo, DevStatus* st, cudaStream_t s) {
  if (out_dtype == BSF_F32)
    return launch_tiles_t<T, NF, float, DS>(img, dtype, ld, H, W, R, boundary, row0, rows, TT, q, cov, kind, rule,
                                            out, ldo, st, s);
  if (out_dtype == BSF_F64)
    return launch_tiles_t<T, NF, double, DS>(img, dtype, ld, H, W, R, boundary, row0, rows, TT, q, cov, kind, rule,
                                             out, ldo, st, s);
  return cudaErrorInvalidValue;
}

template <typename T, int NF>
cudaError_t launch_tiles_d(int dirset, int out_dtype, const void* img, int dtype, long long ld, int H, int W, int R,
                           int boundary, int row0, int rows, int TT, int q, const float* cov, int kind, int rule,
                           void* out, long long ldo, DevStatus* st, cudaStream_t s) {
  if (dirset == BSF_DIRS_CARTESIAN)
    return launch_tiles_o<T, NF, BSF_DIRS_CARTESIAN>(out_dtype, img, dtype, ld, H, W, R, boundary, row0, rows, TT,
                                                     q, cov, kind, rule, out, ldo, st, s);
  if constexpr (IsFixed<T>::value) {  // the direction sets: fixed point only
    if (dirset == BSF_DIRS_SECOND)
      return launch_tiles_o<T, NF, BSF_DIRS_SECOND>(out_dtype, img, dtype, ld, H, W, R, boundary, row0, rows, TT, q,
                                                    cov, kind, rule, out, ldo, st, s);
    if (dirset == BSF_DIRS_PAIR)
      return launch_tiles_o<T, NF, BSF_DIRS_PAIR>(out_dtype, img, dtype, ld, H, W, R, boundary, row0, rows, TT, q,
                                                  cov, kind, rule, out, ldo, st, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int bsf_tile_size(int prec, int R, int max_smem, int windows) {
  const int elem = (prec == BSF_FIX32 ? 4 : (prec == BSF_FIX128 ? 16 : 8)) * windows;
  // two blocks per SM when a tile of at least 64 fits in half of the shared
  // memory, else one block with the largest tile of at least 64
  static const int sizes[3] = {128, 96, 64};
  for (int TT : sizes)
    if (tile_bytes(TT, R, elem) <= (size_t)max_smem / 2 - 1024) return TT;
  for (int TT : sizes)
    if (tile_bytes(TT, R, elem) <= (size_t)max_smem - 1024) return TT;
  return 0;
}

cudaError_t bsf_launch_tiles(int prec, int n, int dirset, const void* img, int dtype, long long ld, int H, int W,
                             int R, int boundary, int row0, int rows, int TT, int q, const float* cov, int cov_kind,
                             int rule, void* out, int out_dtype, long long ldo, DevStatus* st, cudaStream_t s) {
  if (TT <= 0 || TT % 32 != 0) return cudaErrorInvalidValue;
#define BSF_TL(T, NF) \
  return launch_tiles_d<T, NF>(dirset, out_dtype, img, dtype, ld, H, W, R, boundary, row0, rows, TT, q, cov, \
                               cov_kind, rule, out, ldo, st, s)
  switch (prec * 10 + n) {
    case 51: BSF_TL(uint32_t, 1);
    case 52: BSF_TL(uint32_t, 2);
    case 53: BSF_TL(uint32_t, 3);
    case 11: BSF_TL(uint64_t, 1);
    case 12: BSF_TL(uint64_t, 2);
    case 13: BSF_TL(uint64_t, 3);
    case 21: BSF_TL(u128, 1);
    case 22: BSF_TL(u128, 2);
    case 23: BSF_TL(u128, 3);
    case 31: BSF_TL(double, 1);
    case 32: BSF_TL(double, 2);
    case 33: BSF_TL(double, 3);
    case 41: BSF_TL(f32x2, 1);
    case 42: BSF_TL(f32x2, 2);
    case 43: BSF_TL(f32x2, 3);
    default: return cudaErrorInvalidValue;
  }
#undef BSF_TL
}
