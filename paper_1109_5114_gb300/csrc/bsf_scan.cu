// Pre-integration: n-fold running sums along d1, d3, d2, d4 (Section 1.1, the
// running sum; the recursion form of Algorithm 3, step 2) on the padded domain
// P = [-R, W+R) x [-R, H+R), in exact modular integer arithmetic.
//
//   d1 = (1, 0): k_scan_rows -- one block per padded row.  The same pass
//       extends the image by the boundary rule and quantises it,
//       Q(f) = round-half-even(f 2^q), so the input is read once.
//   d3 = (0, 1), d2 = (1, 1), d4 = (-1, 1): the lines move one row down per
//       step and 0, +1 or -1 column across.  In skewed coordinates
//       u = x - skew * y every line is a column, so one thread owns one line
//       and a warp reads 32 consecutive x of a row (coalesced).  Rows are cut
//       into chunks of kScanChunk rows, scanned in three phases:
//         agg   -- per (line, chunk): the n-fold state at the chunk's end
//                  with zero carry-in;
//         carry -- per line: combine the chunk states in order; the state
//                  after a chunk of m rows is
//                  s'_f = sum_{j<=f} C(m-1+j, j) s_{f-j} + agg_f;
//         apply -- per (line, chunk): rescan with the carried-in state and
//                  write the result in place.
//       No block waits on another block.
//
// Arithmetic wraps modulo 2^64 or 2^128 (the element type), which the final
// finite differences cancel exactly.
#include "bsf_device.cuh"

namespace {

// ---------------------------------------------------------------------------
// d1 with fused extension + quantisation: one block of kRowThreads per padded
// row; each thread owns V consecutive elements of a chunk of kRowThreads * V.
// A fold is a thread-local scan, a warp shuffle scan of the thread totals, a
// block scan of the warp totals through shared memory, and a carry per row.
// ---------------------------------------------------------------------------
constexpr int kRowThreads = 256;

template <typename T, typename In>
__device__ __forceinline__ T quantize_one(In fv, int q, float scale_f, bool& ok, float& ax) {
  if constexpr (sizeof(In) == 1) {
    ok = true;
    ax = (float)fv * scale_f;
    return (T)fv << q;
  } else if constexpr (sizeof(In) == 4) {
    ax = fabsf(fv) * scale_f;  // exact unless it overflows to inf (then ok is false too)
    return bsf_quantize_f32<T>(fv, q, ok);
  } else {
    const double xq = (double)fv * (double)scale_f;
    ax = __double2float_ru(fabs(xq));
    return bsf_round_to_elem<T>(xq, ok);
  }
}

template <typename T, int NF, typename In, int V>
__global__ void __launch_bounds__(kRowThreads)
k_scan_rows(const In* __restrict__ img, long long ld, int H, int W, int R, int boundary,
            float scale_f, int q, T* __restrict__ S, long long pitch, int Hp, int Wp,
            DevStatus* st) {
  constexpr int NW = kRowThreads / 32;
  __shared__ T s_warp[NF][NW];
  const int yp = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  bool yvalid;
  const int ys = bsf_map_index(yp - R, H, boundary, yvalid);
  const In* src = img + (long long)ys * ld;
  T* row = S + (long long)yp * pitch;
  T carry[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) carry[f] = 0;
  float amax = 0.f;
  bool all_ok = true;
  for (int x0 = 0; x0 < Wp; x0 += kRowThreads * V) {
    T v[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int xp = x0 + tid * V + j;
      v[j] = 0;
      if (xp < Wp && yvalid) {
        bool xvalid;
        const int xs = bsf_map_index(xp - R, W, boundary, xvalid);
        if (xvalid) {
          bool ok;
          float ax;
          v[j] = quantize_one<T, In>(src[xs], q, scale_f, ok, ax);
          all_ok &= ok;
          amax = fmaxf(amax, ax);
        }
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
#pragma unroll
      for (int j = 1; j < V; ++j) v[j] += v[j - 1];
      const T tot = v[V - 1];
      T incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const T t = bsf_shfl_up(incl, o);
        if (lane >= o) incl += t;
      }
      if (lane == 31) s_warp[f][wid] = incl;
      __syncthreads();
      T wpre = 0, btot = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const T t = s_warp[f][w];
        if (w < wid) wpre += t;
        btot += t;
      }
      const T add = carry[f] + wpre + (incl - tot);
#pragma unroll
      for (int j = 0; j < V; ++j) v[j] += add;
      carry[f] += btot;
    }
    __syncthreads();  // s_warp is rewritten by the next chunk
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int xp = x0 + tid * V + j;
      if (xp < Wp) row[xp] = v[j];
    }
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const bool bad = __any_sync(0xffffffffu, !all_ok);
  if (lane == 0) {
    bsf_atomic_max_pos_float(&st->max_absq_bits, amax);
    if (bad) bsf_set_error(st, BSF_EOVERFLOW);
  }
}

// ---------------------------------------------------------------------------
// d3 / d2 / d4 in skewed coordinates
// ---------------------------------------------------------------------------
template <typename T, int NF, int SKEW>
__global__ void __launch_bounds__(128)
k_vscan_agg(const T* __restrict__ S, long long pitch, int Hp, int Wp, int umin, int Nu,
            T* __restrict__ agg) {
  const int ui = blockIdx.x * blockDim.x + threadIdx.x;
  if (ui >= Nu) return;
  const int u = umin + ui;
  const int c = blockIdx.y;
  const int y0 = c * kScanChunk, y1 = min(y0 + kScanChunk, Hp);
  T s[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) s[f] = 0;
#pragma unroll 8
  for (int y = y0; y < y1; ++y) {
    const int x = u + SKEW * y;
    T v = 0;
    if (x >= 0 && x < Wp) v = S[(long long)y * pitch + x];
    s[0] += v;
#pragma unroll
    for (int f = 1; f < NF; ++f) s[f] += s[f - 1];
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) agg[((long long)c * NF + f) * Nu + ui] = s[f];
}

template <typename T, int NF>
__global__ void __launch_bounds__(128)
k_vscan_carry(const T* __restrict__ agg, T* __restrict__ carry, int nchunks, int Hp, int Nu) {
  const int ui = blockIdx.x * blockDim.x + threadIdx.x;
  if (ui >= Nu) return;
  T s[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) s[f] = 0;
#pragma unroll 8
  for (int c = 0; c < nchunks; ++c) {
    T a[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      carry[((long long)c * NF + f) * Nu + ui] = s[f];
      a[f] = agg[((long long)c * NF + f) * Nu + ui];
    }
    const T m = (T)min(kScanChunk, Hp - c * kScanChunk);
    // state after m zero-input steps plus the chunk's own contribution
    T ns[NF];
    ns[0] = s[0] + a[0];
    if constexpr (NF >= 2) ns[1] = s[1] + m * s[0] + a[1];
    if constexpr (NF >= 3) ns[2] = s[2] + m * s[1] + ((m * (m + 1)) >> 1) * s[0] + a[2];
#pragma unroll
    for (int f = 0; f < NF; ++f) s[f] = ns[f];
  }
}

template <typename T, int NF, int SKEW>
__global__ void __launch_bounds__(128)
k_vscan_apply(T* __restrict__ S, long long pitch, int Hp, int Wp, int umin, int Nu,
              const T* __restrict__ carry) {
  const int ui = blockIdx.x * blockDim.x + threadIdx.x;
  if (ui >= Nu) return;
  const int u = umin + ui;
  const int c = blockIdx.y;
  const int y0 = c * kScanChunk, y1 = min(y0 + kScanChunk, Hp);
  // skip lines that do not cross this chunk
  const int xa = u + SKEW * y0, xb = u + SKEW * (y1 - 1);
  if (max(xa, xb) < 0 || min(xa, xb) >= Wp) return;
  T s[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) s[f] = carry[((long long)c * NF + f) * Nu + ui];
#pragma unroll 8
  for (int y = y0; y < y1; ++y) {
    const int x = u + SKEW * y;
    const bool in = x >= 0 && x < Wp;
    T* p = S + (long long)y * pitch + x;
    T v = 0;
    if (in) v = *p;
    s[0] += v;
#pragma unroll
    for (int f = 1; f < NF; ++f) s[f] += s[f - 1];
    if (in) *p = s[NF - 1];
  }
}

template <typename T, int NF>
cudaError_t launch_rows_t(const void* img, int dtype, long long ld, int H, int W, int R,
                          int boundary, int q, T* S, long long pitch, int Hp, int Wp,
                          DevStatus* st, cudaStream_t s) {
  constexpr int V = sizeof(T) == 8 ? 4 : 2;
  const float scale = ldexpf(1.f, q);  // q <= 100: a normal float32
  switch (dtype) {
    case BSF_U8:
      k_scan_rows<T, NF, uint8_t, V><<<Hp, kRowThreads, 0, s>>>(
          (const uint8_t*)img, ld, H, W, R, boundary, scale, q, S, pitch, Hp, Wp, st);
      break;
    case BSF_F32:
      k_scan_rows<T, NF, float, V><<<Hp, kRowThreads, 0, s>>>(
          (const float*)img, ld, H, W, R, boundary, scale, q, S, pitch, Hp, Wp, st);
      break;
    case BSF_F64:
      k_scan_rows<T, NF, double, V><<<Hp, kRowThreads, 0, s>>>(
          (const double*)img, ld, H, W, R, boundary, scale, q, S, pitch, Hp, Wp, st);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T, int NF, int SKEW>
cudaError_t launch_v_t(T* S, long long pitch, int Hp, int Wp, T* agg, T* carry, cudaStream_t s) {
  // u = x - SKEW * y ranges over [umin, umin + Nu)
  const int umin = SKEW == 1 ? -(Hp - 1) : 0;
  const int Nu = SKEW == 0 ? Wp : Wp + Hp - 1;
  const int nchunks = (Hp + kScanChunk - 1) / kScanChunk;
  const int threads = 128;
  dim3 grid((Nu + threads - 1) / threads, nchunks);
  k_vscan_agg<T, NF, SKEW><<<grid, threads, 0, s>>>(S, pitch, Hp, Wp, umin, Nu, agg);
  k_vscan_carry<T, NF><<<(Nu + threads - 1) / threads, threads, 0, s>>>(agg, carry, nchunks, Hp, Nu);
  k_vscan_apply<T, NF, SKEW><<<grid, threads, 0, s>>>(S, pitch, Hp, Wp, umin, Nu, carry);
  return cudaGetLastError();
}

template <typename T, int NF>
cudaError_t launch_v_skew(int skew, T* S, long long pitch, int Hp, int Wp, T* agg, T* carry,
                          cudaStream_t s) {
  switch (skew) {
    case 0: return launch_v_t<T, NF, 0>(S, pitch, Hp, Wp, agg, carry, s);
    case 1: return launch_v_t<T, NF, 1>(S, pitch, Hp, Wp, agg, carry, s);
    case -1: return launch_v_t<T, NF, -1>(S, pitch, Hp, Wp, agg, carry, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t bsf_launch_scan_rows(int elem_bytes, int n, const void* img, int dtype, long long ld,
                                 int H, int W, int R, int boundary, int q, void* S,
                                 long long pitch, int Hp, int Wp, DevStatus* st, cudaStream_t s) {
#define BSF_ROWS(T, NF) \
  return launch_rows_t<T, NF>(img, dtype, ld, H, W, R, boundary, q, (T*)S, pitch, Hp, Wp, st, s)
  if (elem_bytes == 8) {
    if (n == 1) BSF_ROWS(uint64_t, 1);
    if (n == 2) BSF_ROWS(uint64_t, 2);
    if (n == 3) BSF_ROWS(uint64_t, 3);
  } else if (elem_bytes == 16) {
    if (n == 1) BSF_ROWS(u128, 1);
    if (n == 2) BSF_ROWS(u128, 2);
    if (n == 3) BSF_ROWS(u128, 3);
  }
#undef BSF_ROWS
  return cudaErrorInvalidValue;
}

cudaError_t bsf_launch_vscan(int elem_bytes, int n, int skew, void* S, long long pitch,
                             int Hp, int Wp, void* agg, void* carry, cudaStream_t s) {
#define BSF_V(T, NF) return launch_v_skew<T, NF>(skew, (T*)S, pitch, Hp, Wp, (T*)agg, (T*)carry, s)
  if (elem_bytes == 8) {
    if (n == 1) BSF_V(uint64_t, 1);
    if (n == 2) BSF_V(uint64_t, 2);
    if (n == 3) BSF_V(uint64_t, 3);
  } else if (elem_bytes == 16) {
    if (n == 1) BSF_V(u128, 1);
    if (n == 2) BSF_V(u128, 2);
    if (n == 3) BSF_V(u128, 3);
  }
#undef BSF_V
  return cudaErrorInvalidValue;
}
