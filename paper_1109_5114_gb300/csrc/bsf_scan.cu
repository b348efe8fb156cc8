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
//       into chunks of kScanChunk rows, scanned in phases:
//         agg   -- per (line, chunk): the n-fold state at the chunk's end
//                  with zero carry-in;
//         carry -- combine the earlier chunks' states in order; the state
//                  after a chunk of m rows is
//                  s'_f = sum_{j<=f} C(m-1+j, j) s_{f-j} + agg_f
//                  (folded at the start of the apply kernel);
//         apply -- per (line, chunk): rescan with the carried-in state and
//                  write the result in place.
//       No block waits on another block.  (The single-pass look-back variant
//       below is the default; this one needs no inter-block waits.)
//
// Arithmetic wraps modulo 2^64 or 2^128 (the element type), which the final
// finite differences cancel exactly.
#include <type_traits>

#include "bsf_scan_bodies.cuh"

namespace {

// A block takes rows yp = blockIdx.x, + gridDim.x, ... and updates the status
// word once for all of them.
template <typename T, int NF, typename In, int V>
__global__ void __launch_bounds__(kRowThreads)
k_scan_rows(const In* __restrict__ img, long long ld, int H, int W, int R, int row0, int boundary,
            float scale_f, int q, T* __restrict__ S, long long pitch, int Hp, int Wp,
            DevStatus* st) {
  bsf_grid_dep_launch();  // the first vertical reduction may be scheduled (it waits for this grid)
  float amax = 0.f;
  bool all_ok = true;
  for (int yp = blockIdx.x; yp < Hp; yp += gridDim.x)
    scan_row<T, NF, In, V>(img, ld, H, W, R, row0, boundary, scale_f, q, S, pitch, Wp, yp, amax, all_ok);
  scan_rows_status(amax, all_ok, st);
}

// blocks of the row pass: this many per SM (each loops over rows)
constexpr int kRowBlocksPerSM = 8;

int rows_grid(int Hp) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  const int g = sms * kRowBlocksPerSM;
  return Hp < g ? Hp : g;
}

// The reduction pass with each chunk's rows split between SPLIT warps of a
// block of 128 threads: 128 / SPLIT lines x SPLIT consecutive parts of the
// chunk (thread t: line t mod (128 / SPLIT), part t div (128 / SPLIT)); the
// parts' zero-carry states combine in order through shared memory.  SPLIT
// times the threads of one line per thread, for SPLIT times the loads in
// flight.
constexpr int kAggSplit = 2;
constexpr bool kScanPdl = true;

template <typename T, int NF, int SKEW, bool REV, int SPLIT>
__global__ void __launch_bounds__(128)
k_vscan_agg(const T* __restrict__ S, long long pitch, int Hp, int Wp, int umin, int Nu, int ch,
            T* __restrict__ agg) {
  // a programmatic dependent of the kernel before it: wait for it to finish
  bsf_grid_dep_launch();
  bsf_grid_dep_wait();
  constexpr int LINES = 128 / SPLIT;
  // raw storage: the element types with constructors are written before read
  __shared__ __align__(16) unsigned char s_raw[SPLIT * NF * LINES * sizeof(T)];
  T(*s_part)[NF][LINES] = reinterpret_cast<T(*)[NF][LINES]>(s_raw);
  const int t = threadIdx.x, line = t % LINES, part = t / LINES;
  const int ui = blockIdx.x * LINES + line;
  const int c = blockIdx.y;
  const int y0 = c * ch, y1 = min(y0 + ch, Hp);
  const int plen = (ch + SPLIT - 1) / SPLIT;
  const int r0 = min(y0 + part * plen, y1), r1 = min(r0 + plen, y1);  // this thread's rows (scan order)
  T s[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) s[f] = 0;
  if (ui < Nu) {
    const int u = umin + ui;
    const int A = REV ? u + SKEW * (Hp - 1) : u;
    constexpr int B = REV ? -SKEW : SKEW;
    int lo = r0, hi = r1;
    line_rows<B>(A, Wp, lo, hi);
    if (lo < hi) {
#pragma unroll 8
      for (int yl = lo; yl < hi; ++yl) {
        const int y = REV ? Hp - 1 - yl : yl;
        const T v = S[(long long)y * pitch + (A + B * yl)];
        s[0] += v;
#pragma unroll
        for (int f = 1; f < NF; ++f) s[f] += s[f - 1];
      }
      zero_rows_transfer<T, NF>(s, r1 - hi);  // leading zero rows leave the state at zero
    }
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) s_part[part][f][line] = s[f];
  __syncthreads();
  if (part == 0 && ui < Nu) {
    for (int p = 1; p < SPLIT; ++p) {
      const int q0 = min(y0 + p * plen, y1), q1 = min(q0 + plen, y1);
      T a[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) a[f] = s_part[p][f][line];
      tp_combine<T, NF>(s, a, q1 - q0);  // the parts before, then part p's rows
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) agg[((long long)c * NF + f) * Nu + ui] = s[f];
  }
}

template <typename T, int NF, int SKEW, bool REV>
__global__ void __launch_bounds__(128)
k_vscan_apply(T* __restrict__ S, long long pitch, int Hp, int Wp, int umin, int Nu, int ch,
              const T* __restrict__ agg) {
  // a programmatic dependent of the reduction before it; the next kernel may
  // start its own prologue (it waits for this grid)
  bsf_grid_dep_launch();
  bsf_grid_dep_wait();
  vscan_apply_body<T, NF, SKEW, REV>(S, pitch, Hp, Wp, umin, Nu, ch, agg, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Single-pass variant: chained scan with decoupled look-back.
//
// A tile is kLbLines consecutive lines x LbRows<T> rows.  Tiles take a ticket
// from a global counter in launch order and map it chunk-major, so a tile's
// predecessors (same lines, earlier chunks) always hold smaller tickets and
// are already running or done: every wait ends.  Each tile loads its values
// into registers, publishes its zero-carry state (flag 1), walks back over
// its predecessors -- combining published states until it meets an inclusive
// one (flag 2) -- publishes its own inclusive state and rescans its registers
// with the carried-in state.  S is read and written once.
//
// Every wait is bounded: after spin_limit polls the tile records
// BSF_ETIMEOUT, continues with a zero carry and still publishes, so its
// successors finish too (the result is then wrong and reported, never hung).
// ---------------------------------------------------------------------------
constexpr int kLbLines = 128;
// rows per tile: the default, and a shorter option (more resident tiles)
template <typename T, bool SHORT> struct LbRows {
  static constexpr int value = (sizeof(T) == 8 ? 32 : 16) / (SHORT ? 2 : 1);
};

// state after prefix state P followed by a segment of m rows whose
// zero-carry state is X:  r_f = sum_{i<=f} C(m-1+i, i) P_{f-i} + X_f
template <typename T, int NF>
__device__ __forceinline__ void lb_combine(const T* P, const T* X, long long m, T* r) {
  r[0] = P[0] + X[0];
  if constexpr (NF >= 2) r[1] = P[1] + bsf_mul_int(P[0], m) + X[1];
  if constexpr (NF >= 3) r[2] = P[2] + bsf_mul_int(P[1], m) + bsf_mul_int(P[0], m * (m + 1) / 2) + X[2];
}

__device__ __forceinline__ unsigned lb_load_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename T> __device__ __forceinline__ T lb_load_l2(const T* p);
template <> __device__ __forceinline__ uint64_t lb_load_l2<uint64_t>(const uint64_t* p) {
  return __ldcg(reinterpret_cast<const unsigned long long*>(p));
}
template <> __device__ __forceinline__ u128 lb_load_l2<u128>(const u128* p) {
  const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(p));
  return ((u128)v.y << 64) | (u128)v.x;
}

template <typename T, int NF, int SKEW, bool REV, bool SHORT>
__global__ void __launch_bounds__(kLbLines)
k_vscan_lb(T* __restrict__ S, long long pitch, int Hp, int Wp, int umin, int Nu, int NS,
           T* __restrict__ aggs, T* __restrict__ incls, unsigned* __restrict__ flags,
           unsigned* __restrict__ ticket, int spin_limit, int test_unpublished, DevStatus* st) {
  constexpr int CH = LbRows<T, SHORT>::value;
  __shared__ int s_tile;
  __shared__ unsigned s_flag;
  const int t = threadIdx.x;
  if (t == 0) s_tile = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int tile = s_tile;
  const int c = tile / NS, sidx = tile - c * NS;
  const int ui = sidx * kLbLines + t;
  const bool line_ok = ui < Nu;
  const int u = umin + ui;
  const int y0 = c * CH;
  const int rows = min(CH, Hp - y0);

  // REV: the running sum goes up the line (suffix sum, the transpose); the
  // logical row y0 + r is then the physical row Hp - 1 - (y0 + r)
  T v[CH];
#pragma unroll
  for (int r = 0; r < CH; ++r) {
    const int y = REV ? Hp - 1 - (y0 + r) : y0 + r;
    const int x = u + SKEW * y;
    v[r] = 0;
    if (line_ok && r < rows && x >= 0 && x < Wp) v[r] = S[y * (int)pitch + x];
  }
  T a[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) a[f] = 0;
#pragma unroll
  for (int r = 0; r < CH; ++r) {
    a[0] += v[r];
#pragma unroll
    for (int f = 1; f < NF; ++f) a[f] += a[f - 1];
  }
  // the last chunk may be short; zero rows past it only add the higher folds
  // of a[] after its end, which no successor reads (it is the last chunk)

  const long long slot = (long long)tile * NF * kLbLines + t;
  T E[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) E[f] = 0;
  if (c == 0) {
#pragma unroll
    for (int f = 0; f < NF; ++f) incls[slot + f * kLbLines] = a[f];
    __threadfence();  // every writer makes its own state visible before the flag
    __syncthreads();
    // failure injection for tests: leave the first chunk's flags unset so its
    // successors' bounded waits run out
    if (t == 0 && !test_unpublished) atomicExch(&flags[tile], 2u);
  } else {
#pragma unroll
    for (int f = 0; f < NF; ++f) aggs[slot + f * kLbLines] = a[f];
    __threadfence();
    __syncthreads();
    if (t == 0) atomicExch(&flags[tile], 1u);
    T X[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) X[f] = 0;
    long long mx = 0;
    for (int j = c - 1; j >= 0; --j) {
      const int pj = j * NS + sidx;
      if (t == 0) {
        unsigned fl = 0;
        for (int spins = 0; spins <= spin_limit; ++spins) {
          fl = lb_load_acquire(&flags[pj]);
          if (fl) break;
          __nanosleep(64);
        }
        s_flag = fl;
      }
      __syncthreads();
      const unsigned fl = s_flag;
      __syncthreads();
      if (fl == 0) {  // the bounded wait ran out
        if (t == 0) bsf_set_error(st, BSF_ETIMEOUT);
        break;
      }
      const T* src = (fl == 2 ? incls : aggs) + (long long)pj * NF * kLbLines + t;
      T P[NF], R2[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) P[f] = lb_load_l2(src + f * kLbLines);
      lb_combine<T, NF>(P, X, mx, R2);
      if (fl == 2) {
#pragma unroll
        for (int f = 0; f < NF; ++f) E[f] = R2[f];
        break;
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) X[f] = R2[f];
      mx += CH;
    }
    T I[NF];
    lb_combine<T, NF>(E, a, rows, I);
#pragma unroll
    for (int f = 0; f < NF; ++f) incls[slot + f * kLbLines] = I[f];
    __threadfence();
    __syncthreads();
    if (t == 0) atomicExch(&flags[tile], 2u);
  }
  // rescan with the carried-in state
#pragma unroll
  for (int r = 0; r < CH; ++r) {
    E[0] += v[r];
#pragma unroll
    for (int f = 1; f < NF; ++f) E[f] += E[f - 1];
    const int y = REV ? Hp - 1 - (y0 + r) : y0 + r;
    const int x = u + SKEW * y;
    if (line_ok && r < rows && x >= 0 && x < Wp) S[y * (int)pitch + x] = E[NF - 1];
  }
}

template <typename T, int NF, int SKEW, bool REV, bool SHORT>
cudaError_t launch_lb_t(T* S, long long pitch, int Hp, int Wp, T* aggs, T* incls,
                        unsigned* sync_words, int spin_limit, int test_unpublished, DevStatus* st,
                        cudaStream_t s) {
  constexpr int CH = LbRows<T, SHORT>::value;
  const int umin = SKEW == 1 ? -(Hp - 1) : 0;
  const int Nu = SKEW == 0 ? Wp : Wp + Hp - 1;
  const int NS = (Nu + kLbLines - 1) / kLbLines;
  const int NC = (Hp + CH - 1) / CH;
  cudaError_t e = cudaMemsetAsync(sync_words, 0, sizeof(unsigned) * (1 + (size_t)NS * NC), s);
  if (e != cudaSuccess) return e;
  k_vscan_lb<T, NF, SKEW, REV, SHORT><<<NS * NC, kLbLines, 0, s>>>(S, pitch, Hp, Wp, umin, Nu, NS, aggs, incls,
                                                      sync_words + 1, sync_words, spin_limit,
                                                      test_unpublished, st);
  return cudaGetLastError();
}

template <typename T, int NF, bool REV, bool SHORT>
cudaError_t launch_lb_skew(int skew, T* S, long long pitch, int Hp, int Wp, T* aggs, T* incls,
                           unsigned* sync_words, int spin_limit, int tu, DevStatus* st,
                           cudaStream_t s) {
  switch (skew) {
    case 0: return launch_lb_t<T, NF, 0, REV, SHORT>(S, pitch, Hp, Wp, aggs, incls, sync_words, spin_limit, tu, st, s);
    case 1: return launch_lb_t<T, NF, 1, REV, SHORT>(S, pitch, Hp, Wp, aggs, incls, sync_words, spin_limit, tu, st, s);
    case -1: return launch_lb_t<T, NF, -1, REV, SHORT>(S, pitch, Hp, Wp, aggs, incls, sync_words, spin_limit, tu, st, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// In-place n-fold suffix sums along rows (the transpose of the d1 running
// sum): one block per row, chunks from the right end; the logical index x'
// maps to the physical column Wp - 1 - x'.
// ---------------------------------------------------------------------------
template <typename T, int NF, int V>
__global__ void __launch_bounds__(kRowThreads)
k_suffix_rows(T* __restrict__ S, long long pitch, int Wp) {
  // a programmatic dependent of the kernel before it (waits for it here); the
  // extension fold after it may be scheduled meanwhile
  bsf_grid_dep_launch();
  bsf_grid_dep_wait();
  // suffix sums: scan order runs from the row's end to its start
  T* row = S + (long long)blockIdx.x * pitch;
  row_scan_segments<T, NF, V>(Wp, [&](int xl) -> T { return row[Wp - 1 - xl]; },
                              [&](int xl, T val) { row[Wp - 1 - xl] = val; });
}
template <typename T, int NF, int V>
cudaError_t launch_rows_v(const void* img, int dtype, long long ld, int H, int W, int R, int row0,
                          int boundary, int q, T* S, long long pitch, int Hp, int Wp,
                          DevStatus* st, cudaStream_t s) {
  const float scale = ldexpf(1.f, q);  // q <= 100: a normal float32
  switch (dtype) {
    case BSF_U8:
      k_scan_rows<T, NF, uint8_t, V><<<rows_grid(Hp), kRowThreads, 0, s>>>(
          (const uint8_t*)img, ld, H, W, R, row0, boundary, scale, q, S, pitch, Hp, Wp, st);
      break;
    case BSF_F32:
      k_scan_rows<T, NF, float, V><<<rows_grid(Hp), kRowThreads, 0, s>>>(
          (const float*)img, ld, H, W, R, row0, boundary, scale, q, S, pitch, Hp, Wp, st);
      break;
    case BSF_F64:
      k_scan_rows<T, NF, double, V><<<rows_grid(Hp), kRowThreads, 0, s>>>(
          (const double*)img, ld, H, W, R, row0, boundary, scale, q, S, pitch, Hp, Wp, st);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// V consecutive elements per thread, chosen so that one pass of 256 V
// elements covers most of a padded row without leaving warps idle
template <typename T, int NF>
cudaError_t launch_rows_t(const void* img, int dtype, long long ld, int H, int W, int R, int row0,
                          int boundary, int q, T* S, long long pitch, int Hp, int Wp,
                          DevStatus* st, cudaStream_t s) {
  if (Wp <= kRowThreads * 4)
    return launch_rows_v<T, NF, 4>(img, dtype, ld, H, W, R, row0, boundary, q, S, pitch, Hp, Wp, st, s);
  if constexpr (sizeof(T) > 8) {  // 16-byte elements: V = 9 keeps the transpose under 48 KB
    return launch_rows_v<T, NF, 9>(img, dtype, ld, H, W, R, row0, boundary, q, S, pitch, Hp, Wp, st, s);
  } else {
    if (Wp <= kRowThreads * 9)
      return launch_rows_v<T, NF, 9>(img, dtype, ld, H, W, R, row0, boundary, q, S, pitch, Hp, Wp, st, s);
    return launch_rows_v<T, NF, 12>(img, dtype, ld, H, W, R, row0, boundary, q, S, pitch, Hp, Wp, st, s);
  }
}

template <typename T, int NF, int SKEW, bool REV>
cudaError_t launch_v_t(T* S, long long pitch, int Hp, int Wp, int ch, T* agg, T* carry,
                       cudaStream_t s) {
  // u = x - SKEW * y ranges over [umin, umin + Nu)
  const int umin = SKEW > 0 ? -SKEW * (Hp - 1) : 0;
  const int Nu = Wp + (SKEW < 0 ? -SKEW : SKEW) * (Hp - 1);
  const int nchunks = (Hp + ch - 1) / ch;
  const int threads = 128;
  dim3 grid((Nu + threads - 1) / threads, nchunks);
  (void)carry;
  // both launched as programmatic dependents of the kernel before them (each
  // waits for it at its start, so only the launch and the ramp-up overlap)
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = kScanPdl ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(threads);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((Nu + 128 / kAggSplit - 1) / (128 / kAggSplit), nchunks);
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_vscan_agg<T, NF, SKEW, REV, kAggSplit>, (const T*)S, pitch, Hp, Wp,
                                     umin, Nu, ch, agg);
  if (e != cudaSuccess) return e;
  cfg.gridDim = grid;
  return cudaLaunchKernelEx(&cfg, k_vscan_apply<T, NF, SKEW, REV>, S, pitch, Hp, Wp, umin, Nu, ch, (const T*)agg);
}

template <typename T, int NF, bool REV>
cudaError_t launch_v_skew(int skew, T* S, long long pitch, int Hp, int Wp, int ch, T* agg, T* carry,
                          cudaStream_t s) {
  switch (skew) {
    case 0: return launch_v_t<T, NF, 0, REV>(S, pitch, Hp, Wp, ch, agg, carry, s);
    case 1: return launch_v_t<T, NF, 1, REV>(S, pitch, Hp, Wp, ch, agg, carry, s);
    case -1: return launch_v_t<T, NF, -1, REV>(S, pitch, Hp, Wp, ch, agg, carry, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t bsf_launch_scan_rows(int prec, int n, const void* img, int dtype, long long ld,
                                 int H, int W, int R, int row0, int boundary, int q, void* S,
                                 long long pitch, int Hp, int Wp, DevStatus* st, cudaStream_t s) {
#define BSF_ROWS(T, NF) \
  return launch_rows_t<T, NF>(img, dtype, ld, H, W, R, row0, boundary, q, (T*)S, pitch, Hp, Wp, st, s)
  switch (prec * 10 + n) {
    case 51: BSF_ROWS(uint32_t, 1);
    case 52: BSF_ROWS(uint32_t, 2);
    case 53: BSF_ROWS(uint32_t, 3);
    case 11: BSF_ROWS(uint64_t, 1);
    case 12: BSF_ROWS(uint64_t, 2);
    case 13: BSF_ROWS(uint64_t, 3);
    case 21: BSF_ROWS(u128, 1);
    case 22: BSF_ROWS(u128, 2);
    case 23: BSF_ROWS(u128, 3);
    case 31: BSF_ROWS(double, 1);
    case 32: BSF_ROWS(double, 2);
    case 33: BSF_ROWS(double, 3);
    case 41: BSF_ROWS(f32x2, 1);
    case 42: BSF_ROWS(f32x2, 2);
    case 43: BSF_ROWS(f32x2, 3);
    default: return cudaErrorInvalidValue;
  }
#undef BSF_ROWS
}

namespace {
template <typename T, int NF>
cudaError_t launch_suffix_t(void* S, long long pitch, int Hp, int Wp, cudaStream_t s) {
  // elements per thread chosen like the forward row pass
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(Hp);
  cfg.blockDim = dim3(kRowThreads);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  T* St = (T*)S;
  if (Wp <= kRowThreads * 4) return cudaLaunchKernelEx(&cfg, k_suffix_rows<T, NF, 4>, St, pitch, Wp);
  if constexpr (sizeof(T) > 8) {
    return cudaLaunchKernelEx(&cfg, k_suffix_rows<T, NF, 9>, St, pitch, Wp);
  } else {
    if (Wp <= kRowThreads * 9) return cudaLaunchKernelEx(&cfg, k_suffix_rows<T, NF, 9>, St, pitch, Wp);
    return cudaLaunchKernelEx(&cfg, k_suffix_rows<T, NF, 12>, St, pitch, Wp);
  }
}
}  // namespace

cudaError_t bsf_launch_suffix_rows(int elem_bytes, int n, void* S, long long pitch, int Hp, int Wp,
                                   cudaStream_t s) {
  switch (elem_bytes * 10 + n) {
    case 81: return launch_suffix_t<uint64_t, 1>(S, pitch, Hp, Wp, s);
    case 82: return launch_suffix_t<uint64_t, 2>(S, pitch, Hp, Wp, s);
    case 83: return launch_suffix_t<uint64_t, 3>(S, pitch, Hp, Wp, s);
    case 161: return launch_suffix_t<u128, 1>(S, pitch, Hp, Wp, s);
    case 162: return launch_suffix_t<u128, 2>(S, pitch, Hp, Wp, s);
    case 163: return launch_suffix_t<u128, 3>(S, pitch, Hp, Wp, s);
    default: return cudaErrorInvalidValue;
  }
}

size_t bsf_vscan_lb_bytes(int elem_bytes, int n, int Hp, int Wp, size_t* sync_bytes) {
  // sized for the short tiles (the larger number of tiles)
  const int CH = elem_bytes == 8 ? LbRows<uint64_t, true>::value : LbRows<u128, true>::value;
  const size_t Nu = (size_t)Wp + Hp - 1;
  const size_t NS = (Nu + kLbLines - 1) / kLbLines;
  const size_t NC = (size_t)(Hp + CH - 1) / CH;
  if (sync_bytes) *sync_bytes = sizeof(unsigned) * (1 + NS * NC);
  return NS * NC * (size_t)n * kLbLines * elem_bytes;  // one of the two state arrays
}

namespace {

template <typename T, int NF>
cudaError_t launch_lb_any(int skew, bool reverse, bool short_tiles, void* S, long long pitch,
                          int Hp, int Wp, void* aggs, void* incls, unsigned* sync_words,
                          int spin_limit, int test_unpublished, DevStatus* st, cudaStream_t s) {
  T* S_ = (T*)S;
  T* a_ = (T*)aggs;
  T* i_ = (T*)incls;
  if (reverse) {
    if (short_tiles)
      return launch_lb_skew<T, NF, true, true>(skew, S_, pitch, Hp, Wp, a_, i_, sync_words,
                                               spin_limit, test_unpublished, st, s);
    return launch_lb_skew<T, NF, true, false>(skew, S_, pitch, Hp, Wp, a_, i_, sync_words,
                                              spin_limit, test_unpublished, st, s);
  }
  if (short_tiles)
    return launch_lb_skew<T, NF, false, true>(skew, S_, pitch, Hp, Wp, a_, i_, sync_words,
                                              spin_limit, test_unpublished, st, s);
  return launch_lb_skew<T, NF, false, false>(skew, S_, pitch, Hp, Wp, a_, i_, sync_words,
                                             spin_limit, test_unpublished, st, s);
}

}  // namespace

cudaError_t bsf_launch_vscan_lb(int prec, int n, int skew, bool reverse, bool short_tiles,
                                void* S, long long pitch, int Hp, int Wp, void* aggs, void* incls,
                                unsigned* sync_words, int spin_limit, int test_unpublished,
                                DevStatus* st, cudaStream_t s) {
  const int elem_bytes = prec == 2 ? 16 : 8;
  if (prec != 1 && prec != 2) return cudaErrorInvalidValue;  // fixed point only
  switch (elem_bytes * 10 + n) {
    case 81: return launch_lb_any<uint64_t, 1>(skew, reverse, short_tiles, S, pitch, Hp, Wp, aggs, incls, sync_words, spin_limit, test_unpublished, st, s);
    case 82: return launch_lb_any<uint64_t, 2>(skew, reverse, short_tiles, S, pitch, Hp, Wp, aggs, incls, sync_words, spin_limit, test_unpublished, st, s);
    case 83: return launch_lb_any<uint64_t, 3>(skew, reverse, short_tiles, S, pitch, Hp, Wp, aggs, incls, sync_words, spin_limit, test_unpublished, st, s);
    case 161: return launch_lb_any<u128, 1>(skew, reverse, short_tiles, S, pitch, Hp, Wp, aggs, incls, sync_words, spin_limit, test_unpublished, st, s);
    case 162: return launch_lb_any<u128, 2>(skew, reverse, short_tiles, S, pitch, Hp, Wp, aggs, incls, sync_words, spin_limit, test_unpublished, st, s);
    case 163: return launch_lb_any<u128, 3>(skew, reverse, short_tiles, S, pitch, Hp, Wp, aggs, incls, sync_words, spin_limit, test_unpublished, st, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t bsf_launch_vscan(int prec, int n, int skew, bool reverse, void* S, long long pitch,
                             int Hp, int Wp, int chunk, void* agg, void* carry, cudaStream_t s) {
#define BSF_V(T, NF)                                                                              \
  return reverse ? launch_v_skew<T, NF, true>(skew, (T*)S, pitch, Hp, Wp, chunk, (T*)agg,        \
                                              (T*)carry, s)                                      \
                 : launch_v_skew<T, NF, false>(skew, (T*)S, pitch, Hp, Wp, chunk, (T*)agg,       \
                                               (T*)carry, s)
  switch (prec * 10 + n) {
    case 51: BSF_V(uint32_t, 1);
    case 52: BSF_V(uint32_t, 2);
    case 53: BSF_V(uint32_t, 3);
    case 11: BSF_V(uint64_t, 1);
    case 12: BSF_V(uint64_t, 2);
    case 13: BSF_V(uint64_t, 3);
    case 21: BSF_V(u128, 1);
    case 22: BSF_V(u128, 2);
    case 23: BSF_V(u128, 3);
    case 31: BSF_V(double, 1);
    case 32: BSF_V(double, 2);
    case 33: BSF_V(double, 3);
    case 41: BSF_V(f32x2, 1);
    case 42: BSF_V(f32x2, 2);
    case 43: BSF_V(f32x2, 3);
    default: return cudaErrorInvalidValue;
  }
#undef BSF_V
}

// ---------------------------------------------------------------------------
// Batched kernels: a block finds its image by binary search over the block
// offsets of the phase, then runs the single-image body on it.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ int batch_find(const int* __restrict__ starts, int B, int blk) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T, int NF, typename In>
__global__ void __launch_bounds__(kRowThreads)
k_batch_rows(const BatchImage* __restrict__ imgs, const int* __restrict__ starts, int B,
             int boundary, int q, DevStatus* st) {
  const int i = batch_find(starts, B, blockIdx.x);
  const BatchImage& im = imgs[i];
  scan_rows_body<T, NF, In, 4>((const In*)im.img, im.ld, im.H, im.W, im.R, 0, boundary,
                               bsf_pow2_f32(q), q, (T*)im.S, im.pitch, im.Hp, im.Wp, st,
                               blockIdx.x - starts[i]);
}

template <typename T, int NF, int SKEW, bool APPLY>
__global__ void __launch_bounds__(128)
k_batch_vscan(const BatchImage* __restrict__ imgs, const int* __restrict__ starts, int B) {
  const int i = batch_find(starts, B, blockIdx.x);
  const BatchImage& im = imgs[i];
  const int local = blockIdx.x - starts[i];
  const int Nu = SKEW == 0 ? im.Wp : im.Wp + im.Hp - 1;
  const int umin = SKEW == 1 ? -(im.Hp - 1) : 0;
  const int gx = (Nu + 127) / 128;
  const int bx = local % gx, c = local / gx;
  if (APPLY)
    vscan_apply_body<T, NF, SKEW, false>((T*)im.S, im.pitch, im.Hp, im.Wp, umin, Nu, im.ch,
                                         (const T*)im.agg, bx, c);
  else
    vscan_agg_body<T, NF, SKEW, false>((const T*)im.S, im.pitch, im.Hp, im.Wp, umin, Nu, im.ch,
                                       (T*)im.agg, bx, c);
}

}  // namespace

cudaError_t bsf_launch_batch_rows(int n, int dtype, const BatchImage* imgs, const int* starts, int B,
                                  int total, int boundary, int q, DevStatus* st, cudaStream_t s) {
#define BSF_BR(NF, In) k_batch_rows<uint64_t, NF, In><<<total, kRowThreads, 0, s>>>(imgs, starts, B, boundary, q, st)
  if (dtype == BSF_F32) {
    if (n == 1) BSF_BR(1, float); else if (n == 2) BSF_BR(2, float); else BSF_BR(3, float);
  } else if (dtype == BSF_U8) {
    if (n == 1) BSF_BR(1, uint8_t); else if (n == 2) BSF_BR(2, uint8_t); else BSF_BR(3, uint8_t);
  } else if (dtype == BSF_F64) {
    if (n == 1) BSF_BR(1, double); else if (n == 2) BSF_BR(2, double); else BSF_BR(3, double);
  } else {
    return cudaErrorInvalidValue;
  }
#undef BSF_BR
  return cudaGetLastError();
}

namespace {
template <int NF, int SKEW>
void batch_vscan_t(const BatchImage* imgs, const int* starts, int B, int total, cudaStream_t s) {
  k_batch_vscan<uint64_t, NF, SKEW, false><<<total, 128, 0, s>>>(imgs, starts, B);
  k_batch_vscan<uint64_t, NF, SKEW, true><<<total, 128, 0, s>>>(imgs, starts, B);
}
template <int NF>
void batch_vscan_n(int skew, const BatchImage* imgs, const int* starts, int B, int total,
                   cudaStream_t s) {
  if (skew == 0) batch_vscan_t<NF, 0>(imgs, starts, B, total, s);
  else if (skew == 1) batch_vscan_t<NF, 1>(imgs, starts, B, total, s);
  else batch_vscan_t<NF, -1>(imgs, starts, B, total, s);
}
}  // namespace

cudaError_t bsf_launch_batch_vscan(int n, int skew, const BatchImage* imgs, const int* starts, int B,
                                   int total, cudaStream_t s) {
  if (n == 1) batch_vscan_n<1>(skew, imgs, starts, B, total, s);
  else if (n == 2) batch_vscan_n<2>(skew, imgs, starts, B, total, s);
  else if (n == 3) batch_vscan_n<3>(skew, imgs, starts, B, total, s);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Second direction set (Section 2.3, Algorithm 3, step 2): running sums along
// e1 = (2,1), e2 = (1,2), e3 = (-1,2), e4 = (-2,1).  No direction runs along
// a row, so the extension and quantisation get a pass of their own
// (k_extend); e1 and e4 step one row down and 2 columns across (skew +2 and
// -2 of the three-phase scan); e2 and e3 step two rows down and one column
// across, so each row parity is a grid of its own (pitch 2p) on which they
// are skew +1 and -1 scans; both parities run in one launch (blockIdx.z).
// ---------------------------------------------------------------------------
namespace {

// One block per padded row; the block's maximum |Q| goes to the status word
// with one atomic (a per-warp atomic on that one word serialises).
template <typename T, typename In>
__global__ void __launch_bounds__(256)
k_extend(const In* __restrict__ img, long long ld, int H, int W, int R, int row0, int boundary,
         float scale_f, int q, T* __restrict__ S, long long pitch, int Wp, DevStatus* st) {
  const int yp = blockIdx.x;
  bool yvalid;
  const int ys = bsf_map_index(row0 + yp - R, H, boundary, yvalid);
  const In* src = img + (long long)ys * ld;
  T* row = S + (long long)yp * pitch;
  float amax = 0.f;
  bool ok = true;
  for (int xp = threadIdx.x; xp < Wp; xp += 256) {
    T v = (T)0;
    bool xvalid;
    const int xs = bsf_map_index(xp - R, W, boundary, xvalid);
    if (yvalid && xvalid) {
      bool ok1;
      float ax;
      v = quantize_one<T, In>(src[xs], q, scale_f, ok1, ax);
      ok &= ok1;
      amax = fmaxf(amax, ax);
    }
    row[xp] = v;
  }
  __shared__ float s_max[8];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  __syncthreads();
  if (!ok) s_bad = 1;
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = amax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = s_max[0];
    for (int w = 1; w < 8; ++w) m = fmaxf(m, s_max[w]);
    if (m > 0.f) bsf_atomic_max_pos_float(&st->max_absq_bits, m);
    if (s_bad) bsf_set_error(st, BSF_EOVERFLOW);
  }
}

template <typename T>
cudaError_t launch_extend_t(const void* img, int dtype, long long ld, int H, int W, int R, int row0,
                            int boundary, int q, T* S, long long pitch, int Hp, int Wp, DevStatus* st,
                            cudaStream_t s) {
  const float scale = ldexpf(1.f, q);
  const int grid = Hp;
  switch (dtype) {
    case BSF_U8:
      k_extend<T, uint8_t><<<grid, 256, 0, s>>>((const uint8_t*)img, ld, H, W, R, row0, boundary, scale, q,
                                                S, pitch, Wp, st);
      break;
    case BSF_F32:
      k_extend<T, float><<<grid, 256, 0, s>>>((const float*)img, ld, H, W, R, row0, boundary, scale, q, S,
                                              pitch, Wp, st);
      break;
    case BSF_F64:
      k_extend<T, double><<<grid, 256, 0, s>>>((const double*)img, ld, H, W, R, row0, boundary, scale, q,
                                               S, pitch, Wp, st);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// One row parity of a grid scanned two rows per step: rows par, par + 2, ...
struct ParityGrid {
  int Hs, umin, Nu;
};
template <int SKEW>
__device__ __forceinline__ ParityGrid parity_grid(int Hp, int Wp, int par) {
  ParityGrid g;
  g.Hs = (Hp - par + 1) / 2;
  g.umin = SKEW > 0 ? -(g.Hs - 1) : 0;
  g.Nu = Wp + g.Hs - 1;
  return g;
}

template <typename T, int NF, int SKEW>
__global__ void __launch_bounds__(128)
k_vscan_agg_par(const T* __restrict__ S, long long pitch, int Hp, int Wp, int ch, T* __restrict__ agg,
                long long agg_stride) {
  const int par = blockIdx.z;
  const ParityGrid g = parity_grid<SKEW>(Hp, Wp, par);
  if (g.Hs <= 0) return;
  vscan_agg_body<T, NF, SKEW, false>(S + par * pitch, 2 * pitch, g.Hs, Wp, g.umin, g.Nu, ch,
                                     agg + par * agg_stride, blockIdx.x, blockIdx.y);
}

template <typename T, int NF, int SKEW>
__global__ void __launch_bounds__(128)
k_vscan_apply_par(T* __restrict__ S, long long pitch, int Hp, int Wp, int ch, const T* __restrict__ agg,
                  long long agg_stride) {
  const int par = blockIdx.z;
  const ParityGrid g = parity_grid<SKEW>(Hp, Wp, par);
  if (g.Hs <= 0) return;
  vscan_apply_body<T, NF, SKEW, false>(S + par * pitch, 2 * pitch, g.Hs, Wp, g.umin, g.Nu, ch,
                                       agg + par * agg_stride, blockIdx.x, blockIdx.y);
}

template <typename T, int NF, int SKEW>
cudaError_t launch_par_t(T* S, long long pitch, int Hp, int Wp, int ch, T* agg, cudaStream_t s) {
  const int Hs0 = (Hp + 1) / 2;  // rows of parity 0 (the larger)
  const int Nu0 = Wp + Hs0 - 1;
  const int nch = (Hs0 + ch - 1) / ch;
  const long long stride = (long long)nch * NF * Nu0;
  dim3 grid((Nu0 + 127) / 128, nch, Hp > 1 ? 2 : 1);
  k_vscan_agg_par<T, NF, SKEW><<<grid, 128, 0, s>>>(S, pitch, Hp, Wp, ch, agg, stride);
  k_vscan_apply_par<T, NF, SKEW><<<grid, 128, 0, s>>>(S, pitch, Hp, Wp, ch, agg, stride);
  return cudaGetLastError();
}

template <typename T, int NF>
cudaError_t launch_second_t(T* S, long long pitch, int Hp, int Wp, int ch, T* agg, cudaStream_t s) {
  cudaError_t e;
  // the n folds of each direction are inside each scan; order: e1, e2, e3, e4
  if ((e = launch_v_t<T, NF, 2, false>(S, pitch, Hp, Wp, ch, agg, nullptr, s)) != cudaSuccess) return e;
  if ((e = launch_par_t<T, NF, 1>(S, pitch, Hp, Wp, ch, agg, s)) != cudaSuccess) return e;
  if ((e = launch_par_t<T, NF, -1>(S, pitch, Hp, Wp, ch, agg, s)) != cudaSuccess) return e;
  return launch_v_t<T, NF, -2, false>(S, pitch, Hp, Wp, ch, agg, nullptr, s);
}

}  // namespace

cudaError_t bsf_launch_extend(int prec, const void* img, int dtype, long long ld, int H, int W, int R,
                              int row0, int boundary, int q, void* S, long long pitch, int Hp, int Wp,
                              DevStatus* st, cudaStream_t s) {
  if (prec == BSF_FIX32)
    return launch_extend_t<uint32_t>(img, dtype, ld, H, W, R, row0, boundary, q, (uint32_t*)S, pitch, Hp,
                                     Wp, st, s);
  if (prec == BSF_FIX64)
    return launch_extend_t<uint64_t>(img, dtype, ld, H, W, R, row0, boundary, q, (uint64_t*)S, pitch, Hp,
                                     Wp, st, s);
  if (prec == BSF_FIX128)
    return launch_extend_t<u128>(img, dtype, ld, H, W, R, row0, boundary, q, (u128*)S, pitch, Hp, Wp, st,
                                 s);
  return cudaErrorInvalidValue;
}

size_t bsf_second_scan_elems(int n, int Hp, int Wp, int chunk) {
  // skew +-2 on the whole grid: nchunks x n x (Wp + 2 (Hp - 1)); the parity
  // grids need 2 x ceil(Hs0 / chunk) x n x (Wp + Hs0 - 1), Hs0 = ceil(Hp / 2)
  const size_t full = (size_t)((Hp + chunk - 1) / chunk) * n * ((size_t)Wp + 2 * (size_t)(Hp - 1));
  const int Hs0 = (Hp + 1) / 2;
  const size_t par = 2 * (size_t)((Hs0 + chunk - 1) / chunk) * n * ((size_t)Wp + Hs0 - 1);
  return full > par ? full : par;
}

cudaError_t bsf_launch_scans_second(int prec, int n, void* S, long long pitch, int Hp, int Wp, int chunk,
                                    void* agg, cudaStream_t s) {
  switch (prec * 10 + n) {
    case 51: return launch_second_t<uint32_t, 1>((uint32_t*)S, pitch, Hp, Wp, chunk, (uint32_t*)agg, s);
    case 52: return launch_second_t<uint32_t, 2>((uint32_t*)S, pitch, Hp, Wp, chunk, (uint32_t*)agg, s);
    case 53: return launch_second_t<uint32_t, 3>((uint32_t*)S, pitch, Hp, Wp, chunk, (uint32_t*)agg, s);
    case 11: return launch_second_t<uint64_t, 1>((uint64_t*)S, pitch, Hp, Wp, chunk, (uint64_t*)agg, s);
    case 12: return launch_second_t<uint64_t, 2>((uint64_t*)S, pitch, Hp, Wp, chunk, (uint64_t*)agg, s);
    case 13: return launch_second_t<uint64_t, 3>((uint64_t*)S, pitch, Hp, Wp, chunk, (uint64_t*)agg, s);
    case 21: return launch_second_t<u128, 1>((u128*)S, pitch, Hp, Wp, chunk, (u128*)agg, s);
    case 22: return launch_second_t<u128, 2>((u128*)S, pitch, Hp, Wp, chunk, (u128*)agg, s);
    case 23: return launch_second_t<u128, 3>((u128*)S, pitch, Hp, Wp, chunk, (u128*)agg, s);
    default: return cudaErrorInvalidValue;
  }
}
