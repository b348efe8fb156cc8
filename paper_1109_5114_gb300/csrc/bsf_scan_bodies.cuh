// Device bodies of the running sums (Section 1.1's running sum, Algorithm 3's
// recursion form): the row pass along d1 with the extension and the
// quantisation fused in, and the reduction and rescan bodies of the vertical
// directions d3, d2, d4 in skewed coordinates.  Shared by the kernels of
// bsf_scan.cu (one launch per pass, and the batched launches) and the
// persistent batch kernel of bsf_persistent.cu.
//
// Load: the element loads of the vertical bodies.  BsfLoadCached reads
// through L1 (data written by earlier launches); BsfLoadCoherent reads data
// that other blocks of the same launch wrote before a gpu-scope release
// that this block acquired.
#pragma once

#include <type_traits>

#include "bsf_device.cuh"
#include "bsf_quantize.cuh"

struct BsfLoadCached {
  template <typename T> __device__ __forceinline__ static T load(const T* p) { return *p; }
};
struct BsfLoadCoherent {
  template <typename T> __device__ __forceinline__ static T load(const T* p) { return bsf_load_coherent(p); }
};

namespace {
// ---------------------------------------------------------------------------
// d1 with fused extension + quantisation: one block of kRowThreads per padded
// row.  A pass covers kRowThreads * V elements: warp w owns a segment of
// 32 V, lane l its V consecutive elements.  Each fold is a lane-local scan
// and a warp shuffle scan of the lane totals, so a warp holds the n-fold
// running sums of its segment as if the row started there; the segment's
// carry-in state (the fold values just before it) then enters in closed form:
// with carry-in c_1..c_n, the n-th fold at position i of a segment is the
// local value plus sum_k c_k C(i + n - k, n - k), and the state at its end
// is s_f + sum_{k<=f} c_k C(m - 1 + f - k, f - k) for a segment of m elements
// whose own end state is s.  One barrier per pass exchanges the warps' end
// states.
// ---------------------------------------------------------------------------
constexpr int kRowThreads = 256;

// C(a, j) for j = 0, 1, 2 (the folds n <= 3 need no more)
__device__ __forceinline__ long long binom_small(long long a, int j) {
  return j == 0 ? 1 : (j == 1 ? a : a * (a - 1) / 2);
}

// n-fold running sums of one row of Wp elements by the block, in passes of
// kRowThreads * V elements: element xl (scan order) comes from load(xl) and
// its n-th fold goes to store(xl, value).  The block must call it uniformly.
template <typename T, int NF, int V, typename Load, typename Store>
__device__ __forceinline__ void row_scan_segments(int Wp, Load&& load, Store&& store) {
  constexpr int NW = kRowThreads / 32;
  constexpr int SEG = 32 * V;
  constexpr int VP = V + 1;  // padded stride of the store transpose (fewer bank conflicts)
  // raw storage: the element types with constructors are written before read
  __shared__ __align__(16) unsigned char s_end_raw[NW * NF * sizeof(T)];
  __shared__ __align__(16) unsigned char s_cin_raw[(NW + 1) * NF * sizeof(T)];
  __shared__ __align__(16) unsigned char s_tr_raw[NW * 32 * VP * sizeof(T)];
  T(*s_end)[NF] = reinterpret_cast<T(*)[NF]>(s_end_raw);
  T(*s_cin)[NF] = reinterpret_cast<T(*)[NF]>(s_cin_raw);
  T(*s_tr)[32 * VP] = reinterpret_cast<T(*)[32 * VP]>(s_tr_raw);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  T carry[NF];  // fold values just before the pass (uniform across the block)
#pragma unroll
  for (int f = 0; f < NF; ++f) carry[f] = 0;
  for (int x0 = 0; x0 < Wp; x0 += kRowThreads * V) {
    const int xl0 = x0 + wid * SEG + lane * V;  // this lane's first element
    T v[V];
#pragma unroll
    for (int j = 0; j < V; ++j) v[j] = xl0 + j < Wp ? load(xl0 + j) : (T)0;
    // the folds within the warp's segment (zero carry-in at its start)
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
      const T excl = incl - tot;
#pragma unroll
      for (int j = 0; j < V; ++j) v[j] += excl;
      if (lane == 31) s_end[wid][f] = incl;  // fold f at the segment's last element
    }
    __syncthreads();
    // carry-in state of each warp's segment, and the block's state after the
    // pass: the chain over the warps runs in warp 0 alone (lane w keeps warp
    // w's carry-in) and reaches the others through shared memory
    T cin[NF], cnext[NF];
    if (wid == 0) {
#pragma unroll
      for (int f = 0; f < NF; ++f) cnext[f] = carry[f];
      for (int w = 0; w < NW; ++w) {
        if (w == lane) {
#pragma unroll
          for (int f = 0; f < NF; ++f) s_cin[w][f] = cnext[f];
        }
        T e[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          e[f] = s_end[w][f];
#pragma unroll
          for (int k = 0; k <= f; ++k) e[f] += bsf_mul_int(cnext[k], binom_small(SEG - 1 + f - k, f - k));
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) cnext[f] = e[f];
      }
      if (lane == 0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) s_cin[NW][f] = cnext[f];
      }
    }
    __syncthreads();
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      cin[f] = s_cin[wid][f];
      cnext[f] = s_cin[NW][f];
    }
    // n-th fold += a(i) = sum_k cin_k C(i + n - 1 - k, n - 1 - k), i = position in
    // the segment; a is a polynomial of degree n - 1 in i, stepped by its forward
    // differences: a(i+1) - a(i) = sum_{k<n-1} cin_k C(i + n - 1 - k, n - 2 - k),
    // whose own difference is cin_0 (n = 3)
    {
      const long long i0 = (long long)lane * V;
      T a = cin[NF - 1];
#pragma unroll
      for (int k = 0; k < NF - 1; ++k) a += bsf_mul_int(cin[k], binom_small(i0 + NF - 1 - k, NF - 1 - k));
      T d = 0;
      if constexpr (NF >= 2) {
        d = cin[NF - 2];
        if constexpr (NF == 3) d += bsf_mul_int(cin[0], i0 + 2);
      }
#pragma unroll
      for (int j = 0; j < V; ++j) {
        v[j] += a;
        if constexpr (NF >= 2) {
          a += d;
          if constexpr (NF == 3) d += cin[0];
        }
      }
    }
    // store through shared memory so that each store instruction writes 32
    // consecutive elements of the row
#pragma unroll
    for (int j = 0; j < V; ++j) s_tr[wid][lane * VP + j] = v[j];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < V; ++r) {
      const int e = r * 32 + lane;
      const int xl = x0 + wid * SEG + e;
      if (xl < Wp) store(xl, s_tr[wid][(e / V) * VP + e % V]);
    }
    __syncwarp();
#pragma unroll
    for (int f = 0; f < NF; ++f) carry[f] = cnext[f];
    __syncthreads();  // s_end is rewritten by the next pass
  }
}

template <typename T, int NF, typename In, int V>
__device__ __forceinline__ void scan_row(const In* __restrict__ img, long long ld, int H, int W, int R,
                                         int row0, int boundary, float scale_f, int q, T* __restrict__ S,
                                         long long pitch, int Wp, int yp, float& amax, bool& all_ok) {
  bool yvalid;
  const int ys = bsf_map_index(row0 + yp - R, H, boundary, yvalid);  // row0: first row of a band
  const In* src = img + (long long)ys * ld;
  T* row = S + (long long)yp * pitch;
  row_scan_segments<T, NF, V>(
      Wp,
      [&](int xp) -> T {
        if (!yvalid) return (T)0;
        bool xvalid;
        const int xs = bsf_map_index(xp - R, W, boundary, xvalid);
        if (!xvalid) return (T)0;
        bool ok;
        float ax;
        const T q_ = quantize_one<T, In>(src[xs], q, scale_f, ok, ax);
        all_ok &= ok;
        amax = fmaxf(amax, ax);
        return q_;
      },
      [&](int xp, T val) { row[xp] = val; });
}

// The status of a block's rows: max |Q| and overflow, one atomic per block
// on the status word (per-warp atomics on one word serialise).
__device__ __forceinline__ void scan_rows_status(float amax, bool all_ok, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  __shared__ float s_amax[kRowThreads / 32];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const bool bad = __any_sync(0xffffffffu, !all_ok);
  __syncthreads();
  if (lane == 0) {
    s_amax[threadIdx.x >> 5] = amax;
    if (bad) s_bad = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = s_amax[0];
    for (int w = 1; w < kRowThreads / 32; ++w) m = fmaxf(m, s_amax[w]);
    if (m > 0.f) bsf_atomic_max_pos_float(&st->max_absq_bits, m);
    if (s_bad) bsf_set_error(st, BSF_EOVERFLOW);
  }
}

// One padded row yp: extension, quantisation, n-fold sums, and the block's
// status update.
template <typename T, int NF, typename In, int V>
__device__ __forceinline__ void scan_rows_body(const In* __restrict__ img, long long ld, int H,
                                               int W, int R, int row0, int boundary, float scale_f,
                                               int q, T* __restrict__ S, long long pitch, int Hp,
                                               int Wp, DevStatus* st, int yp) {
  float amax = 0.f;
  bool all_ok = true;
  scan_row<T, NF, In, V>(img, ld, H, W, R, row0, boundary, scale_f, q, S, pitch, Wp, yp, amax, all_ok);
  scan_rows_status(amax, all_ok, st);
}


// ---------------------------------------------------------------------------
// d3 / d2 / d4 in skewed coordinates
// ---------------------------------------------------------------------------
// State after m more rows of zeros: the folds keep adding their lower folds.
template <typename T, int NF>
__device__ __forceinline__ void zero_rows_transfer(T* s, long long m) {
  if constexpr (NF >= 3) s[2] += bsf_mul_int(s[1], m) + bsf_mul_int(s[0], m * (m + 1) / 2);
  if constexpr (NF >= 2) s[1] += bsf_mul_int(s[0], m);
}

// Rows yl of [lo, hi) where the line x = A + B yl lies inside [0, Wp) (the
// interval shrinks to empty when there are none); B in -2..2.
__device__ __forceinline__ int floor_div_pos(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
template <int B>
__device__ __forceinline__ void line_rows(int A, int Wp, int& lo, int& hi) {
  if constexpr (B == 0) {
    if (A < 0 || A >= Wp) hi = lo;
  } else if constexpr (B == 1) {
    lo = max(lo, -A);
    hi = min(hi, Wp - A);
  } else if constexpr (B == -1) {
    lo = max(lo, A - Wp + 1);
    hi = min(hi, A + 1);
  } else if constexpr (B > 0) {  // A + B yl >= 0 and <= Wp - 1
    lo = max(lo, -floor_div_pos(A, B));
    hi = min(hi, floor_div_pos(Wp - 1 - A, B) + 1);
  } else {                       // A - |B| yl <= Wp - 1 and >= 0
    lo = max(lo, -floor_div_pos(Wp - 1 - A, -B));
    hi = min(hi, floor_div_pos(A, -B) + 1);
  }
  if (hi < lo) hi = lo;
}

template <typename T, int NF, int SKEW, bool REV, typename Load = BsfLoadCached>
__device__ __forceinline__ void vscan_agg_body(const T* __restrict__ S, long long pitch, int Hp,
                                               int Wp, int umin, int Nu, int ch,
                                               T* __restrict__ agg, int bx, int c) {
  const int ui = bx * 128 + threadIdx.x;
  if (ui >= Nu) return;
  const int u = umin + ui;
  const int y0 = c * ch, y1 = min(y0 + ch, Hp);
  // in scan order yl the line sits at column x = A + B yl; only the rows with
  // 0 <= x < Wp hold data (the rest of the line is zero)
  const int A = REV ? u + SKEW * (Hp - 1) : u;
  constexpr int B = REV ? -SKEW : SKEW;
  int lo = y0, hi = y1;
  line_rows<B>(A, Wp, lo, hi);
  T s[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) s[f] = 0;
  if (lo < hi) {
#pragma unroll 8
    for (int yl = lo; yl < hi; ++yl) {
      const int y = REV ? Hp - 1 - yl : yl;  // REV: suffix sums, rows bottom-up
      const T v = Load::load(S + (long long)y * pitch + (A + B * yl));
      s[0] += v;
#pragma unroll
      for (int f = 1; f < NF; ++f) s[f] += s[f - 1];
    }
    zero_rows_transfer<T, NF>(s, y1 - hi);  // leading zero rows leave the state at zero
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) agg[((long long)c * NF + f) * Nu + ui] = s[f];
}

// zero-carry combine of the three-phase scan: state after prefix state s
// followed by m rows whose zero-carry state is a
template <typename T, int NF>
__device__ __forceinline__ void tp_combine(T* s, const T* a, long long m) {
  T ns[NF];
  ns[0] = s[0] + a[0];
  if constexpr (NF >= 2) ns[1] = s[1] + bsf_mul_int(s[0], m) + a[1];
  if constexpr (NF >= 3) ns[2] = s[2] + bsf_mul_int(s[1], m) + bsf_mul_int(s[0], m * (m + 1) / 2) + a[2];
#pragma unroll
  for (int f = 0; f < NF; ++f) s[f] = ns[f];
}

// Rescan of one (line, chunk): the carried-in state is folded here from the
// zero-carry states of the earlier chunks of the same line (independent loads
// from L2, so no separate carry pass and no serial chain between launches),
// then the chunk is rescanned in batches of kApplyBatch rows whose loads are
// all issued before any store.
constexpr int kApplyBatch = 16;
constexpr int kFoldUnroll = 4;  // earlier chunks' states loaded per round trip

template <typename T, int NF, int SKEW, bool REV, typename Load = BsfLoadCached>
__device__ __forceinline__ void vscan_apply_body(T* __restrict__ S, long long pitch, int Hp, int Wp,
                                                 int umin, int Nu, int ch, const T* __restrict__ agg,
                                                 int bx, int c) {
  const int ui = bx * 128 + threadIdx.x;
  if (ui >= Nu) return;
  const int u = umin + ui;
  const int y0 = c * ch, y1 = min(y0 + ch, Hp);
  // the rows [glo, ghi) (scan order) where the line holds data: column x = A + B yl
  const int A = REV ? u + SKEW * (Hp - 1) : u;
  constexpr int B = REV ? -SKEW : SKEW;
  int glo = 0, ghi = Hp;
  line_rows<B>(A, Wp, glo, ghi);
  if (glo >= ghi) return;
  const int lo = max(y0, glo), hi = min(y1, ghi);
  if (lo >= hi) return;  // nothing of this line in this chunk
  // carried-in state: the line is zero before its first chunk with data
  T s[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) s[f] = 0;
#pragma unroll kFoldUnroll
  for (int j = glo / ch; j < c; ++j) {
    T a[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) a[f] = Load::load(agg + ((long long)j * NF + f) * Nu + ui);
    tp_combine<T, NF>(s, a, ch);  // every earlier chunk is full
  }
  zero_rows_transfer<T, NF>(s, lo - y0);  // empty rows at the top of this chunk
  const int p32 = (int)pitch;
  for (int yb0 = lo; yb0 < hi; yb0 += kApplyBatch) {
    T v[kApplyBatch];
    int idx[kApplyBatch];
#pragma unroll
    for (int r = 0; r < kApplyBatch; ++r) {
      const int yl = yb0 + r;
      const int y = REV ? Hp - 1 - yl : yl;
      const bool in = yl < hi;
      idx[r] = in ? y * p32 + (A + B * yl) : -1;
      v[r] = in ? Load::load(S + idx[r]) : (T)0;
    }
#pragma unroll
    for (int r = 0; r < kApplyBatch; ++r) {
      s[0] += v[r];
#pragma unroll
      for (int f = 1; f < NF; ++f) s[f] += s[f - 1];
      if (idx[r] >= 0) S[idx[r]] = s[NF - 1];
    }
  }
}

}  // namespace
