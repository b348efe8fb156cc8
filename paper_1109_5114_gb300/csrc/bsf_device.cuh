// Device helpers shared by the kernels of libbsf.so: element types of the
// running sums, boundary extension, fixed-point quantisation, exact
// integer -> float rounding, warp shuffles of wide integers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bsf_internal.h"

typedef unsigned __int128 u128;
typedef __int128 i128;

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the kernel before it on the stream is still
// running; bsf_grid_dep_wait() blocks until that kernel has completed and its
// writes are visible (a no-op when the launch had no such dependency), and
// bsf_grid_dep_launch() lets the dependent kernel's blocks be scheduled once
// every block of this kernel has called it or exited.
__device__ __forceinline__ void bsf_grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void bsf_grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void bsf_set_error(DevStatus* st, int code) {
  atomicCAS(&st->err, 0, code);
}

// Non-negative floating-point values order like their bit patterns, so a
// running maximum can be kept with an integer atomicMax.
__device__ __forceinline__ void bsf_atomic_max_pos_double(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void bsf_atomic_max_pos_float(unsigned* addr, float v) {
  atomicMax(addr, __float_as_uint(v));
}

// ----------------------------------------------------------------------------
// Boundary extension: map a coordinate of the padded domain into [0, N).
// Half-sample symmetric extension repeats with period 2N: d c b a | a b c d.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int bsf_map_index(int i, int N, int boundary, bool& valid) {
  valid = true;
  if (i >= 0 && i < N) return i;
  if (boundary == BSF_ZERO) { valid = false; return 0; }
  if (boundary == BSF_REPLICATE) return i < 0 ? 0 : N - 1;
  int m = i % (2 * N);
  if (m < 0) m += 2 * N;
  return m >= N ? 2 * N - 1 - m : m;
}

// ----------------------------------------------------------------------------
// Element types of the running sums.  The fixed-point types wrap modulo 2^b;
// the floating-point precision variants are float64 and a double-float
// (an unevaluated sum hi + lo of two float32, added with error-free
// transformations: the compensated float32 running sums).
// ----------------------------------------------------------------------------
struct f32x2 {
  float hi, lo;
  __host__ __device__ f32x2() : hi(0.f), lo(0.f) {}
  __host__ __device__ f32x2(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ f32x2(float h, float l) : hi(h), lo(l) {}
};

// Knuth's TwoSum (s + e == a + b exactly) and the renormalisation of a
// double-float, both written out with IEEE round-to-nearest float32 steps.
__device__ __forceinline__ f32x2 ddf_renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return f32x2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ f32x2 ddf_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return f32x2(s, e);
}
__device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b) {
  const f32x2 t = ddf_two_sum(a.hi, b.hi);
  return ddf_renorm(t.hi, __fadd_rn(t.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ f32x2 operator-(f32x2 a) { return f32x2(-a.hi, -a.lo); }
__device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b) { return a + (-b); }
__device__ __forceinline__ f32x2& operator+=(f32x2& a, f32x2 b) { a = a + b; return a; }

template <typename T> struct ElemBits;
template <> struct ElemBits<uint32_t> { static constexpr int value = 32; };
template <> struct ElemBits<uint64_t> { static constexpr int value = 64; };
template <> struct ElemBits<u128> { static constexpr int value = 128; };

template <typename T> struct IsFixed { static constexpr bool value = false; };
template <> struct IsFixed<uint32_t> { static constexpr bool value = true; };
template <> struct IsFixed<uint64_t> { static constexpr bool value = true; };
template <> struct IsFixed<u128> { static constexpr bool value = true; };

// v * m for a small non-negative integer m
template <typename T> __device__ __forceinline__ T bsf_mul_int(T v, long long m) { return v * (T)m; }
template <> __device__ __forceinline__ f32x2 bsf_mul_int<f32x2>(f32x2 v, long long m) {
  const float mf = (float)m;  // exact: m < 2^24
  const float p = __fmul_rn(v.hi, mf);
  const float e = __fmaf_rn(v.hi, mf, -p);  // exact error of the product
  return ddf_renorm(p, __fadd_rn(e, __fmul_rn(v.lo, mf)));
}

template <typename T> __device__ __forceinline__ T bsf_load(const T* p);
template <> __device__ __forceinline__ double bsf_load<double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ f32x2 bsf_load<f32x2>(const f32x2* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return f32x2(v.x, v.y);
}
template <> __device__ __forceinline__ uint32_t bsf_load<uint32_t>(const uint32_t* p) { return __ldg(p); }
template <> __device__ __forceinline__ uint64_t bsf_load<uint64_t>(const uint64_t* p) {
  return __ldg(reinterpret_cast<const unsigned long long*>(p));
}
template <> __device__ __forceinline__ u128 bsf_load<u128>(const u128* p) {
  ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p));
  return ((u128)v.y << 64) | (u128)v.x;
}

// Loads of data that other blocks of the same launch wrote (persistent
// kernels): bsf_load_coherent reads at L2 (the point of coherence) and leaves
// L1 alone; bsf_load_weak is a plain L1-cached load, valid for data that no
// block of the launch writes after the reader's acquire (no L1 line of it was
// filled earlier in the launch).
template <typename T> __device__ __forceinline__ T bsf_load_coherent(const T* p);
template <> __device__ __forceinline__ uint64_t bsf_load_coherent<uint64_t>(const uint64_t* p) {
  return __ldcg(reinterpret_cast<const unsigned long long*>(p));
}
template <typename T> __device__ __forceinline__ T bsf_load_weak(const T* p);
template <> __device__ __forceinline__ uint64_t bsf_load_weak<uint64_t>(const uint64_t* p) {
  unsigned long long v;
  asm volatile("ld.global.ca.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

template <typename T> __device__ __forceinline__ T bsf_shfl_up(T v, int d);
template <> __device__ __forceinline__ double bsf_shfl_up<double>(double v, int d) {
  return __shfl_up_sync(0xffffffffu, v, d);
}
template <> __device__ __forceinline__ f32x2 bsf_shfl_up<f32x2>(f32x2 v, int d) {
  return f32x2(__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d));
}
template <> __device__ __forceinline__ uint32_t bsf_shfl_up<uint32_t>(uint32_t v, int d) {
  return __shfl_up_sync(0xffffffffu, v, d);
}
template <> __device__ __forceinline__ uint64_t bsf_shfl_up<uint64_t>(uint64_t v, int d) {
  return __shfl_up_sync(0xffffffffu, (unsigned long long)v, d);
}
template <> __device__ __forceinline__ u128 bsf_shfl_up<u128>(u128 v, int d) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  lo = __shfl_up_sync(0xffffffffu, lo, d);
  hi = __shfl_up_sync(0xffffffffu, hi, d);
  return ((u128)hi << 64) | (u128)lo;
}
template <typename T> __device__ __forceinline__ T bsf_shfl_idx(T v, int src);
template <> __device__ __forceinline__ double bsf_shfl_idx<double>(double v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
template <> __device__ __forceinline__ f32x2 bsf_shfl_idx<f32x2>(f32x2 v, int src) {
  return f32x2(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}
template <> __device__ __forceinline__ uint32_t bsf_shfl_idx<uint32_t>(uint32_t v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
template <> __device__ __forceinline__ uint64_t bsf_shfl_idx<uint64_t>(uint64_t v, int src) {
  return __shfl_sync(0xffffffffu, (unsigned long long)v, src);
}
template <> __device__ __forceinline__ u128 bsf_shfl_idx<u128>(u128 v, int src) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  lo = __shfl_sync(0xffffffffu, lo, src);
  hi = __shfl_sync(0xffffffffu, hi, src);
  return ((u128)hi << 64) | (u128)lo;
}

// ----------------------------------------------------------------------------
// Fixed-point quantisation Q = round-half-even(x), x = f 2^q already scaled
// (exact for float inputs).  ok = false when |x| does not fit the element.
// ----------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T bsf_round_to_elem(double x, bool& ok);

template <> __device__ __forceinline__ uint32_t bsf_round_to_elem<uint32_t>(double x, bool& ok) {
  // |x| < 2^31 - 1 keeps the rounded value inside int32
  ok = fabs(x) < 2147483647.0;
  return ok ? (uint32_t)__double2int_rn(x) : 0u;
}

template <> __device__ __forceinline__ uint64_t bsf_round_to_elem<uint64_t>(double x, bool& ok) {
  // |x| < 2^63 - 1024 keeps the rounded value inside int64
  ok = fabs(x) < 9223372036854774784.0;
  return ok ? (uint64_t)__double2ll_rn(x) : 0ull;
}

template <> __device__ __forceinline__ u128 bsf_round_to_elem<u128>(double x, bool& ok) {
  double ax = fabs(x);
  if (ax < 9223372036854774784.0) { ok = true; return (u128)(i128)__double2ll_rn(x); }
  ok = ax < 1.7014118346046923e38;  // 2^127
  if (!ok) return 0;
  // |x| >= 2^63 is an integer: value = mantissa * 2^(exponent - 52)
  unsigned long long b = (unsigned long long)__double_as_longlong(ax);
  int e = (int)((b >> 52) & 0x7ff) - 1075;
  u128 m = (u128)((b & 0xfffffffffffffull) | 0x10000000000000ull);
  u128 v = m << e;
  return x < 0 ? (u128)(-(i128)v) : v;
}

// Q = round-half-even(f 2^q) of a float32 f with integer operations only
// (f = M 2^e exactly, so Q = M 2^(e+q) rounded).  ok = false for a
// non-finite f or a |Q| that needs more than bits-1 bits.
template <typename T>
__device__ __forceinline__ T bsf_quantize_f32(float f, int q, bool& ok) {
  const unsigned b = __float_as_uint(f);
  const unsigned E = (b >> 23) & 0xffu;
  unsigned M = b & 0x7fffffu;
  ok = E != 0xffu;
  int e;
  if (E == 0) { e = -149; } else { M |= 0x800000u; e = (int)E - 150; }
  const int s = e + q;
  T Q;
  if (M == 0) {
    Q = 0;
  } else if (s >= 0) {
    const int bl = 32 - __clz(M);
    ok = ok && (bl + s <= (int)(8 * sizeof(T)) - 1);
    Q = ok ? ((T)M << s) : (T)0;
  } else {
    const int r = -s;
    if (r >= 25) {
      Q = 0;
    } else {
      unsigned qi = M >> r;
      const unsigned rem = M & ((1u << r) - 1u);
      const unsigned half = 1u << (r - 1);
      if (rem > half || (rem == half && (qi & 1u))) ++qi;
      Q = (T)qi;
    }
  }
  return (b >> 31) ? (T)((T)0 - Q) : Q;
}

// ----------------------------------------------------------------------------
// Round an exact signed integer to the nearest float32 / float64, ties to
// even.  64-bit values use the CUDA conversion intrinsics (documented as
// round-to-nearest-even); 128-bit values are rounded here with integer ops.
// ----------------------------------------------------------------------------
__device__ __forceinline__ double bsf_pow2_f64(int e) {  // 2^e, -1022 <= e <= 1023
  return __longlong_as_double((long long)(e + 1023) << 52);
}
__device__ __forceinline__ float bsf_pow2_f32(int e) {   // 2^e, -126 <= e <= 127
  return __int_as_float((e + 127) << 23);
}

// keep the top `keep` significant bits of m (bit length bl > keep), rounded
// half to even; returns the rounded top part and sets the scale exponent
__device__ __forceinline__ unsigned long long bsf_round_top(u128 m, int bl, int keep, int& sh) {
  sh = bl - keep;
  u128 top = m >> sh;
  u128 rem = m - (top << sh);
  u128 half = (u128)1 << (sh - 1);
  if (rem > half || (rem == half && (top & 1))) top += 1;
  return (unsigned long long)top;
}

__device__ __forceinline__ int bsf_bitlen128(u128 m) {
  unsigned long long hi = (unsigned long long)(m >> 64);
  if (hi) return 128 - __clzll((long long)hi);
  unsigned long long lo = (unsigned long long)m;
  return lo ? 64 - __clzll((long long)lo) : 0;
}

__device__ __forceinline__ float bsf_rn32(i128 a) {
  bool neg = a < 0;
  u128 m = neg ? (u128)0 - (u128)a : (u128)a;
  if ((m >> 63) == 0) {
    float r = __ll2float_rn((long long)m);
    return neg ? -r : r;
  }
  int sh;
  unsigned long long top = bsf_round_top(m, bsf_bitlen128(m), 24, sh);
  float r = __ull2float_rn(top) * bsf_pow2_f32(sh);  // exact: top <= 2^24
  return neg ? -r : r;
}

__device__ __forceinline__ double bsf_rn64(i128 a) {
  bool neg = a < 0;
  u128 m = neg ? (u128)0 - (u128)a : (u128)a;
  if ((m >> 63) == 0) {
    double r = __ll2double_rn((long long)m);
    return neg ? -r : r;
  }
  int sh;
  unsigned long long top = bsf_round_top(m, bsf_bitlen128(m), 53, sh);
  double r = __ull2double_rn(top) * bsf_pow2_f64(sh);  // exact: top <= 2^53
  return neg ? -r : r;
}

// float32 nearest to an unsigned 64-bit integer, ties to even, built from
// its bits with integer operations
__device__ __forceinline__ float bsf_rn32_u64(unsigned long long m) {
  if (m == 0) return 0.f;
  const int bl = 64 - __clzll((long long)m);
  unsigned long long top;
  int ex = bl - 1;
  if (bl <= 24) {
    top = m << (24 - bl);
  } else {
    const int sh = bl - 24;
    top = m >> sh;
    const unsigned long long rem = m & ((1ull << sh) - 1ull);
    const unsigned long long half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (top & 1ull))) ++top;
    if (top >> 24) { top >>= 1; ++ex; }
  }
  return __uint_as_float(((unsigned)(ex + 127) << 23) | ((unsigned)top & 0x7fffffu));
}
__device__ __forceinline__ float bsf_rn32_i64(long long a) {
  const unsigned long long m = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
  const float r = bsf_rn32_u64(m);
  return a < 0 ? -r : r;
}

__device__ __forceinline__ float bsf_rn32_u(u128 m) {
  if ((m >> 64) == 0) return __ull2float_rn((unsigned long long)m);
  int sh;
  unsigned long long top = bsf_round_top(m, bsf_bitlen128(m), 24, sh);
  return __ull2float_rn(top) * bsf_pow2_f32(sh);
}

__device__ __forceinline__ double bsf_rn64_u(u128 m) {
  if ((m >> 64) == 0) return __ull2double_rn((unsigned long long)m);
  int sh;
  unsigned long long top = bsf_round_top(m, bsf_bitlen128(m), 53, sh);
  return __ull2double_rn(top) * bsf_pow2_f64(sh);
}
