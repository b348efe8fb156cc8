// Fixed-point quantisation of one input value, shared by the kernels that
// read images (the row pass, the extension pass, the fused tiles):
// Q = round-half-even(f 2^q) as an element of T (two's complement modulo
// 2^bits); floating-point element types keep the value itself.  ok = false
// when the value does not fit; ax = |f 2^q| (an upper bound for |Q|).
#pragma once

#include <type_traits>

#include "bsf_device.cuh"

namespace {

template <typename T, typename In>
__device__ __forceinline__ T quantize_one(In fv, int q, float scale_f, bool& ok, float& ax) {
  if constexpr (!IsFixed<T>::value) {  // floating-point variants: the values themselves
    ok = true;
    ax = 0.f;
    if constexpr (std::is_same<T, double>::value) {
      return (double)fv;
    } else if constexpr (sizeof(In) <= 4) {
      return f32x2((float)fv, 0.f);
    } else {  // float64 input: hi + lo carries its 48 leading bits
      const float h = __double2float_rn(fv);
      return f32x2(h, __double2float_rn(fv - (double)h));
    }
  } else if constexpr (sizeof(In) == 1) {
    ok = true;
    ax = (float)fv * scale_f;
    return (T)fv << q;
  } else if constexpr (sizeof(In) == 4) {
    // f 2^q is exact in float32 (a power-of-two scaling of a finite value
    // that stays finite); below 2^63 the conversion rounds it half to even
    const float x = __fmul_rn(fv, scale_f);
    ax = fabsf(x);
    ok = true;
    if (ax < 2147483648.f) return (T)(long long)__float2int_rn(x);  // 32-bit conversion suffices
    if (ax < 9223372036854775808.f) return (T)(long long)__float2ll_rn(x);
    return bsf_quantize_f32<T>(fv, q, ok);  // large or non-finite: integer path
  } else {
    const double xq = (double)fv * (double)scale_f;
    ax = __double2float_ru(fabs(xq));
    return bsf_round_to_elem<T>(xq, ok);
  }
}

}  // namespace
