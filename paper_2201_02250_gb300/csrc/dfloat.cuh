// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, giving a 48-bit significand (unit roundoff about 2^-47) and FP32's exponent
// range, computed entirely on the FP32 pipe.  On GB300 the FP32 pipe issues about 60 times more
// instructions per cycle than the FP64 pipe, so the 10-20 FP32 instructions of a double-float
// multiply-add still beat one FP64 FMA by a wide margin.  The error-free transformations are the
// published ones: TwoSum (Knuth, TAOCP vol. 2) and the FMA form of TwoProduct (Dekker 1971; see
// also Hida, Li and Bailey, "Algorithms for quad-double precision floating point arithmetic", 2001).
// Every primitive uses explicitly rounded intrinsics so that the compiler cannot contract or
// reassociate the compensation steps.
#pragma once

#include <cuda_runtime.h>

namespace a2ls {

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ dfloat(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr dfloat(float x) : hi(x), lo(0.f) {}
  __host__ __device__ dfloat(int x) : dfloat((double)x) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

#ifdef __CUDACC__
// s + e = a + b exactly
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return dfloat(s, e);
}

// s + e = a + b exactly, provided |a| >= |b| or a == 0
__device__ __forceinline__ dfloat df_quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const dfloat s = df_two_sum(a.hi, b.hi);
  return df_quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick_two_sum(p, e);
}
// quotient to double-float accuracy by one correction step of the FP32 estimate
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dfloat r = a - b * dfloat(q1, 0.f);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return df_quick_two_sum(q1, q2);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }

// acc += a * b without the final renormalisation: the pair (hi, lo) keeps the exact sum of the
// rounded partial results, |lo| may exceed ulp(hi) / 2 but stays far below |hi| over a tile's
// worth of terms.  Call df_normalize before the value leaves the accumulator.
__device__ __forceinline__ void df_mac(dfloat& acc, dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const dfloat s = df_two_sum(acc.hi, p);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ dfloat df_normalize(dfloat a) { return df_quick_two_sum(a.hi, a.lo); }

__device__ __forceinline__ dfloat& operator/=(dfloat& a, dfloat b) { return a = a / b; }
// ordering of normalised values (|lo| <= ulp(hi) / 2)
__device__ __forceinline__ bool operator<(dfloat a, dfloat b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(dfloat a, dfloat b) { return b < a; }
__device__ __forceinline__ bool operator<=(dfloat a, dfloat b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(dfloat a, dfloat b) { return !(a < b); }
__device__ __forceinline__ bool operator==(dfloat a, dfloat b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(dfloat a, dfloat b) { return !(a == b); }
// scalar helpers used by the small dense eigensolver when it runs in double-float
__device__ __forceinline__ dfloat se_abs(dfloat a) { return (a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f)) ? -a : a; }
// square root: the FP32 root refined by one Newton step in double-float
__device__ __forceinline__ dfloat se_sqrt(dfloat a) {
  if (!(a.hi > 0.f)) return dfloat(0.f, 0.f);
  const float s = __fsqrt_rn(a.hi);
  const dfloat r = a - dfloat(s, 0.f) * dfloat(s, 0.f);
  return df_quick_two_sum(s, __fdiv_rn(r.hi, 2.f * s));
}
__device__ __forceinline__ double se_dbl(dfloat a) { return (double)a; }
__device__ __forceinline__ void se_mac(dfloat& acc, dfloat a, dfloat b) { df_mac(acc, a, b); }
__device__ __forceinline__ dfloat se_fin(dfloat a) { return df_normalize(a); }

__device__ __forceinline__ dfloat shfl_xor(dfloat v, int lane_mask) {
  return dfloat(__shfl_xor_sync(0xffffffffu, v.hi, lane_mask), __shfl_xor_sync(0xffffffffu, v.lo, lane_mask));
}
#endif

// generic multiply-add and normalisation used by the templated tile products
template <class T>
__device__ __forceinline__ void mac(T& acc, T a, T b) { acc += a * b; }
#ifdef __CUDACC__
template <>
__device__ __forceinline__ void mac<dfloat>(dfloat& acc, dfloat a, dfloat b) { df_mac(acc, a, b); }
#endif
template <class T>
__device__ __forceinline__ T finish(T a) { return a; }
#ifdef __CUDACC__
template <>
__device__ __forceinline__ dfloat finish<dfloat>(dfloat a) { return df_normalize(a); }
#endif

template <class T>
__device__ __forceinline__ T warp_xor(T v, int lane_mask) { return __shfl_xor_sync(0xffffffffu, v, lane_mask); }
#ifdef __CUDACC__
template <>
__device__ __forceinline__ dfloat warp_xor<dfloat>(dfloat v, int lane_mask) { return shfl_xor(v, lane_mask); }
#endif

// unit roundoff of each arithmetic (double-float: 2^-47, allowing for the unnormalised accumulations)
template <class T> struct Unit;
template <> struct Unit<float> { static constexpr double u = 5.9604644775390625e-08; };
template <> struct Unit<double> { static constexpr double u = 1.1102230246251565e-16; };
template <> struct Unit<dfloat> { static constexpr double u = 7.105427357601002e-15; };

}  // namespace a2ls
