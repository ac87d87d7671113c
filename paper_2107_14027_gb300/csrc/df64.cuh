// Double-float arithmetic for the FP64-accuracy kernels on GB300, whose FP64
// pipe delivers 1/74 of the FP32 rate (measured by fr_fma_probe: 1.06 vs
// 78.6 TFLOP/s).  A value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi) / 2, about 48 significant bits (relative rounding
// about 2^-48 = 3.6e-15 per operation) and FP32's exponent range.
//
// Error-free transformations (published methods, written out here):
//   two_sum       Knuth's branch-free sum: s = fl(a + b) and the exact error
//                 (The Art of Computer Programming, vol. 2, 4.2.2);
//   fast_two_sum  Dekker's sum for |a| >= |b| (Numer. Math. 18, 1971);
//   two_prod      the exact product error from one fused multiply-add.
// Addition is the accurate form that adds both error terms (two two_sums,
// then renormalises), multiplication adds the cross terms with FMAs, the
// square root is one Newton correction of the FP32 root.  Every step uses
// round-to-nearest intrinsics, so the compiler can neither contract nor
// reorder them: a given pair of inputs always gives the same bits, which the
// fused kernel needs (both elements of a face evaluate the same common flux).
#pragma once

#include <cuda_runtime.h>

namespace acmhd {

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit df64(int v) : hi(static_cast<float>(v)), lo(0.0f) {}
  __host__ __device__ explicit df64(double v) {
#ifdef __CUDA_ARCH__
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - static_cast<double>(hi));
#else
    hi = static_cast<float>(v);
    lo = static_cast<float>(v - static_cast<double>(hi));
#endif
  }
  __host__ __device__ explicit operator double() const {
    return static_cast<double>(hi) + static_cast<double>(lo);
  }
};

#ifdef __CUDACC__

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 df_add(df64 x, df64 y) {
  float s1, s2, t1, t2;
  two_sum(x.hi, y.hi, s1, s2);
  two_sum(x.lo, y.lo, t1, t2);
  s2 = __fadd_rn(s2, t1);
  fast_two_sum(s1, s2, s1, s2);
  s2 = __fadd_rn(s2, t2);
  df64 r;
  fast_two_sum(s1, s2, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df64 df_neg(df64 x) { return df64(-x.hi, -x.lo); }

__device__ __forceinline__ df64 df_mul(df64 x, df64 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  df64 r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df64 df_sqrt(df64 x) {
  if (!(x.hi > 0.0f)) return df64(0.0f, 0.0f);
  const float s = __fsqrt_rn(x.hi);
  const float p = __fmul_rn(s, s);
  const float e = __fmaf_rn(s, s, -p);
  // x - s^2, then the Newton correction (x - s^2) / (2 s)
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), e), x.lo);
  const float c = __fdiv_rn(d, __fmul_rn(2.0f, s));
  df64 r;
  fast_two_sum(s, c, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) { return df_add(a, b); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ df64 operator-(df64 a) { return df_neg(a); }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) {
  a = df_add(a, b);
  return a;
}
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return df_add(df_mul(a, b), c); }
using ::fma;   // keep the float / double overloads visible inside the namespace

// value conversions between a storage type and a compute type
template <typename T, typename S>
__device__ __forceinline__ T cvt(S x) {
  return static_cast<T>(x);
}
template <>
__device__ __forceinline__ df64 cvt<df64, double>(double x) {
  return df64(x);
}
template <>
__device__ __forceinline__ double cvt<double, df64>(df64 x) {
  return static_cast<double>(x);
}
template <>
__device__ __forceinline__ df64 cvt<df64, df64>(df64 x) {
  return x;
}

// lane exchange of both halves
__device__ __forceinline__ df64 shfl_up(df64 v, int delta, int width) {
  return df64(__shfl_up_sync(0xffffffffu, v.hi, delta, width),
              __shfl_up_sync(0xffffffffu, v.lo, delta, width));
}
__device__ __forceinline__ df64 shfl_down(df64 v, int delta, int width) {
  return df64(__shfl_down_sync(0xffffffffu, v.hi, delta, width),
              __shfl_down_sync(0xffffffffu, v.lo, delta, width));
}
template <typename T>
__device__ __forceinline__ T shfl_up(T v, int delta, int width) {
  return __shfl_up_sync(0xffffffffu, v, delta, width);
}
template <typename T>
__device__ __forceinline__ T shfl_down(T v, int delta, int width) {
  return __shfl_down_sync(0xffffffffu, v, delta, width);
}

#endif  // __CUDACC__

}  // namespace acmhd
