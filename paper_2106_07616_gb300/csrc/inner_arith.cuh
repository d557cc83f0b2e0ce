// inner_arith.cuh -- arithmetic of the inner (FP32-pipe) Krylov iterations.
//
// ArithF32: plain FP32 values, vectors and dot products.
// ArithFF:  float-float ("double-single"): a value is an unevaluated sum
//           hi + lo of two FP32 numbers, about 44-48 significant bits.  Sums
//           use Knuth's TwoSum, products the exact FMA-based TwoProd (Dekker
//           1971; Hida, Li & Bailey 2001 describe the double-double
//           analogue).  Every operation runs on the FP32 pipe, which on
//           GB300 issues 128 lanes per clock per SM against about 1 for FP64,
//           so FF reaches near-FP64 accuracy at a small fraction of FP64 cost.
// Both spell their roundings with __f*_rn intrinsics so the compiler can
// neither contract nor reassociate the error-free transformations.
#pragma once
#include <cuda_runtime.h>

namespace rbffd {

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l = 0.f) : hi(h), lo(l) {}
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return ff_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

// so that the generic reductions (block partials, grid exchange) sum ff
// values on the FP32 pipe
__device__ __forceinline__ ff operator+(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ ff &operator+=(ff &a, ff b) {
  a = ff_add(a, b);
  return a;
}

__device__ __forceinline__ ff ff_from_double(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double ff_to_double(ff v) { return (double)v.hi + (double)v.lo; }

struct ArithF32 {
  using S = float;   // stored values (matrix, vectors)
  using A = float;   // accumulators
  using P = float;   // block / grid partial sums
  using C = float;   // a scalar coefficient in this arithmetic
  static __device__ __forceinline__ A zero() { return 0.f; }
  static __device__ __forceinline__ S szero() { return 0.f; }
  static __device__ __forceinline__ void madd(A &acc, S a, S x) { acc = __fmaf_rn(a, x, acc); }
  static __device__ __forceinline__ A add(A a, A b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ S mul(S a, S b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ S axpy(S y, C al, S x) { return __fmaf_rn(al, x, y); }
  static __device__ __forceinline__ C coef(double v) { return __double2float_rn(v); }
  static __device__ __forceinline__ S from_double(double v) { return __double2float_rn(v); }
  static __device__ __forceinline__ double to_double(S v) { return (double)v; }
  static __device__ __forceinline__ S from_acc(A a) { return a; }
  static __device__ __forceinline__ P part(A a) { return a; }
  static __device__ __forceinline__ double pd(P a) { return (double)a; }
  static __device__ __forceinline__ S ldg(const S *p) { return __ldg(p); }
  static __device__ __forceinline__ S ldcg(const S *p) { return __ldcg(p); }
  static __device__ __forceinline__ A shfl(A v, int src) {
    return __shfl_sync(0xffffffffu, v, src);
  }
};

struct ArithFF {
  using S = ff;
  using A = ff;
  using P = ff;   // partial sums stay float-float: reductions run on the FP32 pipe
  using C = ff;
  static __device__ __forceinline__ A zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ S szero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ void madd(A &acc, S a, S x) { acc = ff_add(acc, ff_mul(a, x)); }
  static __device__ __forceinline__ A add(A a, A b) { return ff_add(a, b); }
  static __device__ __forceinline__ S mul(S a, S b) { return ff_mul(a, b); }
  static __device__ __forceinline__ S axpy(S y, C al, S x) { return ff_add(y, ff_mul(al, x)); }
  static __device__ __forceinline__ C coef(double v) { return ff_from_double(v); }
  static __device__ __forceinline__ S from_double(double v) { return ff_from_double(v); }
  static __device__ __forceinline__ double to_double(S v) { return ff_to_double(v); }
  static __device__ __forceinline__ S from_acc(A a) { return a; }
  static __device__ __forceinline__ P part(A a) { return a; }
  static __device__ __forceinline__ double pd(P a) { return ff_to_double(a); }
  static __device__ __forceinline__ S ldg(const S *p) {
    const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    return {t.x, t.y};
  }
  static __device__ __forceinline__ S ldcg(const S *p) {
    const float2 t = __ldcg(reinterpret_cast<const float2 *>(p));
    return {t.x, t.y};
  }
  static __device__ __forceinline__ A shfl(A v, int src) {
    return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
  }
};

}  // namespace rbffd
