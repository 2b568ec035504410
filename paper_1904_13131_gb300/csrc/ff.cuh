// Double-float ("ff") arithmetic: a value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits. On GB300 the FP32 pipe issues 64 times the FP64 rate, so an FP64-accurate
// tangent action computed in double-float runs on the FP32 pipe instead of the cut FP64 pipe.
//
// Building blocks (all round-to-nearest, written with the _rn intrinsics so that the compiler cannot
// contract or reassociate them):
//   TwoSum (Knuth): s + e = a + b exactly;  FastTwoSum (Dekker): the same when |a| >= |b|;
//   TwoProd with FMA: p + e = a * b exactly.
// The double-word sum is the "sloppy" sum of Dekker (1971): absolute error within a few u^2 (|x| + |y|),
// u = 2^-24, the behaviour of an FP64 sum with a larger unit roundoff. The product follows Dekker's
// mul2 with the FMA form of TwoProd (error a few u^2 |x y|). Transcendentals and reciprocals round-trip
// through FP64 (one operation per Gauss point).
#pragma once
#include <cuda_runtime.h>

namespace hy {

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit constexpr ff(float f) : hi(f), lo(0.f) {}
  __host__ __device__ explicit constexpr ff(int i) : hi((float)i), lo(0.f) {}
};

__host__ __device__ inline double to_double(ff a) { return (double)a.hi + (double)a.lo; }

#ifdef __CUDACC__
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float ap = __fsub_rn(s, b);
  const float bp = __fsub_rn(s, ap);
  return ff(s, __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp)));
}
__device__ __forceinline__ ff operator+(ff x, ff y) {
  const ff s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ ff operator-(ff x) { return ff(-x.hi, -x.lo); }
__device__ __forceinline__ ff operator-(ff x, ff y) { return x + (-y); }
__device__ __forceinline__ ff operator*(ff x, ff y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = __fmaf_rn(x.hi, y.hi, -p);  // exact error of the leading product
  const float t = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
  return fast_two_sum(p, __fadd_rn(e, t));
}
__device__ __forceinline__ ff& operator+=(ff& x, ff y) { return x = x + y; }
__device__ __forceinline__ ff& operator*=(ff& x, ff y) { return x = x * y; }
// x * y + z in one pass: the product's two parts and z summed with one TwoSum
__device__ __forceinline__ ff ff_fma(ff x, ff y, ff z) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e));
  const ff s = two_sum(p, z.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, z.lo)));
}
// conversions between the vector type (double) and ff on the device
__device__ __forceinline__ ff ff_from(double d) {
  const float h = __double2float_rn(d);
  return ff(h, __double2float_rn(__dsub_rn(d, (double)h)));
}
#endif

// Element type of the vectors an action of element type T reads and writes: FP64 for double-float.
template <typename T> struct VecOf { using type = T; };
template <> struct VecOf<ff> { using type = double; };
template <typename T> using vec_t = typename VecOf<T>::type;

#ifdef __CUDACC__
__device__ __forceinline__ float to_elem(float v, float*) { return v; }
__device__ __forceinline__ double to_elem(double v, double*) { return v; }
__device__ __forceinline__ ff to_elem(double v, ff*) { return ff_from(v); }
// read a vector entry as element type T
template <typename T>
__device__ __forceinline__ T vec_in(vec_t<T> v) { return to_elem(v, (T*)nullptr); }
__device__ __forceinline__ float vec_out(float v) { return v; }
__device__ __forceinline__ double vec_out(double v) { return v; }
__device__ __forceinline__ double vec_out(ff v) { return __dadd_rn((double)v.hi, (double)v.lo); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ ff rcp_rn(ff x) { return ff_from(__drcp_rn(vec_out(x))); }
#endif

}  // namespace hy

#ifdef __CUDACC__
// fma and log for double-float live in the global namespace beside the float and double overloads, so that
// the unqualified calls of the generic kernels resolve among all three.
__device__ __forceinline__ hy::ff fma(hy::ff x, hy::ff y, hy::ff z) { return hy::ff_fma(x, y, z); }
__device__ __forceinline__ hy::ff log(hy::ff x) { return hy::ff_from(::log(hy::vec_out(x))); }
#endif
