// fh_dfloat.cuh -- double-float arithmetic for the float64 residual passes.
//
// A double-float number is the unevaluated sum hi + lo of two float32 values
// with |lo| <= ulp(hi) / 2: about 48 significant bits.  Its operations are
// built from error-free transformations:
//   * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and the exact error
//     e = (a + b) - s, in six additions, for any a, b;
//   * Fast2Sum (Dekker 1971): the same in three additions when |a| >= |b|;
//   * the exact product error fl(a b) - a b = fma(a, b, -fl(a b)).
// Addition is the "sloppy" double-float sum (TwoSum of the high parts, the low
// parts added once): its error is a small multiple of 2^-48 (|a| + |b|), which
// is what a Fourier transform's norm-wise error analysis needs.  Products
// carry the cross terms hi*lo through FMAs.  Every float32 step uses the
// explicitly rounded intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn), which the
// compiler never contracts or reassociates.
//
// On this part float64 arithmetic runs at about 1/64 of the float32 rate, and
// one double-float operation costs 7 (product) to 11 (sum) float32
// instructions, so the float64-accuracy Fourier transforms of the refinement
// residual run several times faster in double-float than in float64.
#pragma once

#include <cuda_runtime.h>

namespace fh {

struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  // Nearest double-float to a float64 value: hi = fl32(x), lo = fl32(x - hi)
  // (x - hi is exact in float64).  With a constant argument the compiler
  // folds it; at run time it costs two conversions and one float64 subtraction.
  __host__ __device__ explicit dfl(double x)
      : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ explicit dfl(int x) : dfl((double)x) {}
};

// complex double-float: 16 bytes, the size of a double2, so a float64
// spectrum tile and its double-float copy take the same shared memory
struct __align__(16) dfc {
  dfl x, y;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfl(s, e);
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, e);
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + dfl(-b.hi, -b.lo); }
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { a = a + b; return a; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { a = a - b; return a; }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// double-float times a float32 value
__device__ __forceinline__ dfl df_mul_f(dfl a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return df_fast_two_sum(p, e);
}
// a / b by one correction of the float32 quotient: q1 = a.hi / b.hi,
// q2 = (a - b q1).hi / b.hi, result q1 + q2 (relative error ~2^-46).
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  const float inv = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, inv);
  const dfl r = a - df_mul_f(b, q1);
  const float q2 = __fmul_rn(r.hi, inv);
  return df_fast_two_sum(q1, q2);
}

__device__ __forceinline__ dfl df_from(double x) {
  const float h = __double2float_rn(x);
  return dfl(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfc dfc_from(double2 v) {
  dfc r;
  r.x = df_from(v.x);
  r.y = df_from(v.y);
  return r;
}
__device__ __forceinline__ double2 dfc_to(dfc v) { return make_double2(df_to(v.x), df_to(v.y)); }

__device__ __forceinline__ dfl df_shfl_xor(dfl v, int m) {
  return dfl(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

}  // namespace fh
