// lbm_df64.cuh -- double-float arithmetic for the FP64-storage form that
// computes on the FP32 pipes (storage form 3, LBM_F64_DF).
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| at most
// about an ulp of hi: 48 significant bits, relative rounding error near 2^-47
// per operation, FP32's exponent range. The operations are built from
// error-free transformations: Knuth's TwoSum (s + e = a + b exactly), Dekker's
// Fast2Sum (the same when |a| >= |b|) and the FMA form of TwoProd
// (p + e = a * b exactly, e = fma(a, b, -p)). Addition is the variant that
// bounds the error relative to |a| + |b|; multiplication drops the lo * lo
// term. Every FP32 step goes through an intrinsic that is rounded on its own,
// so the compiler never contracts a multiply and an add into an FMA, which
// would break the transformations.
//
// F is float; the operations are also written for f32x2 (two values per
// register pair, Blackwell's packed add/mul/fma.f32x2), which measured slower
// for this collision on GB300: the packed pair state needs about 220 registers
// a thread, too few warps remain to cover the long dependent chains.
//
// Conversions from FP64 storage work on the bit patterns with integer
// instructions; on the way out hi is widened the same way and lo converted and
// added on the FP64 pipe, two FP64-pipe instructions per stored value (on GB300
// the FP64 pipe runs at 1/64 of the FP32 rate). Magnitudes below 2^-126 (about
// 1.2e-38) convert to zero.
#pragma once

#include <cstdint>

#include "lbm_device.cuh"

namespace olbm {

// ---------------------------------------------------------------- separately rounded FP32 steps
__device__ __forceinline__ float ef_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float ef_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ef_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ef_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float ef_fms(float a, float b, float c) { return __fmaf_rn(a, b, -c); }  // a b - c
__device__ __forceinline__ float ef_rcp(float a) { return __frcp_rn(a); }
// f32x2: its operators are the packed intrinsics, each lane rounded once.
__device__ __forceinline__ f32x2 ef_add(f32x2 a, f32x2 b) { return a + b; }
__device__ __forceinline__ f32x2 ef_sub(f32x2 a, f32x2 b) { return a - b; }
__device__ __forceinline__ f32x2 ef_mul(f32x2 a, f32x2 b) { return a * b; }
__device__ __forceinline__ f32x2 ef_fma(f32x2 a, f32x2 b, f32x2 c) { return fma(a, b, c); }
__device__ __forceinline__ f32x2 ef_fms(f32x2 a, f32x2 b, f32x2 c) {
  return f32x2(__ffma2_rn(a.v, b.v, make_float2(-c.v.x, -c.v.y)));
}
__device__ __forceinline__ f32x2 ef_rcp(f32x2 a) { return f32x2(make_float2(__frcp_rn(a.v.x), __frcp_rn(a.v.y))); }

template <class F> struct dfloat {
  F hi, lo;
  dfloat() = default;
  __host__ __device__ dfloat(F h, F l) : hi(h), lo(l) {}
  // From a double (constants and host-built coefficients): hi the nearest
  // FP32 value, lo the nearest FP32 value of the remainder.
  __host__ __device__ dfloat(double d) : hi(F((float)d)), lo(F((float)(d - (double)(float)d))) {}
  __host__ __device__ dfloat(int i) : dfloat((double)i) {}

  // TwoSum of the high parts, the low parts added to the error, Fast2Sum to renormalise.
  friend __device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const F s = ef_add(a.hi, b.hi);
    const F v = ef_sub(s, a.hi);
    F e = ef_add(ef_sub(a.hi, ef_sub(s, v)), ef_sub(b.hi, v));
    e = ef_add(e, ef_add(a.lo, b.lo));
    const F h = ef_add(s, e);
    return dfloat(h, ef_sub(e, ef_sub(h, s)));
  }
  friend __device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
  friend __device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
  friend __device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
  // TwoProd of the high parts, the cross terms folded into its error. The pair
  // (p, e) is returned without renormalising: |e| stays within about an ulp of p
  // (the product of the high parts dominates), which every operation here accepts.
  friend __device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const F p = ef_mul(a.hi, b.hi);
    F e = ef_fms(a.hi, b.hi, p);
    e = ef_fma(a.hi, b.lo, e);
    e = ef_fma(a.lo, b.hi, e);
    return dfloat(p, e);
  }
  // a b + c: the product as above, then TwoSum with c.
  friend __device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) {
    const F p = ef_mul(a.hi, b.hi);
    F e = ef_fms(a.hi, b.hi, p);
    e = ef_fma(a.hi, b.lo, e);
    e = ef_fma(a.lo, b.hi, e);
    const F s = ef_add(p, c.hi);
    const F v = ef_sub(s, p);
    F t = ef_add(ef_sub(p, ef_sub(s, v)), ef_sub(c.hi, v));
    t = ef_add(t, ef_add(e, c.lo));
    const F h = ef_add(s, t);
    return dfloat(h, ef_sub(t, ef_sub(h, s)));
  }
};

template <class F> __device__ __forceinline__ dfloat<F> scaled(dfloat<F> x, float k) {
  return dfloat<F>(ef_mul(x.hi, F(k)), ef_mul(x.lo, F(k)));
}
template <class F> __device__ __forceinline__ dfloat<F> fma_scaled(dfloat<F> x, float k, dfloat<F> c) {
  return scaled(x, k) + c;
}

using df64 = dfloat<float>;

// 1 / x: the FP32 reciprocal of hi, one Newton step r + r (1 - x r) in
// double-float (relative error about 2^-47).
template <class F> __device__ __forceinline__ dfloat<F> recip(dfloat<F> x) {
  const dfloat<F> r(ef_rcp(x.hi), F(0.0f));
  const dfloat<F> e = dfloat<F>(1.0) - x * r;
  return fma(r, e, r);
}

// ---------------------------------------------------------------- FP64 <-> double-float
// Split a double into hi + lo with integer instructions: hi takes the sign,
// the exponent and the leading 23 stored mantissa bits (a truncation), lo the
// remaining 29 bits rounded to FP32 (so |lo| < ulp(hi): the pair is left
// unnormalised, which the operations above accept). NaN and infinity keep their
// class in hi; magnitudes below 2^-126 become zero, above FP32's range infinity.
// Cases are selected without branches.
__device__ __forceinline__ df64 split_f64(double d) {
  const unsigned h32 = (unsigned)__double2hiint(d), l32 = (unsigned)__double2loint(d);
  const unsigned sign = h32 & 0x80000000u;
  const int E = (int)((h32 >> 20) & 0x7FFu);
  const unsigned m23 = ((h32 & 0xFFFFFu) << 3) | (l32 >> 29);
  const unsigned rest = l32 & 0x1FFFFFFFu;
  const int fe = E - 896;  // FP32 biased exponent of the same power of two
  unsigned hib = sign | ((unsigned)min(max(fe, 0), 255) << 23) | m23;
  hib = fe <= 0 ? sign : (fe >= 255 ? (sign | 0x7F800000u | (E == 0x7FF ? (m23 | (rest != 0u)) : 0u)) : hib);
  // rest * 2^(E - 1075): the scale's FP32 exponent E - 948 is clamped at 0 (scale 0)
  // below FP32's normal range, where lo would underflow anyway
  const float scale = __uint_as_float((unsigned)min(max(E - 948, 0), 254) << 23);
  const float lo = (fe > 0 && fe < 255) ? __fmul_rn(__uint2float_rn(rest), scale) : 0.0f;
  return df64(__uint_as_float(hib), __uint_as_float(__float_as_uint(lo) | sign));
}

// hi + lo rounded to FP64: hi widened with integer instructions, lo converted
// and added on the FP64 pipe (two FP64-pipe instructions a value).
__device__ __forceinline__ double join_f64(df64 v) { return widen_f32(v.hi) + (double)v.lo; }
// The same sum with both conversions on the FP64 pipe: three FP64-pipe
// instructions and no integer work. Faster where the FP64 pipe has room beside
// a long double-float collision (the corrected models: +3 to +4 %), slower
// where it does not (LBGK: -18 %, the uncorrected model: -1 %).
__device__ __forceinline__ double join_f64_fp64pipe(df64 v) { return (double)v.hi + (double)v.lo; }

// Storage form 3: FP64 populations, double-float arithmetic.
template <> struct Form<3> {
  using S = double;
  using T = df64;
  static constexpr bool kShift = false;
};
__device__ __forceinline__ df64 ld_t(const double* p, df64) { return split_f64(__ldg(p)); }
__device__ __forceinline__ void st_t(double* p, df64 v) { *p = join_f64(v); }
__device__ __forceinline__ df64 ld_cg(const double* p, df64) { return split_f64(__ldcg(p)); }
__device__ __forceinline__ double to_double(df64 v) { return join_f64(v); }


}  // namespace olbm
