// lbm_df64.cuh -- double-word arithmetic for the FP64-storage form that
// computes on the FP32 pipes (storage form 3, LBM_F64_DF), and the collision
// of Eq. 1a written for it.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers: about 48
// significant bits and FP32's exponent range. The operations are built from
// error-free transformations: Knuth's TwoSum (s + e = a + b exactly, any a, b)
// and the FMA form of TwoProd (p + e = a * b exactly, e = fma(a, b, -p)).
// Every FP32 step goes through an intrinsic that is rounded on its own, so the
// compiler never contracts a multiply and an add into an FMA, which would break
// the transformations.
//
// Results are left unnormalised: a sum is TwoSum of the high parts with the
// low parts added to its error term (8 FP32 operations, where renormalising
// with Fast2Sum would take 3 more), a product is TwoProd of the high parts with
// the two cross terms added to its error (4 operations; lo * lo dropped).
// Without the renormalisation |lo| is no longer bounded by half an ulp of hi,
// but it stays within a few ulps of the operands' magnitude (the error term of
// a TwoSum or TwoProd plus low parts of earlier results), so every operation
// keeps an absolute error of about 2^-47 of its operands' magnitude -- the
// bound of the renormalised "sloppy" double-word sum, which is also relative
// to |a| + |b| rather than to |a + b|. The one place that needs a normalised
// operand is the FP32 seed of a reciprocal: recip() renormalises first.
// Operations with an FP32 operand (add_f, mul_f) skip the terms that operand's
// zero low part would contribute.
//
// Conversions from FP64 storage work on the bit patterns with integer
// instructions; on the way out the two parts are added on the FP64 pipe (on
// GB300 the FP64 pipe runs at 1/64 of the FP32 rate).
#pragma once

#include <cstdint>

#include "lbm_device.cuh"

namespace olbm {

// ---------------------------------------------------------------- separately rounded FP32 steps
__device__ __forceinline__ float ef_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float ef_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ef_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ef_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Knuth's TwoSum: s + e = a + b exactly, for any order of magnitude of a and b.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = ef_add(a, b);
  const float v = ef_sub(s, a);
  e = ef_add(ef_sub(a, ef_sub(s, v)), ef_sub(b, v));
}

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // From a double (constants and host-built coefficients): hi the nearest
  // FP32 value, lo the nearest FP32 value of the remainder.
  __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ df64(int i) : df64((double)i) {}

  friend __device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return df64(s, ef_add(e, ef_add(a.lo, b.lo)));
  }
  friend __device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
  friend __device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
  friend __device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
  // TwoProd of the high parts, the cross terms folded into its error.
  friend __device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    const float p = ef_mul(a.hi, b.hi);
    float e = ef_fma(a.hi, b.hi, -p);
    e = ef_fma(a.hi, b.lo, e);
    e = ef_fma(a.lo, b.hi, e);
    return df64(p, e);
  }
  // a b + c: the product as above, then TwoSum with c's high part; the
  // product's error and c's low part join TwoSum's error term.
  friend __device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
    const float p = ef_mul(a.hi, b.hi);
    float e = ef_fma(a.hi, b.hi, -p);
    e = ef_fma(a.hi, b.lo, e);
    e = ef_fma(a.lo, b.hi, e);
    float s, w;
    two_sum(p, c.hi, s, w);
    return df64(s, ef_add(w, ef_add(e, c.lo)));
  }
};

// a + b for an FP32 b (7 operations).
__device__ __forceinline__ df64 add_f(df64 a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  return df64(s, ef_add(e, a.lo));
}
// a b for an FP32 b (3 operations).
__device__ __forceinline__ df64 mul_f(df64 a, float b) {
  const float p = ef_mul(a.hi, b);
  return df64(p, ef_fma(a.lo, b, ef_fma(a.hi, b, -p)));
}
// k x for a power of two k: both parts scaled exactly.
__device__ __forceinline__ df64 scaled(df64 x, float k) { return df64(ef_mul(x.hi, k), ef_mul(x.lo, k)); }
__device__ __forceinline__ df64 fma_scaled(df64 x, float k, df64 c) { return scaled(x, k) + c; }
// hi + lo renormalised (Dekker's Fast2Sum; |hi| >= |lo|): |lo| at most half an ulp of hi.
__device__ __forceinline__ df64 normalised(df64 x) {
  const float h = ef_add(x.hi, x.lo);
  return df64(h, ef_sub(x.lo, ef_sub(h, x.hi)));
}

// 1 / x. The operand is renormalised and its high part's FP32 reciprocal r
// (rcp.approx, relative error below 2^-22) gives the residual e = 1 - x r,
// computed from the exact product of x's high part and r (1 - p is exact for
// p near 1); one cubic Newton step r (1 + e + e^2) in double-word arithmetic
// leaves a relative error of about 2^-47 (the rounding of e) plus e^3. A zero,
// infinite or NaN x gives NaN, and so does |x| >= 2^126, where the seed would
// underflow to zero (a density that large only arises in a simulation that has
// blown up).
__device__ __forceinline__ df64 recip(df64 x) {
  x = normalised(x);
  float r = rcp_seed(x.hi);
  r = (__float_as_uint(r) << 1) == 0u ? __uint_as_float(0x7FC00000u) : r;
  const float p = ef_mul(x.hi, r);
  const float pe = ef_fma(x.hi, r, -p);
  const float e = ef_fma(-x.lo, r, ef_sub(ef_sub(1.0f, p), pe));
  return df64(r, ef_mul(r, ef_fma(e, e, e)));
}

// ---------------------------------------------------------------- paired double-word values
// Two double-word values, one per lane of Blackwell's packed FP32 instructions
// (add/mul/fma .f32x2, each lane rounded as the scalar instruction): one
// instruction serves both. The packed instructions take no negated operands,
// so a subtraction is fma(b, -1, a) (exact: one rounding of a - b) and the
// error of a product is formed against the negated product (one more
// instruction than the scalar TwoProd).
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// TwoSum on both lanes.
__device__ __forceinline__ void two_sum(float2 a, float2 b, float2& s, float2& e) {
  s = p_add(a, b);
  const float2 v = p_sub(s, a);
  e = p_add(p_sub(a, p_sub(s, v)), p_sub(b, v));
}
// The product's high part p and its error e (p + e = a b to double-word accuracy).
__device__ __forceinline__ void two_prod(float2 ahi, float2 alo, float2 bhi, float2 blo, float2& p, float2& e) {
  p = p_mul(ahi, bhi);
  e = p_fma(ahi, bhi, p_mul(p, make_float2(-1.0f, -1.0f)));
  e = p_fma(ahi, blo, e);
  e = p_fma(alo, bhi, e);
}

// Operators are hidden friends: found only by argument-dependent lookup on dw2,
// so they never capture the scalar fma(double, ...) of the enclosing namespace.
struct dw2 {
  float2 hi, lo;
  friend __device__ __forceinline__ dw2 operator+(const dw2& a, const dw2& b) {
    float2 s, e;
    two_sum(a.hi, b.hi, s, e);
    return dw2{s, p_add(e, p_add(a.lo, b.lo))};
  }
  // a - b: TwoSum of a and -b written as a difference, no negation needed.
  friend __device__ __forceinline__ dw2 operator-(const dw2& a, const dw2& b) {
    const float2 s = p_sub(a.hi, b.hi);
    const float2 v = p_sub(s, a.hi);
    const float2 e = p_sub(p_sub(a.hi, p_sub(s, v)), p_add(b.hi, v));
    return dw2{s, p_add(e, p_sub(a.lo, b.lo))};
  }
  friend __device__ __forceinline__ dw2 operator*(const dw2& a, const dw2& b) {
    float2 p, e;
    two_prod(a.hi, a.lo, b.hi, b.lo, p, e);
    return dw2{p, e};
  }
  // a b + c
  friend __device__ __forceinline__ dw2 fma(const dw2& a, const dw2& b, const dw2& c) {
    float2 p, e, s, w;
    two_prod(a.hi, a.lo, b.hi, b.lo, p, e);
    two_sum(p, c.hi, s, w);
    return dw2{s, p_add(w, p_add(e, c.lo))};
  }
  // c - a b: TwoSum of c and -p written as a difference, no negation needed.
  friend __device__ __forceinline__ dw2 fnma(const dw2& a, const dw2& b, const dw2& c) {
    float2 p, e;
    two_prod(a.hi, a.lo, b.hi, b.lo, p, e);
    const float2 s = p_sub(c.hi, p);
    const float2 v = p_sub(s, c.hi);
    const float2 w = p_sub(p_sub(c.hi, p_sub(s, v)), p_add(p, v));
    return dw2{s, p_add(w, p_sub(c.lo, e))};
  }
  // a + k for an FP32 pair k.
  friend __device__ __forceinline__ dw2 add_c(const dw2& a, float2 k) {
    float2 s, e;
    two_sum(a.hi, k, s, e);
    return dw2{s, p_add(e, a.lo)};
  }
  // a k for a pair k of powers of two (or -1, 1): both parts scaled exactly.
  friend __device__ __forceinline__ dw2 scaled_c(const dw2& a, float2 k) { return dw2{p_mul(a.hi, k), p_mul(a.lo, k)}; }
};
__device__ __forceinline__ dw2 pair(df64 x, df64 y) { return dw2{make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)}; }
__device__ __forceinline__ dw2 bcast(df64 x) { return pair(x, x); }
__device__ __forceinline__ df64 lane0(const dw2& v) { return df64(v.hi.x, v.lo.x); }
__device__ __forceinline__ df64 lane1(const dw2& v) { return df64(v.hi.y, v.lo.y); }

// ---------------------------------------------------------------- FP64 <-> double-word
// Split a double into hi + lo with integer instructions: hi takes the sign,
// the exponent and the leading 23 stored mantissa bits (a truncation), lo the
// remaining 29 bits rounded to FP32 (so |lo| < ulp(hi)). NaN and infinity keep
// their class in hi; magnitudes below 2^-126 become zero, above FP32's range
// infinity. Cases are selected without branches.
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

// The same split for 2^-74 <= |d| < 2^128, in seven instructions. The high
// word shifted left by 3 (with the low word's top three bits shifted in) holds
// the FP32 exponent's low seven bits and the 23 mantissa bits in place; bit 30
// of the FP32 exponent equals bit 10 of the FP64 exponent (E - 896 >= 128 iff
// E >= 1024) and bit 31 is the sign, both taken from the high word. lo is the
// remaining 29 bits converted to FP32 and scaled by 2^(E - 1075), a power of two
// whose bit pattern is hi's sign and exponent field less 52 (a normal FP32
// number from E >= 949 on).
__device__ __forceinline__ bool in_fast_split_range(double d) {
  const unsigned h2 = (unsigned)__double2hiint(d) << 1;  // exponent in bits 31..21, sign dropped
  return h2 - (0x3B5u << 21) < ((0x47Fu - 0x3B5u) << 21);
}
__device__ __forceinline__ df64 split_f64_fast(double d) {
  const unsigned h32 = (unsigned)__double2hiint(d), l32 = (unsigned)__double2loint(d);
  const unsigned hib = (__funnelshift_l(l32, h32, 3) & 0x3FFFFFFFu) | (h32 & 0xC0000000u);
  const float scale = __uint_as_float((hib & 0xFF800000u) - (52u << 23));
  return df64(__uint_as_float(hib), __fmul_rn(__uint2float_rn(l32 & 0x1FFFFFFFu), scale));
}

// hi + lo rounded to FP64: hi widened with integer instructions, lo converted
// and added on the FP64 pipe (two FP64-pipe instructions a value). The widening
// rebiases the exponent of a normal FP32 value in place: the high word is
// (u >> 3) + 896 * 2^20 with the sign moved from bit 28 to bit 31 (adding
// 7 * 2^28 for a negative u), the low word u << 29; a zero hi keeps its sign
// and nothing else. An FP32 subnormal hi (below 2^-126, only in the final
// digits of an underflowing value) widens to a number below 2^-126 as well.
// A non-finite hi always comes with a non-finite lo (TwoSum and TwoProd turn
// an overflow or a NaN into NaN or infinity in the error term), so the sum is
// non-finite too, whatever the widened hi.
__device__ __forceinline__ double widen_hi(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned neg = (unsigned)((int)u >> 31) & 0x70000000u;
  const unsigned hw = (u << 1) == 0u ? (u & 0x80000000u) : (u >> 3) + 0x38000000u + neg;
  return __hiloint2double((int)hw, (int)(u << 29));
}
// The same widening with FP32 subnormals flushed to a signed zero (for the low
// part, whose subnormal values must not widen to 2^-127).
__device__ __forceinline__ double widen_lo(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned neg = (unsigned)((int)u >> 31) & 0x70000000u;
  const unsigned hw = (u & 0x7F800000u) == 0u ? (u & 0x80000000u) : (u >> 3) + 0x38000000u + neg;
  return __hiloint2double((int)hw, (u & 0x7F800000u) == 0u ? 0 : (int)(u << 29));
}
__device__ __forceinline__ double join_f64(df64 v) { return widen_hi(v.hi) + (double)v.lo; }
// Both parts widened with integer instructions: one FP64-pipe instruction a value.
__device__ __forceinline__ double join_f64_int(df64 v) { return widen_hi(v.hi) + widen_lo(v.lo); }
// The same sum with both conversions on the FP64 pipe: three FP64-pipe
// instructions and no integer work.
__device__ __forceinline__ double join_f64_fp64pipe(df64 v) { return (double)v.hi + (double)v.lo; }

// Storage form 3: FP64 populations, double-word arithmetic.
template <> struct Form<3> {
  using S = double;
  using T = df64;
  static constexpr bool kShift = false;
};
__device__ __forceinline__ df64 ld_t(const double* p, df64) { return split_f64(__ldg(p)); }
__device__ __forceinline__ void st_t(double* p, df64 v) { *p = join_f64(v); }
__device__ __forceinline__ df64 ld_cg(const double* p, df64) { return split_f64(__ldcg(p)); }
__device__ __forceinline__ double to_double(df64 v) { return join_f64(v); }

// Split a row's nine pulled FP64 populations: the seven-instruction split when
// every value lies in its range (all populations of a live simulation), the
// general split otherwise (zeros, tiny or huge magnitudes, infinities, NaNs).
__device__ __forceinline__ void split_node(const double (&r)[9], df64 (&f)[9]) {
  bool fast = true;
#pragma unroll
  for (int i = 0; i < 9; ++i) fast = fast & in_fast_split_range(r[i]);
  if (fast) {
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = split_f64_fast(r[i]);
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = split_f64(r[i]);
  }
}

// ---------------------------------------------------------------- collision
// The collision of Eq. 1a on double-word values: the product form of
// collide() (lbm_device.cuh) with the same per-axis factors and the same
// closed forms of psi (Eq. 6a), the Eq. 12 prefactor and Pi~ (Eq. 11b), with
// the constants 1 and -1 as FP32 operands and P(a) of Eq. 10 built from
// w = theta + u^2: P(0) = 1 - w, P(+-1) = (w +- u)/2. f holds the pulled
// pre-collision populations; out(i, value) receives each post-collision
// population as soon as it is known (so that its conversion and store overlap
// the rest of the node's arithmetic).
template <int MODEL> __host__ __device__ constexpr bool has_correction(int i) {
  return MODEL == 2 ? (i >= 1 && i <= 4) : ((MODEL == 3 || MODEL == 4) ? i != 0 : false);
}

template <int MODEL, typename Sink, typename Out>
__device__ __forceinline__ void collide_df(const df64 (&f)[9], const Coef<df64>& c, Sink&& sink, Out&& out) {
  // moments (Sec. 1). For the shorter collisions the sums of opposite populations are
  // paired on the packed instructions, lanes (1, 2) with (3, 4) and (5, 6) with (7, 8)
  // (4096^2, diagnostics every step: LBGK 37.9 -> 39.0 GLUPS, the uncorrected model
  // 30.6 -> 30.9); the completely corrected models keep them scalar (25.3 against
  // 25.1 GLUPS paired: their collision already holds the FMA pipe that the packed
  // instructions use, and the warps wait on it).
  constexpr bool kPairMoments = MODEL <= 2 || MODEL == 5;
  df64 s13, s24, s57, s68, d13, d24, d57, d68, t0, t1;
  if constexpr (kPairMoments) {
    const dw2 P12 = pair(f[1], f[2]), P34 = pair(f[3], f[4]), P56 = pair(f[5], f[6]), P78 = pair(f[7], f[8]);
    const dw2 S1 = P12 + P34, D1 = P12 - P34;  // (s13, s24), (d13, d24)
    const dw2 S2 = P56 + P78, D2 = P56 - P78;  // (s57, s68), (d57, d68)
    const dw2 T = S1 + S2;                     // (s13 + s57, s24 + s68)
    s13 = lane0(S1), s24 = lane1(S1), s57 = lane0(S2), s68 = lane1(S2);
    d13 = lane0(D1), d24 = lane1(D1), d57 = lane0(D2), d68 = lane1(D2);
    t0 = lane0(T), t1 = lane1(T);
  } else {
    s13 = f[1] + f[3], d13 = f[1] - f[3];
    s24 = f[2] + f[4], d24 = f[2] - f[4];
    s57 = f[5] + f[7], d57 = f[5] - f[7];
    s68 = f[6] + f[8], d68 = f[6] - f[8];
    t0 = s13 + s57, t1 = s24 + s68;
  }
  const df64 m0 = f[0] + (t0 + t1);
  const df64 jx = d13 + (d57 - d68);
  const df64 jy = d24 + (d57 + d68);
  const df64 rho = m0;
  const df64 inv_rho = recip(rho);
  const df64 ux = jx * inv_rho, uy = jy * inv_rho;
  {
    NodeMoments<df64> mom;
    mom.m0 = m0;
    mom.jx = jx;
    mom.jy = jy;
    mom.ux = ux;
    mom.uy = uy;
    sink(mom);
  }
  const df64 ux2 = ux * ux, uy2 = uy * uy;
  // per-axis GEq factors (Eq. 10)
  const df64 wx = ux2 + c.theta, wy = uy2 + c.theta;
  const df64 px[3] = {scaled(wx - ux, 0.5f), add_f(-wx, 1.0f), scaled(wx + ux, 0.5f)};
  const df64 py[3] = {scaled(wy - uy, 0.5f), add_f(-wy, 1.0f), scaled(wy + uy, 0.5f)};

  if constexpr (MODEL == 5) {
    // LBGK on the polynomial equilibrium: f^eq_(a,b) = rho W_a W_b [1 + s (1 + s/2) - |u|^2/(2 theta)],
    // s = (a u_x + b u_y)/theta (the collide() of lbm_device.cuh, model 5)
    const df64 vx = ux * c.inv_theta, vy = uy * c.inv_theta;
    const df64 t0 = add_f(-((ux2 + uy2) * scaled(c.inv_theta, 0.5f)), 1.0f);  // 1 - |u|^2/(2 theta)
    const df64 orho = c.omega * rho;
    const df64 ow[3] = {orho * c.half_theta, orho * c.one_m_theta, orho * c.half_theta};
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        const int i = pop_index(a, b);
        const df64 sx = a > 0 ? vx : -vx;
        const df64 sy = b > 0 ? vy : -vy;
        const df64 t = a == 0 && b == 0 ? t0
                       : (a == 0 ? fma(sy, add_f(scaled(sy, 0.5f), 1.0f), t0)
                                 : (b == 0 ? fma(sx, add_f(scaled(sx, 0.5f), 1.0f), t0)
                                           : fma(sx + sy, add_f(scaled(sx + sy, 0.5f), 1.0f), t0)));
        const df64 wb = b == 0 ? c.one_m_theta : c.half_theta;
        out(i, fma(ow[a + 1] * wb, t, c.one_m_omega * f[i]));
      }
  } else if constexpr (MODEL == 0) {
    // LBGK: f* = (1 - 1/tau) f + (1/tau) f^eq
    const df64 orho = c.omega * rho;
    const df64 e[3] = {orho * px[0], orho * px[1], orho * px[2]};
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        const int i = pop_index(a, b);
        out(i, fma(e[a + 1], py[b + 1], c.one_m_omega * f[i]));
      }
  } else {
    // Onsager-regularised models (Eq. 2) with corrections (Eqs. 14, 15)
    const df64 Dxy = s13 - s24;    // sum (c_x^2 - c_y^2) f
    const df64 nPxy = s68 - s57;   // -sum c_x c_y f
    const df64 ncy[3] = {add_f(uy, 1.0f), uy, add_f(uy, -1.0f)};  // -C_y(b)
    const df64 dyx2 = uy2 - ux2;
    const df64 A1 = c.k1 * fma(rho, dyx2, Dxy);   // omega' K1
    const df64 nA2 = c.k2 * fma(jx, uy, nPxy);    // -omega' K2
    df64 cor[9];
    if constexpr (MODEL >= 2) {
      const df64 wpsx = (A1 * ux) * (c.c3 - ux2);  // omega' psi_x
      const df64 wpsy = (A1 * uy) * (uy2 - c.c3);  // omega' psi_y
      if constexpr (MODEL == 2) {
        cor[1] = scaled(wpsx, -0.5f);
        cor[3] = scaled(wpsx, 0.5f);
        cor[2] = scaled(wpsy, -0.5f);
        cor[4] = scaled(wpsy, 0.5f);
      } else {
        // u_a^2 (u_a^2 - 1), shared by Eq. 12's mu sum and Eq. 11b's Pi~
        const df64 X = ux2 * add_f(ux2, -1.0f), Y = uy2 * add_f(uy2, -1.0f);
        df64 nhw;  // -omega' pref / 2
        if constexpr (MODEL == 3) {
          nhw = (c.q_inv2t2 * A1) * ((X + Y) + c.tt2);
        } else {
          nhw = scaled(A1, 0.5f);
        }
        const df64 hPxx = nhw * (X + c.tt);        // omega' Pi~_xx / 2
        const df64 hPyy = -(nhw * (Y + c.tt));     // omega' Pi~_yy / 2
        const df64 qPxy = (scaled(nhw, 0.5f) * (ux * uy)) * dyx2;  // omega' Pi~_xy / 4
        const df64 hpsx = scaled(wpsx, 0.5f), hpsy = scaled(wpsy, 0.5f);
        cor[1] = hPyy - hpsx;
        cor[3] = hPyy + hpsx;
        cor[2] = hPxx - hpsy;
        cor[4] = hPxx + hpsy;
        const df64 dsum = scaled(hPxx + hPyy, -0.5f);
        cor[5] = dsum - qPxy;  // c_x c_y = +1
        cor[7] = cor[5];
        cor[6] = dsum + qPxy;  // c_x c_y = -1
        cor[8] = cor[6];
      }
    }
    // f*_(a,b) = P_y(b) [E(a) + C_y(b) (G(a) - B(a) C_y(b))] + omega' Psi_(a,b),
    // E(a) = P_x(a) (rho + A1 C_x(a)^2), B(a) = A1 P_x(a), G(a) = -nA2 P_x(a) C_x(a).
    // Column a = 0 in scalar arithmetic; the columns a = -1 and a = +1 as pairs
    // (lane 0: a = -1, lane 1: a = +1) that share each row's P_y(b), C_y(b).
    const df64 B0 = A1 * px[1];
    const df64 G0 = nA2 * (px[1] * ux);
    const df64 E0 = fma(B0, ux2, rho * px[1]);  // C_x(0)^2 = u_x^2
    const dw2 NCX = add_c(bcast(ux), make_float2(1.0f, -1.0f));                                   // u_x - a
    const dw2 PX = scaled_c(bcast(wx) + scaled_c(bcast(ux), make_float2(-1.0f, 1.0f)), make_float2(0.5f, 0.5f));
    const dw2 B2 = bcast(A1) * PX;
    const dw2 G2 = bcast(nA2) * (PX * NCX);
    const dw2 E2 = fma(B2, NCX * NCX, bcast(rho) * PX);
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
      const int i0 = pop_index(0, b), im = pop_index(-1, b), ip = pop_index(1, b);
      {
        const df64 inner = fma(B0, ncy[b + 1], G0);  // G(0) - B(0) C_y(b)
        const df64 t = fma(-ncy[b + 1], inner, E0);
        out(i0, has_correction<MODEL>(i0) ? fma(py[b + 1], t, cor[i0]) : py[b + 1] * t);
      }
      const dw2 NCY = bcast(ncy[b + 1]);
      const dw2 inner = fma(B2, NCY, G2);
      const dw2 t = fnma(NCY, inner, E2);
      const dw2 F = has_correction<MODEL>(im) ? fma(bcast(py[b + 1]), t, pair(cor[im], cor[ip])) : bcast(py[b + 1]) * t;
      out(im, lane0(F));
      out(ip, lane1(F));
    }
  }
}

}  // namespace olbm
