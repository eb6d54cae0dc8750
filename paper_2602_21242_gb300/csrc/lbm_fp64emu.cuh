// lbm_fp64emu.cuh -- IEEE 754 binary64 addition and multiplication, rounded to
// nearest with ties to even, computed with integer instructions.
//
// On GB300 the FP64 pipe retires two FP64 operations per clock per SM (1/64 of
// the FP32 rate) and bounds the FP64 kernels, while their integer and FP32
// pipes stand almost idle. These routines give the correctly rounded binary64
// sum and product from the bit fields of the operands (IEEE 754-2019, 4.3.1 and
// 6.1: the exact result, rounded once), so an FP64 kernel can hand part of its
// additions and products to the integer pipes and get the same bits as the FP64
// pipe would give. Written from the definition: align, add, normalise, round on
// the guard bits with a sticky bit (a textbook soft-float scheme, e.g. Muller
// et al., Handbook of Floating-Point Arithmetic, ch. 8).
//
// Fast paths cover normal operands with a normal result (for sums, exponents
// at most 31 apart and no cancellation of more than 31 bits; for products, on
// request, zero operands too). Everything else (a zero, subnormal, infinite or
// NaN operand, a result below the normal range or past the largest finite value
// before rounding) goes to the FP64 instruction itself, which gives the same
// correctly rounded result, or, in the product's unchecked form, comes out as a
// quiet NaN for the caller to find and redo; a rounding that carries past the
// largest finite value comes out as infinity, as it must.
//
// The routines compile for the host as well (plain C++ with 128-bit integer
// products), where tests compare them bit for bit with the host's binary64
// arithmetic.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define OLBM_EMU_HD __host__ __device__ __forceinline__
#else
#define OLBM_EMU_HD inline
#endif

namespace olbm {
namespace emu {

OLBM_EMU_HD uint64_t bits_of(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}

OLBM_EMU_HD double double_of(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, sizeof x);
  return x;
#endif
}

// 32-bit word helpers: leading zeros (32 for zero), and the high word of
// (hi:lo) << s and the low word of (hi:lo) >> s for 0 <= s <= 31.
OLBM_EMU_HD int clz32(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __clz((int)x);
#else
  return x != 0 ? __builtin_clz(x) : 32;
#endif
}
OLBM_EMU_HD uint32_t shl_hi(uint32_t lo, uint32_t hi, int s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_l(lo, hi, s);
#else
  return (uint32_t)(((((uint64_t)hi << 32) | lo) << (s & 31)) >> 32);
#endif
}
OLBM_EMU_HD uint32_t shr_lo(uint32_t lo, uint32_t hi, int s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_r(lo, hi, s);
#else
  return (uint32_t)((((uint64_t)hi << 32) | lo) >> (s & 31));
#endif
}

// The FP64 instructions, for the cases the fast paths leave out. On the device
// they sit out of line, so the rare branch that takes them is a real branch and
// not an FP64 instruction issued under a predicate by every thread.
#if defined(__CUDACC__)
__device__ __noinline__ inline double add_fp64(double a, double b) { return __dadd_rn(a, b); }
__device__ __noinline__ inline double mul_fp64(double a, double b) { return __dmul_rn(a, b); }
#endif
OLBM_EMU_HD double add_fallback(double a, double b) {
#if defined(__CUDA_ARCH__)
  return add_fp64(a, b);
#else
  volatile double s = a + b;
  return s;
#endif
}
OLBM_EMU_HD double mul_fallback(double a, double b) {
#if defined(__CUDA_ARCH__)
  return mul_fp64(a, b);
#else
  volatile double p = a * b;
  return p;
#endif
}

// Whether any thread of the warp needs the FP64 instruction: a warp-uniform
// branch, so the compiler cannot turn the rare fallback into an FP64
// instruction that every thread issues under a predicate.
OLBM_EMU_HD bool take_fallback(bool fast) {
#if defined(__CUDA_ARCH__)
  return __any_sync(__activemask(), !fast);
#else
  return !fast;
#endif
}

constexpr uint64_t kSign = 0x8000000000000000ull;

// m (53 bits, leading bit at 52, before rounding) with the 11 bits below it in
// rem (half = 0x400, any lower non-zero bits already ORed into bit 0), rounded
// to nearest, ties to even, and packed with exponent field e (1 <= e <= 2046)
// and the sign bit: a mantissa that rounds up to 2^53 carries into the exponent
// field (infinity past the largest finite value).
OLBM_EMU_HD uint64_t round_pack(uint64_t sign, int e, uint64_t m, uint32_t rem) {
  const uint64_t inc = (rem > 0x400u || (rem == 0x400u && (m & 1u))) ? 1u : 0u;
  return sign | ((((uint64_t)(e - 1)) << 52) + m + inc);
}

// a + b, correctly rounded (round to nearest, ties to even). Works on 32-bit
// words throughout (a 64-bit magnitude comparison, for one, would take an
// FP64-pipe instruction): the operands are ordered by exponent, and a negative
// difference (possible only for equal exponents, where nothing is shifted out)
// is negated exactly. The fast path takes alignment shifts of at most 31 bits
// and results that keep their leading bit in the high word before
// normalisation (a cancellation of more than 31 bits goes to the FP64
// instruction).
OLBM_EMU_HD double add64(double a, double b) {
  const uint64_t ua = bits_of(a), ub = bits_of(b);
  const uint32_t ah = (uint32_t)(ua >> 32), bh = (uint32_t)(ub >> 32);
  const int ea = (int)((ah >> 20) & 0x7FF), eb = (int)((bh >> 20) & 0x7FF);
  const bool swap = eb > ea;
  const uint64_t x = swap ? ub : ua, y = swap ? ua : ub;
  const int ex = swap ? eb : ea, ey = swap ? ea : eb;
  const uint32_t xh = (uint32_t)(x >> 32), xl = (uint32_t)x, yh = (uint32_t)(y >> 32), yl = (uint32_t)y;
  // significands with the hidden bit at 62: ten guard bits below, one bit of headroom above
  const uint32_t Ah = shl_hi(xl, (xh & 0xFFFFFu) | 0x100000u, 10), Al = xl << 10;
  const uint32_t Bh = shl_hi(yl, (yh & 0xFFFFFu) | 0x100000u, 10), Bl = yl << 10;
  const int d = ex - ey, s = d & 31;
  uint32_t Bsl = shr_lo(Bl, Bh, s);
  const uint32_t Bsh = Bh >> s;
  Bsl |= (Bl & ((1u << s) - 1u)) != 0 ? 1u : 0u;  // sticky: y's bits shifted out leave the sum odd
  const uint64_t A = ((uint64_t)Ah << 32) | Al, Bs = ((uint64_t)Bsh << 32) | Bsl;
  const bool sub = ((ah ^ bh) & 0x80000000u) != 0;
  uint64_t S = sub ? A - Bs : A + Bs;
  const bool neg = sub && (int64_t)S < 0;
  S = neg ? (uint64_t)0 - S : S;
  // normalise the leading bit to 63: no shift after a carry, one bit for an
  // ordinary sum, more only after a cancellation (d <= 1, nothing shifted out)
  const uint32_t Sh = (uint32_t)(S >> 32), Sl = (uint32_t)S;
  const int lz = clz32(Sh), l = lz & 31;
  const uint32_t Nh = shl_hi(Sl, Sh, l), Nl = Sl << l;
  const int e = ex + 1 - lz;
  const bool fast = ey != 0 && ex != 0x7FF && d <= 31 && Sh != 0 && e >= 1 && e <= 2046;
  const uint64_t m = ((uint64_t)(Nh >> 11) << 32) | shr_lo(Nl, Nh, 11);
  const double r = double_of(round_pack((x & kSign) ^ (neg ? kSign : 0u), e, m, Nl & 0x7FFu));
  return take_fallback(fast) ? (fast ? r : add_fallback(a, b)) : r;
}

// a * b, correctly rounded (round to nearest, ties to even), in 32-bit words:
// the significands with the hidden bit at 63 (the shift drops sign and exponent
// bits; the lowest exponent bit lands on 63 and is set to one), their 128-bit
// product from four 32 x 32 -> 64-bit multiply-adds, a normalisation by at most
// one bit, and the rounding increment (rem + lsb > half) carried into the packed
// exponent field.
// CHECKED = false leaves out the fallback: a product outside the fast path
// comes out as a quiet NaN, which every later sum, product or FMA propagates,
// so a caller that checks its results for non-finite values once (and redoes
// those with the FP64 instruction) needs no branch per product. ZEROS = true
// takes zero operands on the fast path too (a few more instructions).
template <bool CHECKED = true, bool ZEROS = false>
OLBM_EMU_HD double mul64(double a, double b) {
  const uint64_t ua = bits_of(a), ub = bits_of(b);
  const uint32_t ah = (uint32_t)(ua >> 32), al = (uint32_t)ua, bh = (uint32_t)(ub >> 32), bl = (uint32_t)ub;
  const int ea = (int)((ah >> 20) & 0x7FF), eb = (int)((bh >> 20) & 0x7FF);
  const uint32_t a1 = shl_hi(al, ah, 11) | 0x80000000u, a0 = al << 11;
  const uint32_t b1 = shl_hi(bl, bh, 11) | 0x80000000u, b0 = bl << 11;
  // 128-bit product (w3 w2 w1 w0)
  const uint64_t p00 = (uint64_t)a0 * b0;
  const uint64_t t = (uint64_t)a0 * b1 + (p00 >> 32);
  const uint64_t u = (uint64_t)a1 * b0 + (uint32_t)t;
  const uint64_t hi = (uint64_t)a1 * b1 + (t >> 32) + (u >> 32);
  const uint32_t w1 = (uint32_t)u, w0 = (uint32_t)p00;
  // A B lies in [2^126, 2^128): hi in [2^62, 2^64); normalise its leading bit to 63
  const uint32_t h1 = (uint32_t)(hi >> 32), h0 = (uint32_t)hi;
  const bool top = (h1 >> 31) != 0;
  const uint32_t n1 = top ? h1 : shl_hi(h0, h1, 1), n0 = top ? h0 : shl_hi(w1, h0, 1);
  const uint32_t low = top ? (w1 | w0) : ((w1 << 1) | w0);  // the bits below the 64 kept
  const int e = ea + eb - 1023 + (top ? 1 : 0);
  // m = n >> 11 (53 bits), rem its 11 guard bits with the sticky bit ORed in
  const uint32_t m1 = n1 >> 11, m0 = shr_lo(n0, n1, 11);
  const uint32_t rem = (n0 & 0x7FFu) | (low != 0 ? 1u : 0u);
  const uint32_t inc = rem + (m0 & 1u) > 0x400u ? 1u : 0u;
  const uint64_t m = ((uint64_t)m1 << 32) | m0;
  const bool na = (unsigned)(ea - 1) < 2046u, nb = (unsigned)(eb - 1) < 2046u;
  const uint64_t sign = ((uint64_t)((ah ^ bh) & 0x80000000u)) << 32;
  bool fast = na && nb && (unsigned)(e - 1) < 2046u;
  double r = double_of(sign | ((((uint64_t)(e - 1)) << 52) + m + inc));
  if constexpr (ZEROS) {
    // a zero operand times a normal one (or zero) gives a zero of the product's sign
    const bool za = ((ah << 1) | al) == 0, zb = ((bh << 1) | bl) == 0;
    const bool zero = (za && (nb || zb)) || (zb && na);
    fast = fast || zero;
    r = zero ? double_of(sign) : r;
  }
  if constexpr (CHECKED) {
    return take_fallback(fast) ? (fast ? r : mul_fallback(a, b)) : r;
  } else {
    return fast ? r : double_of(0x7FF8000000000000ull);  // a quiet NaN where the fast path does not apply
  }
}

}  // namespace emu
}  // namespace olbm
