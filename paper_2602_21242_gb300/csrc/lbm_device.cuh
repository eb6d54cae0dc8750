// lbm_device.cuh -- device-side building blocks of the D2Q9 OReg-GEq step
// (arXiv 2602.21242): storage forms, per-run coefficients, the per-node
// collision of Eq. 1a for the four models, the guided equilibrium of Eq. 10,
// and the fixed-order block reduction used by the diagnostics.
//
// Product form. The guided equilibrium factorises per axis (Eq. 10):
//   f^eq_(a,b) = rho * P_x(a) * P_y(b),  P(0) = 1 - theta - u^2,
//   P(+-1) = (theta + u^2 +- u)/2,        a, b in {-1, 0, 1},
// and, with C = c - u, so does every term of the Onsager-regularised
// non-equilibrium of Eq. 2 (traceless second-moment contraction, D = 2):
//   f^OReg_(a,b) = K1 [Q_x(a) P_y(b) - P_x(a) Q_y(b)] + K2 R_x(a) R_y(b)
// with R(a) = P(a) C(a), Q(a) = P(a) C(a)^2, K1 = N_d / (2 theta^2),
// K2 = N_xy / theta^2, N_d = (Pi^neq_xx - Pi^neq_yy)/2, N_xy = Pi^neq_xy.
// The moments of f^OReg that the corrections need follow in closed form from
// sum_a P = 1, sum_a a P = u, sum_a a^2 P = theta + u^2 (exact identities of
// Eq. 10, not the Chapman-Enskog estimates of Eq. 11a):
//   psi_x = K1 u_x (1 - 3 theta - u_x^2),  psi_y = -K1 u_y (1 - 3 theta - u_y^2)    (Eq. 6a)
//   sum_i (c_ix^2 - c_iy^2) f^OReg_i = 2 theta^2 K1 (mu_xx + mu_yy)
//   => pref = -(K1/2)(mu_xx + mu_yy),  mu_aa = (theta - u_a^2)(1 - theta - u_a^2)/(2 theta^2)  (Eqs. 12, 13b)
// so no population-level moment sums are needed beyond those of f itself.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lbm_fp64emu.cuh"

namespace olbm {

// ---------------------------------------------------------------- storage forms
// PREC 0: FP64 absolute populations. PREC 1: FP32 deviations from the rest
// state rho_ref * W(a) W(b). PREC 2: FP16 deviations, FP32 arithmetic.
template <int PREC> struct Form;
template <> struct Form<0> {
  using S = double;
  using T = double;
  static constexpr bool kShift = false;
};
template <> struct Form<1> {
  using S = float;
  using T = float;
  static constexpr bool kShift = true;
};
template <> struct Form<2> {
  using S = __half;
  using T = float;
  static constexpr bool kShift = true;
};

__device__ __forceinline__ double ld_t(const double* p, double) { return __ldg(p); }
__device__ __forceinline__ float ld_t(const float* p, float) { return __ldg(p); }
__device__ __forceinline__ float ld_t(const __half* p, float) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void st_t(double* p, double v) { *p = v; }
__device__ __forceinline__ void st_t(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_t(__half* p, float v) { *p = __float2half_rn(v); }

__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(__half v) { return (double)__half2float(v); }

template <typename S> __device__ __forceinline__ S from_double(double v);
template <> __device__ __forceinline__ double from_double<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_double<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __half from_double<__half>(double v) {
  return __float2half_rn((float)v);
}

// ---------------------------------------------------------------- packed FP32
// Two nodes' values in one register pair, operated on by Blackwell's packed
// FP32 instructions (add/mul/fma .f32x2, sm_100 and later): one instruction
// per operation for two nodes, each lane rounded exactly as the scalar
// operation. a - b is formed as fma(b, -1, a), exact like a scalar subtraction.
struct f32x2 {
  float2 v;
  f32x2() = default;
  __host__ __device__ f32x2(float s) : v(make_float2(s, s)) {}
  __host__ __device__ f32x2(double s) : v(make_float2((float)s, (float)s)) {}
  __host__ __device__ f32x2(int s) : v(make_float2((float)s, (float)s)) {}
  __host__ __device__ explicit f32x2(float2 a) : v(a) {}
  // Hidden friends: found only by argument-dependent lookup on f32x2, so they
  // never capture a scalar fma(double, ...) call.
  friend __device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b) { return f32x2(__fadd2_rn(a.v, b.v)); }
  friend __device__ __forceinline__ f32x2 operator*(f32x2 a, f32x2 b) { return f32x2(__fmul2_rn(a.v, b.v)); }
  friend __device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b) {
    return f32x2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v));
  }
  friend __device__ __forceinline__ f32x2 operator-(f32x2 a) {
    return f32x2(__fmul2_rn(a.v, make_float2(-1.0f, -1.0f)));
  }
  friend __device__ __forceinline__ f32x2& operator+=(f32x2& a, f32x2 b) { return a = a + b; }
  friend __device__ __forceinline__ f32x2 fma(f32x2 a, f32x2 b, f32x2 c) {
    return f32x2(__ffma2_rn(a.v, b.v, c.v));
  }
};

// ---------------------------------------------------------------- lattice
// Population index of velocity (a, b), a, b in {-1, 0, 1}: IDX[a + 1][b + 1]
// (Fig. 1a numbering: c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1) c5=(1,1) c6=(-1,1)
// c7=(-1,-1) c8=(1,-1)).
__host__ __device__ constexpr int pop_index(int a, int b) {
  return (a == -1) ? (b == -1 ? 7 : (b == 0 ? 3 : 6))
                   : (a == 0 ? (b == -1 ? 4 : (b == 0 ? 0 : 2)) : (b == -1 ? 8 : (b == 0 ? 1 : 5)));
}
__host__ __device__ constexpr int cx_of(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}

// Geometry of one population buffer.
struct Geometry {
  int nx, ny;
  long long pitch;  // elements between rows
  long long plane;  // elements between planes
};

// Per-run coefficients, computed once on the host in FP64 and rounded to T.
template <typename T> struct Coef {
  T theta;        // theta
  T one_m_theta;  // 1 - theta            (P(0) at u = 0)
  T half_theta;   // theta / 2            (P(+-1) at u = 0)
  T omega;        // 1 / tau
  T one_m_omega;  // 1 - 1/tau            (omega')
  T k1;           // omega' / (4 theta^2): omega' K1 = k1 * (D - rho (u_x^2 - u_y^2))
  T k2;           // omega' / theta^2:     omega' K2 = k2 * N_xy
  T c3;           // 1 - 3 theta
  T tt;           // theta (1 - 3 theta)
  T inv2t2;       // 1 / (2 theta^2)
  T mq_inv2t2;    // -1 / (8 theta^2)
  T q_inv2t2;     // 1 / (8 theta^2)
  T ntt;          // -theta (1 - 3 theta)
  T tt2;          // 2 theta (1 - theta)
  T inv_theta;    // 1 / theta                (polynomial equilibrium of model 5)
  T rho_ref;      // reference density of the shifted forms (0 for absolute storage)
  T rw0, rwp;     // rho_ref W(0) and rho_ref W(+-1): the rest state is rho_ref W(a) W(b), W(0) = 1 - theta, W(+-1) = theta/2
  T nrw0, nrwp;   // -rw0, -rwp
};

template <typename T> __host__ Coef<T> make_coef(double theta, double tau, double rho_ref) {
  Coef<T> c;
  const double om = 1.0 / tau, omp = 1.0 - om;
  c.theta = (T)theta;
  c.one_m_theta = (T)(1.0 - theta);
  c.half_theta = (T)(0.5 * theta);
  c.omega = (T)om;
  c.one_m_omega = (T)omp;
  c.k1 = (T)(omp / (4.0 * theta * theta));
  c.k2 = (T)(omp / (theta * theta));
  c.c3 = (T)(1.0 - 3.0 * theta);
  c.tt = (T)(theta * (1.0 - 3.0 * theta));
  c.inv2t2 = (T)(1.0 / (2.0 * theta * theta));
  c.mq_inv2t2 = (T)(-0.25 / (2.0 * theta * theta));
  c.q_inv2t2 = (T)(0.25 / (2.0 * theta * theta));
  c.ntt = (T)(-theta * (1.0 - 3.0 * theta));
  c.tt2 = (T)(2.0 * theta * (1.0 - theta));
  c.inv_theta = (T)(1.0 / theta);
  c.rho_ref = (T)rho_ref;
  c.rw0 = (T)(rho_ref * (1.0 - theta));
  c.rwp = (T)(rho_ref * 0.5 * theta);
  c.nrw0 = (T)(-rho_ref * (1.0 - theta));
  c.nrwp = (T)(-rho_ref * 0.5 * theta);
  return c;
}

// The same coefficients in another arithmetic type (a batch stores FP32
// coefficients per domain and broadcasts them to packed pairs).
template <typename U, typename T> __host__ __device__ Coef<U> coef_cast(const Coef<T>& a) {
  static_assert(sizeof(Coef<float>) == 20 * sizeof(float), "coef_cast lists every field of Coef");
  Coef<U> c;
  c.theta = U(a.theta);
  c.one_m_theta = U(a.one_m_theta);
  c.half_theta = U(a.half_theta);
  c.omega = U(a.omega);
  c.one_m_omega = U(a.one_m_omega);
  c.k1 = U(a.k1);
  c.k2 = U(a.k2);
  c.c3 = U(a.c3);
  c.tt = U(a.tt);
  c.inv2t2 = U(a.inv2t2);
  c.mq_inv2t2 = U(a.mq_inv2t2);
  c.q_inv2t2 = U(a.q_inv2t2);
  c.ntt = U(a.ntt);
  c.tt2 = U(a.tt2);
  c.inv_theta = U(a.inv_theta);
  c.rho_ref = U(a.rho_ref);
  c.rw0 = U(a.rw0);
  c.rwp = U(a.rwp);
  c.nrw0 = U(a.nrw0);
  c.nrwp = U(a.nrwp);
  return c;
}

// Moments of one node kept for the diagnostics.
template <typename T> struct NodeMoments {
  T m0;  // sum of stored values: rho (absolute) or rho - rho_ref (shifted)
  T jx, jy;
  T ux, uy;  // the kinetic energy is (j_x u_x + j_y u_y) / 2
};

// ---------------------------------------------------------------- FP64 helpers off the FP64 pipe
// On GB300 the FP64 pipe runs at 1/64 of the FP32 rate and bounds the FP64
// kernels; these helpers do exact work on the integer pipe instead.

// FP32 -> FP64 by exponent rebias (exact; FP32 subnormals become zero).
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned fe = (u >> 23) & 0xFFu;
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  if (fe == 0) return __longlong_as_double((long long)sign);
  const unsigned long long E = fe == 0xFFu ? 0x7FFull : (unsigned long long)(fe + 896u);
  return __longlong_as_double((long long)(sign | (E << 52) | m));
}

// FP64 -> FP32 by truncating the mantissa to 23 bits: magnitudes below FP32's
// normal range give a signed zero, above it (and infinities, NaNs) infinity.
__device__ __forceinline__ float narrow_trunc(double d) {
  const unsigned h = (unsigned)__double2hiint(d), l = (unsigned)__double2loint(d);
  const unsigned sign = h & 0x80000000u;
  const int fe = (int)((h >> 20) & 0x7FFu) - 896;  // FP32 biased exponent of the same power of two
  const unsigned r = sign | ((unsigned)fe << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29);
  return __uint_as_float(fe <= 0 ? sign : (fe >= 255 ? (sign | 0x7F800000u) : r));
}

// 1 / x. FP64: a single-precision seed (rcp.approx of x truncated to FP32,
// relative error below 2^-21) refined by one cubic Newton step
// r = r0 (1 + e + e^2), e = 1 - x r0, which leaves a relative error
// O(e^3) < 2^-62 before the final rounding: 3 FP64 operations instead of a full
// IEEE division, the conversions on the integer pipe. Valid for
// 2^-126 <= |x| < 2^126 (the seed and its reciprocal FP32 normal numbers);
// every other x gives a non-finite result, which the diagnostics report: x = 0,
// non-finite or smaller x through the Newton step (rcp.approx returns infinity
// for a zero seed, the step then forms 0 * inf or inf - inf), larger x through a
// NaN seed in place of the zero that rcp.approx returns for them (a density
// that large only arises in a simulation that has blown up).
__device__ __forceinline__ float rcp_seed(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double recip(double x) {
  const float s = rcp_seed(narrow_trunc(x));
  const double r0 = widen_f32(__float_as_uint(s) << 1 == 0u ? __uint_as_float(0x7FC00000u) : s);
  const double e = fma(-x, r0, 1.0);
  return fma(r0, fma(e, e, e), r0);
}
// FP32: the same seed and one Newton step r0 + r0 (1 - x r0) (within an ulp or
// two of 1/x; the shifted forms round their stored deviations far more coarsely).
__device__ __forceinline__ float recip(float x) {
  const float r0 = rcp_seed(x);
  return __fmaf_rn(r0, __fmaf_rn(-x, r0, 1.0f), r0);
}
__device__ __forceinline__ f32x2 recip(f32x2 x) {
  const f32x2 r0(make_float2(rcp_seed(x.v.x), rcp_seed(x.v.y)));
  return fma(r0, fma(-x, r0, f32x2(1.0f)), r0);
}

// k x and k x + c for a power of two k (exact scaling); the double-float type
// overloads them with a scaling of both parts, two instructions instead of a
// full product.
template <typename T> __device__ __forceinline__ T scaled(T x, float k) { return T(k) * x; }
template <typename T> __device__ __forceinline__ T fma_scaled(T x, float k, T c) { return fma(T(k), x, c); }
// FP64: the exponent field moves by log2 |k| and the sign flips for k < 0, on
// the integer pipe. Zeros, infinities and NaNs keep their exponent field, so
// they come out as k x does. Normal results only: x and k x must lie in
// FP64's normal range (the callers scale moments of O(1) populations by 1/2
// or 1/4; a normal x below 2^-1020 would not come out as k x).
__device__ __forceinline__ double scaled(double x, float k) {
  const unsigned kb = __float_as_uint(k);
  const int e = (int)((kb >> 23) & 0xFFu) - 127;
  const unsigned h = (unsigned)__double2hiint(x);
  const bool normal = (h & 0x7FF00000u) - 0x00100000u < 0x7FE00000u;
  const unsigned nh = (normal ? h + ((unsigned)e << 20) : h) ^ (kb & 0x80000000u);
  return __hiloint2double((int)nh, __double2loint(x));
}

// ---------------------------------------------------------------- collision
// In-place collision of one node (Eq. 1a). f holds the stored values of the
// pulled pre-collision populations (absolute, or deviations from the rest
// state in the shifted forms); on return it holds the post-collision values
// in the same representation. sink(NodeMoments) receives the node's moments as
// soon as they are known (the diagnostics accumulate them there, so they need
// not stay live through the rest of the collision).
//
// With P(b), C(b) = b - u the per-axis factors, every post-collision
// population of the Onsager-regularised models is written as
//   f*_(a,b) = P_y(b) [E(a) + C_y(b) (G(a) - B(a) C_y(b))] + omega' Psi_(a,b)
// where E(a) = P_x(a) (rho + A1 C_x(a)^2), B(a) = A1 P_x(a), G(a) = A2 P_x(a) C_x(a),
// A1 = omega' K1, A2 = omega' K2: the expansion of
// f^eq + omega' [K1 (Q_x P_y - P_x Q_y) + K2 R_x R_y] at three FMAs per population.
// u = j / rho as j * (1 / rho): the velocities go to the diagnostics before the
// collision ends, so the FP64 form takes these two products with their fallback.
template <typename T> __device__ __forceinline__ T mul_u(T a, T b) { return a * b; }

template <int MODEL, bool SHIFT, typename T, typename Sink>
__device__ __forceinline__ void collide_form(T (&f)[9], const Coef<T>& c, Sink&& sink) {
  // Moments (Sec. 1). The rest state has zero momentum, zero
  // sum (c_x^2 - c_y^2) W and zero sum c_x c_y W, so these sums are the same for
  // absolute and shifted values.
  const T s13 = f[1] + f[3], d13 = f[1] - f[3];
  const T s24 = f[2] + f[4], d24 = f[2] - f[4];
  const T s57 = f[5] + f[7], d57 = f[5] - f[7];
  const T s68 = f[6] + f[8], d68 = f[6] - f[8];
  const T m0 = f[0] + (s13 + s24) + (s57 + s68);
  const T jx = d13 + (d57 - d68);
  const T jy = d24 + (d57 + d68);
  const T rho = SHIFT ? c.rho_ref + m0 : m0;
  const T inv_rho = recip(rho);
  const T ux = mul_u(jx, inv_rho), uy = mul_u(jy, inv_rho);
  {
    NodeMoments<T> mom;
    mom.m0 = m0;
    mom.jx = jx;
    mom.jy = jy;
    mom.ux = ux;
    mom.uy = uy;
    sink(mom);
  }

  const T ux2 = ux * ux, uy2 = uy * uy;
  // Per-axis GEq factors P(a) (Eq. 10), a = -1, 0, +1, and their deviations
  // dP = P - W from the rest values (dP(0) = -u^2, dP(+-1) = (u^2 +- u)/2).
  const T hux = scaled(ux, 0.5f), huy = scaled(uy, 0.5f);
  // Shifted forms need dP exactly (no cancellation against W); the absolute form
  // only needs P, one operation cheaper per axis.
  T dx[3], dy[3], px[3], py[3];
  if constexpr (SHIFT) {
    dx[2] = fma(T(0.5), ux2, hux), dx[1] = -ux2, dx[0] = dx[2] - ux;
    dy[2] = fma(T(0.5), uy2, huy), dy[1] = -uy2, dy[0] = dy[2] - uy;
    px[0] = c.half_theta + dx[0], px[1] = c.one_m_theta - ux2, px[2] = c.half_theta + dx[2];
    py[0] = c.half_theta + dy[0], py[1] = c.one_m_theta - uy2, py[2] = c.half_theta + dy[2];
  } else {
    const T hx = fma_scaled(ux2, 0.5f, c.half_theta), hy = fma_scaled(uy2, 0.5f, c.half_theta);
    px[0] = hx - hux, px[1] = c.one_m_theta - ux2, px[2] = hx + hux;
    py[0] = hy - huy, py[1] = c.one_m_theta - uy2, py[2] = hy + huy;
  }

  if constexpr (MODEL == 5) {
    // LBGK on the polynomial equilibrium (second reading of Sec. 5.1's standard
    // LBGK): f^eq_(a,b) = rho W_a W_b [1 + s + s^2/2 - |u|^2/(2 theta)],
    // s = (a u_x + b u_y)/theta. Shifted forms: f^eq - rho_ref W_a W_b =
    // W_a W_b [m0 + rho (t - 1)], t - 1 = s (1 + s/2) - |u|^2/(2 theta), every
    // term small.
    const T vx = ux * c.inv_theta, vy = uy * c.inv_theta;
    const T q1 = -(ux2 + uy2) * scaled(c.inv_theta, 0.5f);  // -|u|^2/(2 theta)
    const T w[3] = {c.half_theta, c.one_m_theta, c.half_theta};
    const T rw[3] = {rho * w[0], rho * w[1], rho * w[2]};
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        const int i = pop_index(a, b);
        const T sx = a == 0 ? T(0.0) : (a > 0 ? vx : -vx);
        const T s = b == 0 ? sx : (a == 0 ? (b > 0 ? vy : -vy) : (b > 0 ? sx + vy : sx - vy));
        const T t1 = fma(s, fma(T(0.5), s, T(1.0)), q1);  // t - 1
        if constexpr (SHIFT) {
          // f^eq - rest = W_a W_b (m0 + rho t1)
          const T feq = w[b + 1] * fma(rw[a + 1], t1, m0 * w[a + 1]);
          f[i] = fma(c.omega, feq - f[i], f[i]);
        } else {
          const T feq = w[b + 1] * fma(rw[a + 1], t1, rw[a + 1]);
          f[i] = fma(c.omega, feq - f[i], f[i]);
        }
      }
  } else if constexpr (MODEL == 0) {
    // LBGK: f* = f + (f^eq - f)/tau = (1 - 1/tau) f + (1/tau) f^eq.
    if constexpr (!SHIFT) {
      const T orho = c.omega * rho;
      const T e[3] = {orho * px[0], orho * px[1], orho * px[2]};
#pragma unroll
      for (int a = -1; a <= 1; ++a)
#pragma unroll
        for (int b = -1; b <= 1; ++b) {
          const int i = pop_index(a, b);
          f[i] = fma(e[a + 1], py[b + 1], c.one_m_omega * f[i]);
        }
    } else {
      // Shifted: with P = W + dP and rho = rho_ref + m0,
      //   f^eq - rho_ref W_a W_b = P_y(b) (rho dP_x(a) + m0 W_a) + rho_ref W_a dP_y(b),
      // every term small, so no O(1) terms cancel.
      const T m0w0 = m0 * c.one_m_theta, m0wp = m0 * c.half_theta;
      const T ex[3] = {fma(rho, dx[0], m0wp), fma(rho, dx[1], m0w0), fma(rho, dx[2], m0wp)};
      const T rdy0[3] = {c.rw0 * dy[0], c.rw0 * dy[1], c.rw0 * dy[2]};
      const T rdyp[3] = {c.rwp * dy[0], c.rwp * dy[1], c.rwp * dy[2]};
#pragma unroll
      for (int a = -1; a <= 1; ++a)
#pragma unroll
        for (int b = -1; b <= 1; ++b) {
          const int i = pop_index(a, b);
          const T feq = fma(ex[a + 1], py[b + 1], a == 0 ? rdy0[b + 1] : rdyp[b + 1]);
          f[i] = fma(c.omega, feq - f[i], f[i]);
        }
    }
  } else {
    // Onsager-regularised models (Eq. 2) with corrections (Eqs. 14, 15).
    // Non-equilibrium stress (Eq. 4 gives Pi^eq = rho (u u + theta I) exactly):
    //   2 N_d = sum (c_x^2 - c_y^2) f - rho (u_x^2 - u_y^2),  N_xy = sum c_x c_y f - rho u_x u_y.
    // (rho u_x u_y = j_x u_y.) FP64 instructions negate operands for free; the
    // packed FP32 instructions have no negated operands, so the products below
    // are arranged with -C_x(a) = u_x - a and -K2, whose signs cancel exactly.
    const T Dxy = s13 - s24;
    const T nPxy = s68 - s57;                                // -sum c_x c_y f
    const T ncx[3] = {ux + T(1.0), ux, ux - T(1.0)};         // -C_x(a)
    const T cym[3] = {T(-1.0) - uy, -uy, T(1.0) - uy};       // C_y(b) = b - u_y
    constexpr bool kNegFree = !std::is_same<T, f32x2>::value;  // scalar and double-float negations are free
    const T dyx2 = uy2 - ux2;
    const T A1 = c.k1 * fma(rho, dyx2, Dxy);    // omega' K1
    const T nA2 = c.k2 * fma(jx, uy, nPxy);     // -omega' K2
    // omega' Psi per population (Eqs. 14, 15), from closed-form psi and Pi~.
    T cor[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) cor[i] = T(0.0);
    if constexpr (MODEL >= 2) {
      const T wpsx = A1 * ux * (c.c3 - ux2);   // omega' psi_x
      const T wpsy = A1 * uy * (uy2 - c.c3);   // omega' psi_y
      if constexpr (MODEL == 2) {
        // Psi^P: -1/2 c_ia psi_a on the axis populations.
        cor[1] = scaled(wpsx, -0.5f);
        cor[3] = scaled(wpsx, 0.5f);
        cor[2] = scaled(wpsy, -0.5f);
        cor[4] = scaled(wpsy, 0.5f);
      } else {
        // Psi^C with Pi~ of Eq. 11b and pref of Eq. 12, evaluated on f^OReg (model 3):
        // pref = -(K1/2)(mu_xx + mu_yy); or on f^neq (model 4): pref = -K1.
        const T e1x = ux2 - T(1.0), e1y = uy2 - T(1.0);
        T nhw;  // -omega' pref / 2
        if constexpr (MODEL == 3) {
          // 2 theta^2 (mu_xx + mu_yy) = (theta - u_x^2) P_x(0) + (theta - u_y^2) P_y(0)
          //   = 2 theta (1 - theta) + u_x^2 (u_x^2 - 1) + u_y^2 (u_y^2 - 1)
          nhw = c.q_inv2t2 * A1 * fma(ux2, e1x, fma(uy2, e1y, c.tt2));
        } else {
          nhw = scaled(A1, 0.5f);
        }
        const T hPxx = nhw * fma(ux2, e1x, c.tt);  // omega' Pi~_xx / 2
        const T hPyy = nhw * (kNegFree ? fma(-uy2, e1y, c.ntt) : fma(uy2, T(1.0) - uy2, c.ntt));  // omega' Pi~_yy / 2
        const T qPxy = scaled(nhw, 0.5f) * (ux * uy) * dyx2;             // omega' Pi~_xy / 4
        const T hpsx = scaled(wpsx, 0.5f), hpsy = scaled(wpsy, 0.5f);
        cor[1] = hPyy - hpsx;
        cor[3] = hPyy + hpsx;
        cor[2] = hPxx - hpsy;
        cor[4] = hPxx + hpsy;
        const T dsum = scaled(hPxx + hPyy, -0.5f);
        cor[5] = dsum - qPxy;  // c_x c_y = +1
        cor[7] = dsum - qPxy;
        cor[6] = dsum + qPxy;  // c_x c_y = -1
        cor[8] = dsum + qPxy;
      }
    }
    // Shifted forms: f^eq - rho_ref W_a W_b = P_y(b) (rho dP_x(a) + m0 W_a) + rho_ref W_a dP_y(b)
    // (P = W + dP, rho = rho_ref + m0); the first part joins E(a), the second is added per population.
    T E[3], B[3], G[3];
    T m0w0, m0wp;
    if constexpr (SHIFT) m0w0 = m0 * c.one_m_theta, m0wp = m0 * c.half_theta;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      B[k] = A1 * px[k];
      G[k] = nA2 * (px[k] * ncx[k]);
      if (SHIFT && k == 1) {
        E[k] = fma(ux2, B[k] - rho, m0w0);  // m0 W(0) - rho u_x^2 + B(0) C_x(0)^2
      } else {
        // f^eq part carried by P_y(b)
        const T base = SHIFT ? fma(rho, dx[k], m0wp) : rho * px[k];
        E[k] = fma(B[k], k == 1 ? ux2 : ncx[k] * ncx[k], base);  // C_x(0)^2 = u_x^2
      }
    }
    // G(a) - B(a) C_y(b): the packed forms take B(a) (-C_y(b)) instead of a negated B(a).
    const T ncy[3] = {uy + T(1.0), uy, uy - T(1.0)};  // -C_y(b)
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        const int i = pop_index(a, b);
        T rest = cor[i];
        // rho_ref W_a dP_y(b), dP_y(0) = -u_y^2
        if constexpr (SHIFT)
          rest = b == 0 ? fma(a == 0 ? c.nrw0 : c.nrwp, uy2, rest) : fma(a == 0 ? c.rw0 : c.rwp, dy[b + 1], rest);
        const T inner = kNegFree ? fma(-B[a + 1], cym[b + 1], G[a + 1]) : fma(B[a + 1], ncy[b + 1], G[a + 1]);
        f[i] = fma(py[b + 1], fma(cym[b + 1], inner, E[a + 1]), rest);
      }
  }
}

// FP64 values whose products run on the integer pipes (emu::mul64, bit-identical
// to the FP64 instruction); sums and FMAs stay on the FP64 pipe. The FP64
// collision runs on this type, so the FP64 pipe, which bounds the FP64 form on
// GB300, carries only the sums and FMAs, while the products overlap with them on
// the otherwise idle integer pipes (complete model at 4096^2, diagnostics every
// step: 4.78 -> 6.33 GLUPS). The products leave out their fallback (a product
// outside the fast path is a quiet NaN), and collide() checks the node's nine
// results once instead: a branch per product measured 6 % slower. Sums on the
// integer pipes as well (emu::add64) measured slower wherever they were put: the
// moments, which head the collision's dependency chain, 4.9; the corrections,
// the factors P or C, or the diagnostics sums, 5.2 to 5.6 (against 5.76).
#ifndef OLBM_F64_EMU_MUL
#define OLBM_F64_EMU_MUL 1
#endif
// How an FP64 wrapper type below forms its products.
enum class Mul64 {
  kIntUnchecked,  // integer pipes, a quiet NaN outside the fast path (the caller checks its results)
  kIntZeros,      // the same with zero operands on the fast path
  kIntChecked,    // integer pipes, the FP64 instruction behind a warp-uniform branch outside the fast path
  kFp64           // the FP64 instruction (__dmul_rn, never contracted into an FMA)
};
template <Mul64 M> struct d64 {
  double v;
  d64() = default;
  __host__ __device__ constexpr d64(double x) : v(x) {}
  // Hidden friends: found only by argument-dependent lookup on d64, so they
  // never capture a call on plain doubles.
  friend __device__ __forceinline__ d64 operator+(d64 a, d64 b) { return d64(a.v + b.v); }
  friend __device__ __forceinline__ d64 operator-(d64 a, d64 b) { return d64(a.v - b.v); }
  friend __device__ __forceinline__ d64 operator-(d64 a) { return d64(-a.v); }
  friend __device__ __forceinline__ d64 operator*(d64 a, d64 b) {
    if constexpr (M == Mul64::kFp64) return d64(__dmul_rn(a.v, b.v));
    else return d64(emu::mul64<M == Mul64::kIntChecked, M == Mul64::kIntZeros>(a.v, b.v));
  }
  // u = j / rho: checked in every integer form (the velocities reach the diagnostics early)
  friend __device__ __forceinline__ d64 mul_u(d64 a, d64 b) {
    if constexpr (M == Mul64::kFp64) return d64(__dmul_rn(a.v, b.v));
    else return d64(emu::mul64<true>(a.v, b.v));
  }
  friend __device__ __forceinline__ d64 fma(d64 a, d64 b, d64 c) { return d64(::fma(a.v, b.v, c.v)); }
  friend __device__ __forceinline__ d64 recip(d64 x) { return d64(recip(x.v)); }
  friend __device__ __forceinline__ d64 scaled(d64 x, float k) { return d64(scaled(x.v, k)); }
};
// The FP64 collision's type; the one its warps switch to after zero operands sent
// a node to a redo; the adjoint step's (every product checked on its own: it
// cannot switch a warp, see adj_step_body); and the type a node whose integer
// products left the fast path is redone on, which gives the integer products'
// bits where they applied and the FP64 instruction's elsewhere.
using d64m = d64<Mul64::kIntUnchecked>;
using d64z = d64<Mul64::kIntZeros>;
using d64c = d64<Mul64::kIntChecked>;
using d64f = d64<Mul64::kFp64>;

// Bit 31 set iff x is infinite or NaN (its exponent field all ones).
__device__ __forceinline__ unsigned nonfinite_bit(double x) {
  return (((unsigned)__double2hiint(x)) & 0x7FF00000u) + 0x00100000u;
}

// No way to fetch a node's populations again: collide() keeps its own copy.
struct KeepInputs {
  __device__ void operator()(double (&)[9]) const {}
};

// In-place collision of one node (see collide_form); the FP64 form takes its
// products on the integer pipes. Its results are checked once: a node with a
// non-finite result (a product outside the integer fast path, such as a zero
// velocity, or non-finite data) is collided again with its products on the FP64
// pipe, which gives the integer products' bits where they applied and the FP64
// instruction's elsewhere; the redo is a warp-uniform branch. refetch(f) loads
// the node's pulled populations again for the redo (callers that can: no copy of
// them stays live through the collision); with KeepInputs collide() keeps a copy.
// mode (optional, per thread, the same in every thread of a warp) steps up each
// time the warp needs a redo: 0 the integer products, 1 the integer products
// with zero operands on the fast path (zeros come in regions: a flow at rest, a
// velocity component that vanishes everywhere), 2 the FP64 products.
template <int MODEL, bool SHIFT, typename T, typename Sink, typename Refetch = KeepInputs>
__device__ __forceinline__ void collide(T (&f)[9], const Coef<T>& c, Sink&& sink, Refetch&& refetch = Refetch(),
                                        int* mode = nullptr) {
  if constexpr (std::is_same<T, double>::value && OLBM_F64_EMU_MUL) {
    constexpr bool kKeep = std::is_same<std::decay_t<Refetch>, KeepInputs>::value;
    auto to_double = [&](const auto& m) {
      NodeMoments<double> md;
      md.m0 = m.m0.v, md.jx = m.jx.v, md.jy = m.jy.v, md.ux = m.ux.v, md.uy = m.uy.v;
      return md;
    };
    const int md = mode != nullptr ? *mode : 0;
    if (md >= 2) {
      d64f h[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) h[i] = d64f(f[i]);
      collide_form<MODEL, SHIFT, d64f>(h, coef_cast<d64f>(c),
                                       [&](const NodeMoments<d64f>& m) { sink(to_double(m)); });
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = h[i].v;
      return;
    }
    double g[9];
    if (md == 0) {
      d64m e[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) e[i] = d64m(f[i]);
      collide_form<MODEL, SHIFT, d64m>(e, coef_cast<d64m>(c),
                                       [&](const NodeMoments<d64m>& m) { sink(to_double(m)); });
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = e[i].v;
    } else {
      d64z e[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) e[i] = d64z(f[i]);
      collide_form<MODEL, SHIFT, d64z>(e, coef_cast<d64z>(c),
                                       [&](const NodeMoments<d64z>& m) { sink(to_double(m)); });
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = e[i].v;
    }
    unsigned bad = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) bad |= nonfinite_bit(g[i]);
    if (__any_sync(__activemask(), (int)bad < 0)) {
      if (mode != nullptr) *mode = md + 1;
      if ((int)bad < 0) {
        if constexpr (!kKeep) refetch(f);
        d64f h[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = d64f(f[i]);
        collide_form<MODEL, SHIFT, d64f>(h, coef_cast<d64f>(c), [](const NodeMoments<d64f>&) {});
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = h[i].v;
      }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = g[i];
  } else {
    collide_form<MODEL, SHIFT, T>(f, c, sink);
  }
}

// Per-axis factor of the guided equilibrium (Eq. 10) in FP64, for velocity
// component a in {-1, 0, 1}: 1 - theta - u^2, or (theta + u^2 + a u) / 2; the
// equilibrium is rho P(c_ix; u_x) P(c_iy; u_y). Used by lbm_init.
__device__ __forceinline__ double geq_factor(int a, double u, double theta) {
  return a == 0 ? 1.0 - theta - u * u : 0.5 * (theta + u * u + (a > 0 ? u : -u));
}

// Rest-state value of population i for the shifted forms: rho_ref W(c_ix) W(c_iy).
__device__ __forceinline__ double rest_value(int i, double theta, double rho_ref) {
  const double wx = cx_of(i) == 0 ? 1.0 - theta : 0.5 * theta;
  const double wy = cy_of(i) == 0 ? 1.0 - theta : 0.5 * theta;
  return rho_ref * wx * wy;
}

// ---------------------------------------------------------------- reductions
// Sum NV doubles over a block of NT threads in a fixed order: xor-butterfly in
// each warp, then warp totals in warp order by thread 0. The result is valid in
// thread 0 only. Deterministic for a fixed block shape.
template <int NV, int NT>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (&out)[NV]) {
  static_assert(NT % 32 == 0, "block size must be a multiple of 32");
  constexpr int NW = NT / 32;
  __shared__ double red[NW][NV];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  if ((tid & 31) == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[tid >> 5][k] = v[k];
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) s += red[w][k];
      out[k] = s;
    }
  }
}

}  // namespace olbm
