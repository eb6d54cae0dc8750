// lbm_adjoint.cuh -- transposed Jacobian of one collision (Eq. 1a) for the
// hand-written adjoint of the D2Q9 OReg-GEq step (arXiv 2602.21242).
//
// Every model's post-collision populations are a function of five node
// quantities z = (rho, u_x, u_y, A1, A2) (and, for LBGK, of f itself):
//   f*_(a,b) = P_x(a) P_y(b) [rho + A1 (C_x(a)^2 - C_y(b)^2) + A2 C_x(a) C_y(b)] + omega' Psi_(a,b)
//   (OReg models; omega' Psi depends on A1 and u only), and
//   f*_i = (1 - omega) f_i + omega rho P_x(a) P_y(b)   (LBGK),
// with u = j / rho, A1 = omega'/(4 theta^2) (D - rho (u_x^2 - u_y^2)),
// A2 = omega'/theta^2 (Pi_xy - rho u_x u_y), and (rho, j, D, Pi_xy) linear in f
// (D = sum (c_x^2 - c_y^2) f). Given mu = dL/df*, the reverse sweep forms
// dL/dz, pushes it through A1, A2 and u = j / rho onto the five moments, and
// expands lambda_i = dL/df_i = rho~ + c_ix jx~ + c_iy jy~ + (c_ix^2 - c_iy^2) D~
// + c_ix c_iy Pi~_xy (plus (1 - omega) mu_i for LBGK).
#pragma once

#include "lbm_device.cuh"

namespace olbm {

// v + k x for a lattice coefficient k in {-1, 0, 1} (known after unrolling):
// an add, a subtract or nothing, rather than a product with 0 that IEEE
// arithmetic cannot drop.
template <typename T> __device__ __forceinline__ T signed_add(T v, int k, T x) {
  return k == 0 ? v : (k > 0 ? v + x : v - x);
}

template <int MODEL, bool SHIFT, typename T>
__device__ __forceinline__ void collide_vjp(const T (&f)[9], const T (&mu)[9], const Coef<T>& c, T (&lam)[9]) {
  // ---- forward intermediates, as in collide()
  const T s13 = f[1] + f[3], d13 = f[1] - f[3];
  const T s24 = f[2] + f[4], d24 = f[2] - f[4];
  const T s57 = f[5] + f[7], d57 = f[5] - f[7];
  const T s68 = f[6] + f[8], d68 = f[6] - f[8];
  const T m0 = f[0] + (s13 + s24) + (s57 + s68);
  const T jx = d13 + (d57 - d68);
  const T jy = d24 + (d57 + d68);
  const T rho = SHIFT ? c.rho_ref + m0 : m0;
  const T r = recip(rho);
  const T ux = jx * r, uy = jy * r;
  const T ux2 = ux * ux, uy2 = uy * uy;
  const T hux = scaled(ux, 0.5f), huy = scaled(uy, 0.5f);
  const T px[3] = {c.half_theta + fma(T(0.5), ux2, -hux), c.one_m_theta - ux2, c.half_theta + fma(T(0.5), ux2, hux)};
  const T py[3] = {c.half_theta + fma(T(0.5), uy2, -huy), c.one_m_theta - uy2, c.half_theta + fma(T(0.5), uy2, huy)};
  // dP/du: P(0) = 1 - theta - u^2 -> -2u; P(+-1) = (theta + u^2 +- u)/2 -> u +- 1/2
  const T dpx[3] = {ux - T(0.5), scaled(ux, -2.0f), ux + T(0.5)};
  const T dpy[3] = {uy - T(0.5), scaled(uy, -2.0f), uy + T(0.5)};

  T rb = T(0.0), uxb = T(0.0), uyb = T(0.0);  // adjoints of rho (at fixed u), u_x, u_y
  if constexpr (MODEL == 0) {
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        const T w = mu[pop_index(a, b)];
        rb = fma(w, px[a + 1] * py[b + 1], rb);
        uxb = fma(w, dpx[a + 1] * py[b + 1], uxb);
        uyb = fma(w, px[a + 1] * dpy[b + 1], uyb);
      }
    rb = c.omega * rb;
    uxb = c.omega * rho * uxb;
    uyb = c.omega * rho * uyb;
    const T jxb = uxb * r, jyb = uyb * r;
    rb = rb - (uxb * ux + uyb * uy) * r;
#pragma unroll
    for (int i = 0; i < 9; ++i)
      lam[i] = fma(c.one_m_omega, mu[i], signed_add(signed_add(rb, cx_of(i), jxb), cy_of(i), jyb));
  } else {
    const T Dxy = s13 - s24;
    const T Pxy = s57 - s68;
    const T A1 = c.k1 * fma(-rho, ux2 - uy2, Dxy);
    const T A2 = c.k2 * fma(-jx, uy, Pxy);
    const T cxm[3] = {T(-1.0) - ux, -ux, T(1.0) - ux};
    const T cym[3] = {T(-1.0) - uy, -uy, T(1.0) - uy};
    // Per population (a, b), with S = A1 (C_x^2 - C_y^2) + A2 C_x C_y + rho and
    // Q = P_x(a) P_y(b), the forward value is f* = Q S + omega' Psi. Its pullback
    // sums mu_ab Q (.) over the nine populations; every term is a product of a
    // factor of a and a factor of b, so the sums are taken over b first:
    //   Y_k(a) = sum_b mu_ab P_y(b) C_y(b)^k,  Z_k(a) = sum_b mu_ab P_y'(b) C_y(b)^k,
    // and then over a (dS/du_x = -2 A1 C_x - A2 C_y, dS/du_y = 2 A1 C_y - A2 C_x).
    T py1[3], py2[3], dpy1[3], dpy2[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      py1[b] = py[b] * cym[b];
      py2[b] = py1[b] * cym[b];
      dpy1[b] = dpy[b] * cym[b];
      dpy2[b] = dpy1[b] * cym[b];
    }
    const T twoA1 = scaled(A1, 2.0f);
    T A1b = T(0.0), A2b = T(0.0);
#pragma unroll
    for (int a = -1; a <= 1; ++a) {
      const T w0 = mu[pop_index(a, -1)], w1 = mu[pop_index(a, 0)], w2 = mu[pop_index(a, 1)];
      auto bsum = [&](const T (&v)[3]) { return fma(w0, v[0], fma(w1, v[1], w2 * v[2])); };
      const T Y0 = bsum(py), Y1 = bsum(py1), Y2 = bsum(py2);
      const T Z0 = bsum(dpy), Z1 = bsum(dpy1), Z2 = bsum(dpy2);
      const T cx = cxm[a + 1];
      const T cx2 = a == 0 ? ux2 : cx * cx;
      const T pxa = px[a + 1];
      const T E = fma(A1, cx2, rho);  // A1 C_x^2 + rho
      const T A2cx = A2 * cx;
      rb = fma(pxa, Y0, rb);
      A1b = fma(pxa, fma(cx2, Y0, -Y2), A1b);
      A2b = fma(pxa * cx, Y1, A2b);
      // sum_b mu P_y S = E Y0 - A1 Y2 + A2 C_x Y1
      const T SY = fma(A2cx, Y1, fma(E, Y0, -(A1 * Y2)));
      uxb = fma(dpx[a + 1], SY, uxb);
      uxb = fma(-pxa, fma(twoA1, cx * Y0, A2 * Y1), uxb);
      // sum_b mu (P_y' S + P_y dS/du_y) = E Z0 - A1 Z2 + A2 C_x (Z1 - Y0) + 2 A1 Y1
      const T SZ = fma(A2cx, Z1 - Y0, fma(E, Z0, fma(-A1, Z2, twoA1 * Y1)));
      uyb = fma(pxa, SZ, uyb);
    }
    if constexpr (MODEL == 2) {
      // Psi^P: omega' Psi_1,3 = -+ psi'_x / 2, omega' Psi_2,4 = -+ psi'_y / 2,
      // psi'_x = A1 u_x (c3 - u_x^2), psi'_y = -A1 u_y (c3 - u_y^2)
      const T Mx = scaled(mu[1] - mu[3], -0.5f);
      const T My = scaled(mu[2] - mu[4], -0.5f);
      A1b = A1b + Mx * ux * (c.c3 - ux2) - My * uy * (c.c3 - uy2);
      uxb = fma(Mx * A1, c.c3 - T(3.0) * ux2, uxb);
      uyb = uyb - My * A1 * (c.c3 - T(3.0) * uy2);
    } else if constexpr (MODEL >= 3) {
      // Psi^C through h = omega' pref / 2 (model 3: mq A1 (mu_xx' + mu_yy'); model 4:
      // -A1 / 2), the halved Pi~ terms hPxx = -h Fx, hPyy = h Fy, qPxy = h G / 2 and hps = psi' / 2.
      // 2 theta^2 (mu_xx' + mu_yy') = 2 theta (1 - theta) + u_x^2 (u_x^2 - 1) + u_y^2 (u_y^2 - 1)
      const T e1x = ux2 - T(1.0), e1y = uy2 - T(1.0);
      const T musum = fma(ux2, e1x, fma(uy2, e1y, c.tt2));
      const T h = MODEL == 3 ? c.mq_inv2t2 * A1 * musum : scaled(A1, -0.5f);
      const T Fx = fma(ux2, e1x, c.tt), Fy = fma(uy2, e1y, c.tt);
      const T G = ux * uy * (ux2 - uy2);
      const T Sd = (mu[5] + mu[7]) + (mu[6] + mu[8]);
      const T hPyyb = mu[1] + mu[3] - T(0.5) * Sd;
      const T hPxxb = mu[2] + mu[4] - T(0.5) * Sd;
      const T qPxyb = (mu[6] + mu[8]) - (mu[5] + mu[7]);
      const T wpsxb = scaled(mu[3] - mu[1], 0.5f);
      const T wpsyb = scaled(mu[4] - mu[2], 0.5f);
      // psi'_x = A1 u_x (c3 - u_x^2), psi'_y = -A1 u_y (c3 - u_y^2)
      A1b = A1b + wpsxb * ux * (c.c3 - ux2) - wpsyb * uy * (c.c3 - uy2);
      uxb = fma(wpsxb * A1, c.c3 - T(3.0) * ux2, uxb);
      uyb = uyb - wpsyb * A1 * (c.c3 - T(3.0) * uy2);
      // through Fx, Fy, G at fixed h
      const T dFx = scaled(ux, 2.0f) * fma(T(2.0), ux2, T(-1.0));
      const T dFy = scaled(uy, 2.0f) * fma(T(2.0), uy2, T(-1.0));
      const T dGx = uy * fma(T(3.0), ux2, -uy2);
      const T dGy = ux * fma(T(-3.0), uy2, ux2);
      const T hqb = scaled(qPxyb, 0.5f);
      uxb = fma(h, fma(hqb, dGx, -(hPxxb * dFx)), uxb);
      uyb = fma(h, fma(hqb, dGy, hPyyb * dFy), uyb);
      // through h: model 3, h = mq A1 (mu_xx' + mu_yy') with d mu_aa'/du_a = -2 u_a (1 - 2 u_a^2);
      // model 4, h = -A1 / 2
      const T hb = fma(hqb, G, fma(hPyyb, Fy, -(hPxxb * Fx)));
      if constexpr (MODEL == 3) {
        A1b = fma(hb * c.mq_inv2t2, musum, A1b);
        const T m2hA = scaled(hb * c.mq_inv2t2 * A1, -2.0f);
        uxb = fma(m2hA * ux, fma(T(-2.0), ux2, T(1.0)), uxb);
        uyb = fma(m2hA * uy, fma(T(-2.0), uy2, T(1.0)), uyb);
      } else {
        A1b = fma(T(-0.5), hb, A1b);
      }
    }
    // through A1 = k1 (D - rho (u_x^2 - u_y^2)) and A2 = k2 (Pi_xy - rho u_x u_y)
    const T Db = c.k1 * A1b;
    const T Pb = c.k2 * A2b;
    const T rD2 = scaled(rho * Db, 2.0f), rP = rho * Pb;
    rb = fma(-(ux2 - uy2), Db, fma(-(ux * uy), Pb, rb));
    uxb = fma(-rD2, ux, fma(-rP, uy, uxb));
    uyb = fma(rD2, uy, fma(-rP, ux, uyb));
    // through u = j / rho
    const T jxb = uxb * r, jyb = uyb * r;
    rb = rb - (uxb * ux + uyb * uy) * r;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int cx = cx_of(i), cy = cy_of(i);
      lam[i] = signed_add(signed_add(signed_add(signed_add(rb, cx, jxb), cy, jyb), cx * cx - cy * cy, Db), cx * cy, Pb);
    }
  }
}

}  // namespace olbm
