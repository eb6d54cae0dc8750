// lbm_adjoint.cu -- lbm_vjp: reverse-mode derivative of n LBE steps
// (arXiv 2602.21242, Eq. 1) started from the guided equilibrium (Eq. 10).
//
// Forward map: f(0) = f^eq(rho0, u0); f(t + 1) = S C f(t) (C: collision at every
// node, S: streaming); outputs (rho, u)(x, n) = moments of f(n). Reverse:
//   lambda(n)_i  = g_rho + (c_ix - u_x) g_ux / rho + (c_iy - u_y) g_uy / rho
//   lambda(t)(x) = J_C(f(x, t))^T mu(x),  mu_i(x) = lambda_i(t + 1)(x + c_i)   (S^T: a push-read)
//   g_rho0 = sum_i lambda_i(0) df^eq_i/drho0, g_u0 likewise.
// States are recomputed in segments of K steps from checkpoints taken every K
// steps (memory: ceil(n/K) checkpoints + K recomputed states + 2 adjoint fields).
#include <algorithm>
#include <cstdio>

#include "lbm.h"
#include "lbm_adjoint.cuh"
#include "lbm_ctx.h"
#include "lbm_kernels.cuh"
#include "lbm_walls.h"

namespace olbm {

constexpr int kABX = 32, kABY = 8;

// lambda(n) from the cotangents of the final moments (any may be NULL = 0).
template <int PREC>
__global__ void __launch_bounds__(kABX* kABY) adj_seed_kernel(const typename Form<PREC>::S* __restrict__ fbuf,
                                                              Geometry g, double rho_ref,
                                                              const double* __restrict__ g_rho,
                                                              const double* __restrict__ g_ux,
                                                              const double* __restrict__ g_uy,
                                                              typename Form<PREC>::T* __restrict__ lam) {
  using T = typename Form<PREC>::T;
  const int x = blockIdx.x * kABX + threadIdx.x, y = blockIdx.y * kABY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  long long o[9];
  pull_offsets(x, y, g, o);
  double m0 = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double v = to_double(fbuf[i * g.plane + o[i]]);
    m0 += v;
    jx += (double)cx_of(i) * v;
    jy += (double)cy_of(i) * v;
  }
  const double rho = rho_ref + m0, ux = jx / rho, uy = jy / rho;
  const long long n = (long long)y * g.nx + x;
  const double gr = g_rho ? g_rho[n] : 0.0, gx = g_ux ? g_ux[n] / rho : 0.0, gy = g_uy ? g_uy[n] / rho : 0.0;
  const long long here = (long long)y * g.pitch + x;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    lam[i * g.plane + here] = (T)(gr + ((double)cx_of(i) - ux) * gx + ((double)cy_of(i) - uy) * gy);
}

// lambda(t)(x) = J_C(f(x, t))^T mu(x), mu_i(x) = lambda_i(t + 1)(x + c_i).
template <int MODEL, int PREC>
__device__ __forceinline__ void adj_step_body(const typename Form<PREC>::S* __restrict__ fbuf,
                                              const typename Form<PREC>::T* __restrict__ lam_next,
                                              typename Form<PREC>::T* __restrict__ lam, const Geometry& g,
                                              const Coef<typename Form<PREC>::T>& c) {
  using T = typename Form<PREC>::T;
  const int x = blockIdx.x * kABX + threadIdx.x, y = blockIdx.y * kABY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  // f pulled at (x, y); mu_i = lambda_i(t + 1) at x + c_i, periodic
  auto load = [&](T (&f)[9], T (&mu)[9]) {
    long long o[9];
    pull_offsets(x, y, g, o);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = ld_t(fbuf + i * g.plane + o[i], T());
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      int xd = x + cx_of(i), yd = y + cy_of(i);
      xd = xd < 0 ? xd + g.nx : (xd >= g.nx ? xd - g.nx : xd);
      yd = yd < 0 ? yd + g.ny : (yd >= g.ny ? yd - g.ny : yd);
      mu[i] = lam_next[i * g.plane + (long long)yd * g.pitch + xd];
    }
  };
  T f[9], mu[9], out[9];
  load(f, mu);
  if constexpr (std::is_same<T, double>::value && OLBM_F64_EMU_MUL) {
    // FP64: the products on the integer pipes, each with its own fallback to the
    // FP64 instruction. (Without the fallbacks, checking the nine results once and
    // redoing a node measured 1.4 % faster on the 1024^2 gradient, but a field that
    // is zero over a region would redo every node there: one node a thread gives
    // no later rows to switch to FP64 products for.)
    d64c fe[9], me[9], oe[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fe[i] = d64c(f[i]), me[i] = d64c(mu[i]);
    collide_vjp<MODEL, Form<PREC>::kShift, d64c>(fe, me, coef_cast<d64c>(c), oe);
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i] = oe[i].v;
  } else {
    collide_vjp<MODEL, Form<PREC>::kShift, T>(f, mu, c, out);
  }
  const long long here = (long long)y * g.pitch + x;
#pragma unroll
  for (int i = 0; i < 9; ++i) lam[i * g.plane + here] = out[i];
}

template <int MODEL, int PREC>
__global__ void __launch_bounds__(kABX* kABY) adj_step_kernel(const typename Form<PREC>::S* __restrict__ fbuf,
                                                              const typename Form<PREC>::T* __restrict__ lam_next,
                                                              typename Form<PREC>::T* __restrict__ lam, Geometry g,
                                                              Coef<typename Form<PREC>::T> c) {
  adj_step_body<MODEL, PREC>(fbuf, lam_next, lam, g, c);
}

// The FP64 form, compiled for two blocks a SM (118 registers; with one it takes
// 174 and the 1024^2 FP64 gradient's backward pass took 320 ms instead of 292).
#ifndef OLBM_ADJ_F64_MINB
#define OLBM_ADJ_F64_MINB 2
#endif
template <int MODEL>
__global__ void __launch_bounds__(kABX* kABY, OLBM_ADJ_F64_MINB) adj_step_f64_kernel(const double* __restrict__ fbuf,
                                                                                     const double* __restrict__ lam_next,
                                                                                     double* __restrict__ lam, Geometry g,
                                                                                     Coef<double> c) {
  adj_step_body<MODEL, 0>(fbuf, lam_next, lam, g, c);
}

// The FP32 form on node pairs (x, x + 1), x even, with packed f32x2 arithmetic
// (nx even): f pulled as the forward pair kernels pull it, mu push-read as pairs
// (the c_ix = 0 planes aligned, the others element by element), lambda stored
// as aligned pairs.
// Three blocks a SM (80 registers): the 1024^2 FP32 gradient's backward pass
// 18.99 -> 18.04 ms (four blocks spill: 23.35 ms).
#ifndef OLBM_ADJ_PAIR_MINB
#define OLBM_ADJ_PAIR_MINB 3
#endif
template <int MODEL>
__global__ void __launch_bounds__(kABX* kABY, OLBM_ADJ_PAIR_MINB) adj_step_pair_kernel(const float* __restrict__ fbuf,
                                                                   const float* __restrict__ lam_next,
                                                                   float* __restrict__ lam, Geometry g,
                                                                   Coef<f32x2> c) {
  const int x = 2 * (blockIdx.x * kABX + threadIdx.x), y = blockIdx.y * kABY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int xm = x == 0 ? g.nx - 1 : x - 1;           // x - 1, periodic
  const int xp = x + 2 >= g.nx ? x + 2 - g.nx : x + 2;  // x + 2, periodic
  f32x2 f[9], mu[9], out[9];
  Column<MODEL, 1, false, true>::pull(fbuf, g, x, xm, xp, y, f);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    int yd = y + cy_of(i);  // y + c_iy, periodic
    yd = yd < 0 ? yd + g.ny : (yd >= g.ny ? yd - g.ny : yd);
    const float* q = lam_next + i * g.plane + (long long)yd * g.pitch;
    mu[i] = cx_of(i) == 0 ? ld_pair(q + x) : (cx_of(i) > 0 ? ld_two(q + x + 1, q + xp) : ld_two(q + xm, q + x));
  }
  collide_vjp<MODEL, true, f32x2>(f, mu, c, out);
  float* o = lam + (long long)y * g.pitch + x;
#pragma unroll
  for (int i = 0; i < 9; ++i) st_pair(o + i * g.plane, out[i]);
}

// Cotangents of (rho0, u0) from lambda(0), through f(x, 0) = f^eq(rho0(x), u0(x)).
template <int PREC>
__global__ void __launch_bounds__(kABX* kABY) adj_final_kernel(const typename Form<PREC>::T* __restrict__ lam,
                                                               Geometry g, double theta,
                                                               const double* __restrict__ rho0,
                                                               const double* __restrict__ ux0,
                                                               const double* __restrict__ uy0,
                                                               double* __restrict__ g_rho0,
                                                               double* __restrict__ g_ux0,
                                                               double* __restrict__ g_uy0) {
  const int x = blockIdx.x * kABX + threadIdx.x, y = blockIdx.y * kABY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long long n = (long long)y * g.nx + x, here = (long long)y * g.pitch + x;
  const double rho = rho0[n], ux = ux0[n], uy = uy0[n];
  const double px[3] = {0.5 * (theta + ux * ux - ux), 1.0 - theta - ux * ux, 0.5 * (theta + ux * ux + ux)};
  const double py[3] = {0.5 * (theta + uy * uy - uy), 1.0 - theta - uy * uy, 0.5 * (theta + uy * uy + uy)};
  const double dpx[3] = {ux - 0.5, -2.0 * ux, ux + 0.5};
  const double dpy[3] = {uy - 0.5, -2.0 * uy, uy + 0.5};
  double gr = 0.0, gx = 0.0, gy = 0.0;
#pragma unroll
  for (int a = -1; a <= 1; ++a)
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
      const double l = to_double(lam[pop_index(a, b) * g.plane + here]);
      gr += l * px[a + 1] * py[b + 1];
      gx += l * dpx[a + 1] * py[b + 1];
      gy += l * px[a + 1] * dpy[b + 1];
    }
  if (g_rho0) g_rho0[n] = gr;
  if (g_ux0) g_ux0[n] = rho * gx;
  if (g_uy0) g_uy0[n] = rho * gy;
}

inline dim3 adj_grid(const Geometry& g) { return dim3((g.nx + kABX - 1) / kABX, (g.ny + kABY - 1) / kABY); }

template <int PREC> struct Adjoint {
  using S = typename Form<PREC>::S;
  using T = typename Form<PREC>::T;

  static cudaError_t seed(const void* fbuf, const Geometry& g, double rho_ref, const double* gr, const double* gx,
                          const double* gy, void* lam, cudaStream_t st) {
    adj_seed_kernel<PREC><<<adj_grid(g), dim3(kABX, kABY), 0, st>>>((const S*)fbuf, g, rho_ref, gr, gx, gy, (T*)lam);
    return cudaGetLastError();
  }

  template <int MODEL>
  static cudaError_t step_m(const void* fbuf, const void* lam_next, void* lam, const Geometry& g, const Coef<T>& c,
                            double theta, double tau, double rho_ref, cudaStream_t st) {
    if constexpr (PREC == 1) {
      if (g.nx % 2 == 0) {
        const dim3 grid((g.nx / 2 + kABX - 1) / kABX, (g.ny + kABY - 1) / kABY);
        adj_step_pair_kernel<MODEL><<<grid, dim3(kABX, kABY), 0, st>>>(
            (const float*)fbuf, (const float*)lam_next, (float*)lam, g, make_coef<f32x2>(theta, tau, rho_ref));
        return cudaGetLastError();
      }
    }
    if constexpr (PREC == 0) {
      adj_step_f64_kernel<MODEL><<<adj_grid(g), dim3(kABX, kABY), 0, st>>>((const double*)fbuf,
                                                                          (const double*)lam_next, (double*)lam, g, c);
    } else {
      adj_step_kernel<MODEL, PREC><<<adj_grid(g), dim3(kABX, kABY), 0, st>>>((const S*)fbuf, (const T*)lam_next,
                                                                            (T*)lam, g, c);
    }
    return cudaGetLastError();
  }

  static cudaError_t step(int model, const void* fbuf, const void* lam_next, void* lam, const Geometry& g,
                          double theta, double tau, double rho_ref, cudaStream_t st) {
    const Coef<T> c = make_coef<T>(theta, tau, rho_ref);
    switch (model) {
      case 0: return step_m<0>(fbuf, lam_next, lam, g, c, theta, tau, rho_ref, st);
      case 1: return step_m<1>(fbuf, lam_next, lam, g, c, theta, tau, rho_ref, st);
      case 2: return step_m<2>(fbuf, lam_next, lam, g, c, theta, tau, rho_ref, st);
      case 3: return step_m<3>(fbuf, lam_next, lam, g, c, theta, tau, rho_ref, st);
      default: return step_m<4>(fbuf, lam_next, lam, g, c, theta, tau, rho_ref, st);
    }
  }

  static cudaError_t final_(const void* lam, const Geometry& g, double theta, const double* r0, const double* u0,
                            const double* v0, double* gr, double* gx, double* gy, cudaStream_t st) {
    adj_final_kernel<PREC><<<adj_grid(g), dim3(kABX, kABY), 0, st>>>((const T*)lam, g, theta, r0, u0, v0, gr, gx,
                                                                     gy);
    return cudaGetLastError();
  }
};

}  // namespace olbm

namespace {

int vfail(lbm_ctx* c, int status, const char* msg, cudaError_t e = cudaSuccess) {
  if (e != cudaSuccess)
    snprintf(c->err, sizeof(c->err), "%s: %s", msg, cudaGetErrorString(e));
  else
    snprintf(c->err, sizeof(c->err), "%s", msg);
  return status;
}

int elem_bytes(const lbm_ctx* c) { return c->prec == LBM_F32_SHIFT ? 4 : 8; }

cudaError_t adj_seed(lbm_ctx* c, const double* gr, const double* gx, const double* gy, void* lam) {
  switch (c->prec) {
    case LBM_F64: return olbm::Adjoint<0>::seed(c->buf[c->cur], c->g, c->rho_ref, gr, gx, gy, lam, c->stream);
    case LBM_F64_DF: return olbm::Adjoint<3>::seed(c->buf[c->cur], c->g, c->rho_ref, gr, gx, gy, lam, c->stream);
    default: return olbm::Adjoint<1>::seed(c->buf[c->cur], c->g, c->rho_ref, gr, gx, gy, lam, c->stream);
  }
}

cudaError_t adj_step(lbm_ctx* c, const void* fbuf, const void* lam_next, void* lam) {
  switch (c->prec) {
    case LBM_F64: return olbm::Adjoint<0>::step(c->model, fbuf, lam_next, lam, c->g, c->theta, c->tau, c->rho_ref, c->stream);
    case LBM_F64_DF: return olbm::Adjoint<3>::step(c->model, fbuf, lam_next, lam, c->g, c->theta, c->tau, c->rho_ref, c->stream);
    default: return olbm::Adjoint<1>::step(c->model, fbuf, lam_next, lam, c->g, c->theta, c->tau, c->rho_ref, c->stream);
  }
}

cudaError_t adj_final(lbm_ctx* c, const void* lam, const double* r0, const double* u0, const double* v0, double* gr,
                      double* gx, double* gy) {
  switch (c->prec) {
    case LBM_F64: return olbm::Adjoint<0>::final_(lam, c->g, c->theta, r0, u0, v0, gr, gx, gy, c->stream);
    case LBM_F64_DF: return olbm::Adjoint<3>::final_(lam, c->g, c->theta, r0, u0, v0, gr, gx, gy, c->stream);
    default: return olbm::Adjoint<1>::final_(lam, c->g, c->theta, r0, u0, v0, gr, gx, gy, c->stream);
  }
}

cudaError_t fwd_step(lbm_ctx* c, const void* src, void* dst) {
  olbm::StepArgs a;
  a.model = c->model;
  a.diag = false;
  a.src = src;
  a.dst = dst;
  a.g = c->g;
  a.theta = c->theta;
  a.tau = c->tau;
  a.rho_ref = c->rho_ref;
  a.partials = c->d_parts[0];
  a.cfg = c->cfg;
  a.err = c->d_err;
  a.sched = c->d_sched;
  cudaError_t e = c->prec == LBM_F64      ? olbm::launch_step_f64(a, c->stream)
                  : c->prec == LBM_F64_DF ? olbm::launch_step_f64df(a, c->stream)
                                          : olbm::launch_step_f32(a, c->stream);
  if (e == cudaSuccess && c->n_walls > 0)
    e = olbm::launch_walls(elem_bytes(c), src, dst, c->g, c->d_walls, c->n_walls, c->stream);
  return e;
}

}  // namespace

namespace {

// Work memory of lbm_vjp for n steps in segments of K: ceil(n / K) checkpoints,
// a ring of K recomputed states, two adjoint fields.
struct VjpLayout {
  int K = 1, nseg = 0;
  size_t sb = 0;
  char* base = nullptr;
  void* ckpt(int s) const { return base + sb * (size_t)s; }
  void* ring(int j) const { return base + sb * ((size_t)nseg + (size_t)j); }
  void* lam(int k) const { return base + sb * ((size_t)nseg + (size_t)K + (size_t)k); }
};

// Two forward steps src -> dst in one launch (launch kind 2 of the shifted forms;
// bit-identical to two single steps), where the lattice's launch allows it.
bool two_steps_apply(const lbm_ctx* c) {
  return c->n_walls == 0 && c->prec == LBM_F32_SHIFT && olbm::uses_step2(c->prec, c->g, c->cfg);
}

cudaError_t fwd_step2(lbm_ctx* c, const void* src, void* dst) {
  olbm::StepArgs a;
  a.model = c->model;
  a.diag = false;
  a.diag2 = false;
  a.src = src;
  a.dst = dst;
  a.g = c->g;
  a.theta = c->theta;
  a.tau = c->tau;
  a.rho_ref = c->rho_ref;
  a.partials = c->d_parts[0];
  a.partials2 = c->d_parts[0];
  a.cfg = c->cfg;
  a.err = c->d_err;
  a.sched = c->d_sched;
  return olbm::launch_step2_f32(a, c->stream);
}

int vjp_layout(lbm_ctx* c, int n, int ckpt_every, VjpLayout& L) {
  L.K = std::min(ckpt_every, std::max(n, 1));
  L.nseg = (n + L.K - 1) / L.K;
  L.sb = (size_t)c->state_bytes;  // one state, and one adjoint field in the same layout
  const size_t need = L.sb * ((size_t)L.nseg + (size_t)L.K + 2);
  cudaError_t e;
  if (need > c->vjp_bytes) {
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return vfail(c, LBM_ECUDA, "lbm_vjp sync", e);
    cudaFree(c->d_vjp);
    c->d_vjp = nullptr;
    c->vjp_bytes = 0;
    c->vjp_gen = -1;
    if ((e = cudaMalloc(&c->d_vjp, need)) != cudaSuccess) {
      cudaGetLastError();
      return vfail(c, LBM_ENOMEM, "lbm_vjp work memory", e);
    }
    c->vjp_bytes = need;
  }
  L.base = static_cast<char*>(c->d_vjp);
  return LBM_OK;
}

// Forward pass: init, then n steps with a checkpoint at the start of every
// segment; the last segment's states go straight to the ring (the backward pass
// does not recompute them). The lattice ends holding f(x, n). Segments whose
// states are not kept take two steps a launch where the lattice's launch does.
int vjp_forward(lbm_ctx* c, int n, const VjpLayout& L, const double* d_rho0, const double* d_ux0,
                const double* d_uy0) {
  int s = lbm_init(c, d_rho0, d_ux0, d_uy0);
  if (s != LBM_OK) return s;
  cudaError_t e;
  for (int seg = 0; seg < L.nseg; ++seg) {
    if ((e = cudaMemcpyAsync(L.ckpt(seg), c->buf[c->cur], L.sb, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
      return vfail(c, LBM_ECUDA, "lbm_vjp checkpoint", e);
    const int len = std::min(L.K, n - seg * L.K);
    const bool last = seg == L.nseg - 1;
    for (int k = 0; k < len;) {
      if (!last && k + 1 < len && two_steps_apply(c)) {  // no state of this segment is kept: two a launch
        if ((e = fwd_step2(c, c->buf[c->cur], c->buf[c->cur ^ 1])) != cudaSuccess)
          return vfail(c, LBM_ECUDA, "lbm_vjp forward", e);
        c->cur ^= 1;
        c->t += 2;
        k += 2;
        continue;
      }
      const void* src = (last && k > 0) ? L.ring(k) : c->buf[c->cur];
      void* dst = (last && k + 1 < len) ? L.ring(k + 1) : c->buf[c->cur ^ 1];
      if ((e = fwd_step(c, src, dst)) != cudaSuccess) return vfail(c, LBM_ECUDA, "lbm_vjp forward", e);
      if (!last || k + 1 == len) c->cur ^= 1;
      c->t += 1;
      k += 1;
    }
  }
  c->vjp_gen = c->state_gen;
  c->vjp_n = n;
  c->vjp_k = L.K;
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_vjp_forward(lbm_ctx* c, int n, int ckpt_every, const double* d_rho0, const double* d_ux0,
                               const double* d_uy0) {
  if (!c) return LBM_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
    return vfail(c, LBM_EINVAL, "lbm_vjp_forward: the current CUDA device is not the lattice's device");
  if (n < 0 || ckpt_every < 1) return vfail(c, LBM_EINVAL, "lbm_vjp_forward: need n >= 0 and ckpt_every >= 1");
  if (!d_rho0 || !d_ux0 || !d_uy0) return vfail(c, LBM_EINVAL, "lbm_vjp_forward: NULL initial field");
  if (c->prec == LBM_F16_SHIFT)
    return vfail(c, LBM_EINVAL, "lbm_vjp_forward: storage forms LBM_F64, LBM_F64_DF and LBM_F32_SHIFT only");
  if (c->model > LBM_OREG_COMPLETE_NEQ)
    return vfail(c, LBM_EINVAL, "lbm_vjp_forward: no adjoint for LBM_LBGK_POLY");
  VjpLayout L;
  int s = vjp_layout(c, n, ckpt_every, L);
  if (s != LBM_OK) return s;
  return vjp_forward(c, n, L, d_rho0, d_ux0, d_uy0);
}

extern "C" int lbm_vjp_ex(lbm_ctx* c, int n, int ckpt_every, const double* d_rho0, const double* d_ux0,
                          const double* d_uy0, const double* g_rho, const double* g_ux, const double* g_uy,
                          double* g_rho0, double* g_ux0, double* g_uy0, int flags) {
  if (!c) return LBM_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
    return vfail(c, LBM_EINVAL, "lbm_vjp: the current CUDA device is not the lattice's device");
  if (n < 0 || ckpt_every < 1) return vfail(c, LBM_EINVAL, "lbm_vjp: need n >= 0 and ckpt_every >= 1");
  if (!d_rho0 || !d_ux0 || !d_uy0) return vfail(c, LBM_EINVAL, "lbm_vjp: NULL initial field");
  if (flags & ~LBM_VJP_REUSE_FORWARD) return vfail(c, LBM_EINVAL, "lbm_vjp_ex: unknown flags");
  if (c->prec == LBM_F16_SHIFT)
    return vfail(c, LBM_EINVAL, "lbm_vjp: storage forms LBM_F64, LBM_F64_DF and LBM_F32_SHIFT only");
  if (c->model > LBM_OREG_COMPLETE_NEQ) return vfail(c, LBM_EINVAL, "lbm_vjp: no adjoint for LBM_LBGK_POLY");
  VjpLayout L;
  int s;
  if (flags & LBM_VJP_REUSE_FORWARD) {
    const int K = std::min(ckpt_every, std::max(n, 1));
    if (c->vjp_gen != c->state_gen || c->vjp_n != n || c->vjp_k != K)
      return vfail(c, LBM_ESTATE, "lbm_vjp_ex: no forward pass of lbm_vjp_forward with these n and ckpt_every "
                                  "describes the lattice (it changed since, or none was run)");
    L.K = K;
    L.nseg = (n + K - 1) / K;
    L.sb = (size_t)c->state_bytes;
    L.base = static_cast<char*>(c->d_vjp);
  } else {
    if ((s = vjp_layout(c, n, ckpt_every, L)) != LBM_OK) return s;
    if ((s = vjp_forward(c, n, L, d_rho0, d_ux0, d_uy0)) != LBM_OK) return s;
  }
  cudaError_t e;
  c->vjp_gen = -1;  // the backward pass overwrites the ring of the last segment
  // seed lambda(n)
  void* lam[2] = {L.lam(0), L.lam(1)};
  int li = 0;
  e = adj_seed(c, g_rho, g_ux, g_uy, lam[li]);
  if (e != cudaSuccess) return vfail(c, LBM_ECUDA, "lbm_vjp seed", e);
  // backward over segments: recompute the segment's states (the last one is still in
  // the ring from the forward pass), then reverse them
  for (int seg = L.nseg - 1; seg >= 0; --seg) {
    const int len = std::min(L.K, n - seg * L.K);
    if (seg < L.nseg - 1) {
      const void* prev = L.ckpt(seg);
      for (int j = 1; j < len; ++j) {
        if ((e = fwd_step(c, prev, L.ring(j))) != cudaSuccess) return vfail(c, LBM_ECUDA, "lbm_vjp recompute", e);
        prev = L.ring(j);
      }
    }
    for (int j = len - 1; j >= 0; --j) {
      const void* fbuf = j == 0 ? L.ckpt(seg) : L.ring(j);
      e = adj_step(c, fbuf, lam[li], lam[li ^ 1]);
      if (e == cudaSuccess && c->n_walls > 0)
        e = olbm::launch_walls_adjoint(elem_bytes(c), lam[li], lam[li ^ 1], c->g, c->d_walls, c->n_walls, c->stream);
      if (e != cudaSuccess) return vfail(c, LBM_ECUDA, "lbm_vjp adjoint step", e);
      li ^= 1;
    }
  }
  // through the equilibrium initialisation
  e = adj_final(c, lam[li], d_rho0, d_ux0, d_uy0, g_rho0, g_ux0, g_uy0);
  if (e != cudaSuccess) return vfail(c, LBM_ECUDA, "lbm_vjp final", e);
  return LBM_OK;
}

extern "C" int lbm_vjp(lbm_ctx* c, int n, int ckpt_every, const double* d_rho0, const double* d_ux0,
                       const double* d_uy0, const double* g_rho, const double* g_ux, const double* g_uy,
                       double* g_rho0, double* g_ux0, double* g_uy0) {
  return lbm_vjp_ex(c, n, ckpt_every, d_rho0, d_ux0, d_uy0, g_rho, g_ux, g_uy, g_rho0, g_ux0, g_uy0, 0);
}
