// lbm_kernels.cuh -- CUDA kernels of the fused D2Q9 step (arXiv 2602.21242,
// Eq. 1) and its companions, templated on the collision model and the storage
// form. Included by one translation unit per storage form (lbm_f64.cu,
// lbm_f32.cu, lbm_f16.cu), each of which instantiates the launchers declared in
// lbm_launch.h.
//
// Buffer convention. A population buffer B holds, at node x, the
// post-collision values of the previous step still at their source node:
//   B_i(x) = f*_i(x, t - 1) = f_i(x + c_i, t)        (Eq. 1b)
// so one step is a pure pull:  f_i(x, t) = B_i(x - c_i)  (periodic wrap),
// collide at x (Eq. 1a), write f*_i(x, t) to B'_i(x). lbm_init and set_state
// write the push-shifted image of the pre-collision state; get_state and the
// moments pull it back.
#pragma once

#include <algorithm>
#include <type_traits>
#include <utility>

#include "lbm_device.cuh"
#include "lbm_df64.cuh"
#include "lbm_launch.h"

namespace olbm {

constexpr int kBX = 32;  // threads along x of the auxiliary kernels (init, moments, state copies, diagnostics)
constexpr int kBY = 8;   // rows per block of the auxiliary kernels
constexpr int kNT = kBX * kBY;
constexpr int kNDiag = 5;  // partial sums per block: m0, jx, jy, ke, non-finite nodes
constexpr int kDiagRows = 8;  // rows per thread of the diagnostics kernel (one block reduction per 8 nodes)
#ifndef OLBM_DF_JOIN
#define OLBM_DF_JOIN 2
#endif
// Double-word form: how a post-collision population is joined into FP64.
// 0: hi widened with integer instructions, lo converted on the FP64 pipe, both
// added there (two FP64-pipe instructions); 1: both converted on the FP64 pipe
// (three); 2: both widened with integer instructions and added on the FP64 pipe
// (one). With the collision's populations paired on the FP32 pipe, the FP64
// pipe is the first to fill: complete model at 4096^2, diagnostics every step,
// 96 registers: 24.2 GLUPS with 0 (FP64 pipe 68 % busy, warps waiting on it),
// 25.2 with 2.
constexpr int kDfJoin = OLBM_DF_JOIN;

// Source offsets of the pull f_i(x) = B_i(x - c_i) inside one plane.
__device__ __forceinline__ void pull_offsets(int x, int y, const Geometry& g, long long (&o)[9]) {
  const int xm = (x == 0) ? g.nx - 1 : x - 1;
  const int xp = (x == g.nx - 1) ? 0 : x + 1;
  const int ym = (y == 0) ? g.ny - 1 : y - 1;
  const int yp = (y == g.ny - 1) ? 0 : y + 1;
  const long long r = (long long)y * g.pitch, rm = (long long)ym * g.pitch, rp = (long long)yp * g.pitch;
  o[0] = r + x;    // c0 = ( 0, 0)
  o[1] = r + xm;   // c1 = ( 1, 0)
  o[2] = rm + x;   // c2 = ( 0, 1)
  o[3] = r + xp;   // c3 = (-1, 0)
  o[4] = rp + x;   // c4 = ( 0,-1)
  o[5] = rm + xm;  // c5 = ( 1, 1)
  o[6] = rm + xp;  // c6 = (-1, 1)
  o[7] = rp + xp;  // c7 = (-1,-1)
  o[8] = rp + xm;  // c8 = ( 1,-1)
}

// Finite test on the bit pattern (integer pipe, no FP64 compare): exponent not all ones.
__device__ __forceinline__ bool finite_bits(double v) {
  return (__double2hiint(v) & 0x7ff00000) != 0x7ff00000;
}
__device__ __forceinline__ bool finite_bits(float v) {
  return (__float_as_int(v) & 0x7f800000) != 0x7f800000;
}

// Block-wide sum of per-thread diagnostics, entirely in the compute type T
// (FP64 for the FP64 form, FP32 for the shifted forms, whose per-node values are
// small deviations): an xor butterfly in each warp (identical in every lane),
// then the warp totals in warp order by thread 0, which converts the four sums
// to FP64 for the global reduction. The non-finite count is an integer.
// Deterministic for a given block shape; at most kMaxWarps warps per block.
constexpr int kMaxWarps = 16;
template <typename T>
__device__ __forceinline__ void block_diag(T (&v)[4], int bad, double* __restrict__ out5) {
  __shared__ T red[kMaxWarps][4];
  __shared__ int redbad[kMaxWarps];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nw = (blockDim.x * blockDim.y) >> 5;
  if ((tid & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) red[tid >> 5][k] = v[k];
    redbad[tid >> 5] = bad;
  }
  __syncthreads();
  if (tid == 0) {
    T acc[4] = {T(0), T(0), T(0), T(0)};
    int nb = 0;
    for (int w = 0; w < nw; ++w) {
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += red[w][k];
      nb += redbad[w];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) out5[k] = (double)acc[k];
    out5[4] = (double)nb;
  }
}

// ------------------------------------------------------------------ fused step: one column of nodes
// Element loads/stores of one node pair (shifted forms, x even).
__device__ __forceinline__ f32x2 ld_pair(const float* p) { return f32x2(__ldg(reinterpret_cast<const float2*>(p))); }
__device__ __forceinline__ f32x2 ld_pair(const __half* p) {
  return f32x2(__half22float2(__ldg(reinterpret_cast<const __half2*>(p))));
}
__device__ __forceinline__ f32x2 ld_two(const float* p0, const float* p1) {
  return f32x2(make_float2(__ldg(p0), __ldg(p1)));
}
__device__ __forceinline__ f32x2 ld_two(const __half* p0, const __half* p1) {
  return f32x2(make_float2(__half2float(__ldg(p0)), __half2float(__ldg(p1))));
}
// L2-coherent variants (ld.global.cg) for kernels that read data written by
// other blocks of the same launch (the persistent batched kernel).
__device__ __forceinline__ double ld_cg(const double* p, double) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float* p, float) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const __half* p, float) {
  return __half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short*>(p))));
}
__device__ __forceinline__ f32x2 ld_pair_cg(const float* p) { return f32x2(__ldcg(reinterpret_cast<const float2*>(p))); }
__device__ __forceinline__ f32x2 ld_pair_cg(const __half* p) {
  const unsigned u = __ldcg(reinterpret_cast<const unsigned*>(p));
  return f32x2(__half22float2(*reinterpret_cast<const __half2*>(&u)));
}
__device__ __forceinline__ f32x2 ld_two_cg(const float* p0, const float* p1) {
  return f32x2(make_float2(__ldcg(p0), __ldcg(p1)));
}
__device__ __forceinline__ f32x2 ld_two_cg(const __half* p0, const __half* p1) {
  return f32x2(make_float2(ld_cg(p0, 0.0f), ld_cg(p1, 0.0f)));
}
__device__ __forceinline__ void st_pair(float* p, f32x2 v) { *reinterpret_cast<float2*>(p) = v.v; }
__device__ __forceinline__ void st_pair(__half* p, f32x2 v) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(v.v); }

// Per-thread diagnostics accumulator in the compute type CT: sums of m0, j_x,
// j_y and of j_x u_x + j_y u_y (twice the kinetic energy: two FMAs a node, the
// factor 1/2 applied once per block) over the nodes whose m0 is finite, and the
// count of the others.
__device__ __forceinline__ bool finite_lead(double x) { return finite_bits(x); }
__device__ __forceinline__ bool finite_lead(float x) { return finite_bits(x); }
__device__ __forceinline__ bool finite_lead(df64 x) { return finite_bits(x.hi); }
template <typename CT> struct DiagAcc {
  CT v[4];
  int bad;
  __device__ DiagAcc() : bad(0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = CT(0.0);
  }
  __device__ __forceinline__ void add(const NodeMoments<CT>& m) {
    if (finite_lead(m.m0)) {
      v[0] += m.m0;
      v[1] += m.jx;
      v[2] += m.jy;
      v[3] = fma(m.jx, m.ux, fma(m.jy, m.uy, v[3]));
    } else {
      ++bad;
    }
  }
};
// Packed pairs accumulate into four FP32 scalars: both nodes of a pair go into
// the same sums, which holds four registers fewer through the collision than
// packed sums would (measured on the FP16 form at 4096^2 with diagnostics every
// step: 138.6 -> 143.0 GLUPS) for the same FMA-pipe work.
template <> struct DiagAcc<f32x2> {
  float v[4];
  int bad;
  __device__ DiagAcc() : bad(0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = 0.0f;
  }
  __device__ __forceinline__ void add(const NodeMoments<f32x2>& m) {
    const bool ok0 = finite_bits(m.m0.v.x), ok1 = finite_bits(m.m0.v.y);
    auto acc = [&](float2 m0, float2 jx, float2 jy, float2 ux, float2 uy) {
      v[0] += m0.x + m0.y;
      v[1] += jx.x + jx.y;
      v[2] += jy.x + jy.y;
      v[3] = fmaf(jx.x, ux.x, fmaf(jx.y, ux.y, fmaf(jy.x, uy.x, fmaf(jy.y, uy.y, v[3]))));
    };
    if (ok0 && ok1) {
      acc(m.m0.v, m.jx.v, m.jy.v, m.ux.v, m.uy.v);
    } else {  // keep the finite node of the pair (selects, so that no NaN enters), count the other
      auto keep = [&](const f32x2& a) { return make_float2(ok0 ? a.v.x : 0.0f, ok1 ? a.v.y : 0.0f); };
      acc(keep(m.m0), keep(m.jx), keep(m.jy), keep(m.ux), keep(m.uy));
      bad += (ok0 ? 0 : 1) + (ok1 ? 0 : 1);
    }
  }
};

// Reduce a thread's accumulator over the block into out5 (thread 0 writes).
template <typename CT> __device__ __forceinline__ void block_diag_acc(DiagAcc<CT>& a, double* out5) {
  a.v[3] = scaled(a.v[3], 0.5f);  // kinetic energy
  if constexpr (std::is_same<CT, f32x2>::value) {
    block_diag<float>(a.v, a.bad, out5);
  } else if constexpr (std::is_same<CT, df64>::value) {
    double v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = join_f64(a.v[k]);
    block_diag<double>(v, a.bad, out5);

  } else {
    block_diag<CT>(a.v, a.bad, out5);
  }
}

// Update `rows` nodes (or node pairs) of column x: rows y0, y0 + dy, ...,
// pulling each row's 9 populations (Eq. 1b, periodic), colliding (Eq. 1a) and
// storing aligned. The next row's loads are issued before the current row's
// arithmetic, so each thread keeps two rows of loads in flight. With PAIRS
// (shifted forms, even nx, x even) the nodes x and x + 1 are updated together
// on packed f32x2 values; planes with c_ix = 0 are read as aligned 2-element
// vectors, the others element by element. With CG the loads bypass L1 (for
// data written earlier in the same launch by other blocks).
template <int MODEL, int PREC, bool DIAG, bool PAIRS, bool CG = false> struct Column {
  using S = typename Form<PREC>::S;
  using CT = typename std::conditional<PAIRS, f32x2, typename Form<PREC>::T>::type;

  __device__ static __forceinline__ void pull(const S* __restrict__ src, const Geometry& g, int x, int xm, int xp,
                                              int y, CT (&f)[9]) {
    const int ym = (y == 0) ? g.ny - 1 : y - 1;
    const int yp = (y == g.ny - 1) ? 0 : y + 1;
    const S* p0 = src + (long long)y * g.pitch;
    const S* pm = src + (long long)ym * g.pitch;
    const S* pp = src + (long long)yp * g.pitch;
    if constexpr (PAIRS) {
      // xm = x - 1, xp = x + 2 (periodic); the pair's second node is x + 1
      auto P = [](const S* q) { return CG ? ld_pair_cg(q) : ld_pair(q); };
      auto T2 = [](const S* q0, const S* q1) { return CG ? ld_two_cg(q0, q1) : ld_two(q0, q1); };
      f[0] = P(p0 + x);
      f[1] = T2(p0 + 1 * g.plane + xm, p0 + 1 * g.plane + x);
      f[2] = P(pm + 2 * g.plane + x);
      f[3] = T2(p0 + 3 * g.plane + x + 1, p0 + 3 * g.plane + xp);
      f[4] = P(pp + 4 * g.plane + x);
      f[5] = T2(pm + 5 * g.plane + xm, pm + 5 * g.plane + x);
      f[6] = T2(pm + 6 * g.plane + x + 1, pm + 6 * g.plane + xp);
      f[7] = T2(pp + 7 * g.plane + x + 1, pp + 7 * g.plane + xp);
      f[8] = T2(pp + 8 * g.plane + xm, pp + 8 * g.plane + x);
    } else {
      // xm = x - 1, xp = x + 1 (periodic)
      auto L = [](const S* q) { return CG ? ld_cg(q, CT()) : ld_t(q, CT()); };
      f[0] = L(p0 + x);
      f[1] = L(p0 + 1 * g.plane + xm);
      f[2] = L(pm + 2 * g.plane + x);
      f[3] = L(p0 + 3 * g.plane + xp);
      f[4] = L(pp + 4 * g.plane + x);
      f[5] = L(pm + 5 * g.plane + xm);
      f[6] = L(pm + 6 * g.plane + xp);
      f[7] = L(pp + 7 * g.plane + xp);
      f[8] = L(pp + 8 * g.plane + xm);
    }
  }

  __device__ static __forceinline__ void run(const S* __restrict__ src, S* __restrict__ dst, const Geometry& g,
                                             const Coef<CT>& c, int x, int y0, int dy, int rows,
                                             DiagAcc<CT>& acc) {
    if (x >= g.nx) return;
    const int xm = (x == 0) ? g.nx - 1 : x - 1;
    int xp;
    if constexpr (PAIRS) {
      xp = (x + 2 >= g.nx) ? x + 2 - g.nx : x + 2;
    } else {
      xp = (x == g.nx - 1) ? 0 : x + 1;
    }
    if constexpr (PREC == 3) {
      // Double-word form: the loads stay raw FP64 until their row is computed,
      // so the next row's loads are in flight during the current row's arithmetic
      // (splitting them at load time would wait for each load at once).
      using Raw = Column<MODEL, 0, DIAG, false, CG>;
      double r[9];
      int y = y0;
      if (y < g.ny) Raw::pull(src, g, x, xm, xp, y, r);
      for (int k = 0; k < rows && y < g.ny; ++k, y += dy) {
        df64 f[9];
        split_node(r, f);
        // r is free once split: the next row's loads go into it and are in
        // flight during this row's collision (no second set of registers).
        if ((k + 1 < rows) && (y + dy < g.ny)) Raw::pull(src, g, x, xm, xp, y + dy, r);
        S* q = dst + (long long)y * g.pitch + x;
        collide_df<MODEL>(
            f, c,
            [&](const NodeMoments<df64>& m) {
              if constexpr (DIAG) acc.add(m);
            },
            [&](int i, df64 v) {
              q[i * g.plane] = kDfJoin == 2 ? join_f64_int(v) : (kDfJoin == 1 ? join_f64_fp64pipe(v) : join_f64(v));
            });
      }
      return;
    }
    CT f[9], fn[9];
    int y = y0;
    int mode = 0;  // FP64: which products this warp's nodes take (see collide)
    if (y < g.ny) pull(src, g, x, xm, xp, y, f);
    for (int r = 0; r < rows && y < g.ny; ++r, y += dy) {
      const bool more = (r + 1 < rows) && (y + dy < g.ny);
      if (more) pull(src, g, x, xm, xp, y + dy, fn);
      collide<MODEL, Form<PREC>::kShift, CT>(
          f, c,
          [&](const NodeMoments<CT>& m) {
            if constexpr (DIAG) acc.add(m);
          },
          [&](CT (&r)[9]) { pull(src, g, x, xm, xp, y, r); }, &mode);
      S* q = dst + (long long)y * g.pitch + x;
      if constexpr (PAIRS) {
#pragma unroll
        for (int i = 0; i < 9; ++i) st_pair(q + i * g.plane, f[i]);
      } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) st_t(q + i * g.plane, f[i]);
      }
      if (more) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fn[i];
      }
    }
  }
};

// One lattice: block (bx, by) threads, bx a multiple of 32, bx * by <= 512; a
// thread updates column x (pairs: x and x + 1) at rows y0 + r * by, r < rows.
// With DIAG, per-block sums of mass (as the stored deviation m0), momentum,
// kinetic energy and the number of nodes whose pulled populations do not sum to
// a finite value go to partials[block * 5 + k].
template <int MODEL, int PREC, bool DIAG, bool PAIRS>
__device__ __forceinline__ void step_body(const typename Form<PREC>::S* __restrict__ src,
                                          typename Form<PREC>::S* __restrict__ dst, const Geometry& g,
                                          const Coef<typename Column<MODEL, PREC, DIAG, PAIRS>::CT>& c,
                                          double* __restrict__ partials, int rows) {
  using Col = Column<MODEL, PREC, DIAG, PAIRS>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int x = PAIRS ? 2 * t : t;
  const int y0 = blockIdx.y * blockDim.y * rows + threadIdx.y;
  DiagAcc<typename Col::CT> acc;
  Col::run(src, dst, g, c, x, y0, (int)blockDim.y, rows, acc);
  if constexpr (DIAG) block_diag_acc(acc, partials + (long long)(blockIdx.y * gridDim.x + blockIdx.x) * 5);
}

template <int MODEL, int PREC, bool DIAG, bool PAIRS>
__global__ void __launch_bounds__(512) step_kernel(const typename Form<PREC>::S* __restrict__ src,
                                                   typename Form<PREC>::S* __restrict__ dst, Geometry g,
                                                   Coef<typename Column<MODEL, PREC, DIAG, PAIRS>::CT> c,
                                                   double* __restrict__ partials, int rows) {
  step_body<MODEL, PREC, DIAG, PAIRS>(src, dst, g, c, partials, rows);
}

// Double-word form (3): launched with at most 256 threads a block and capped
// at 96 registers a thread, five blocks of 128 threads per SM. The complete
// model with fused diagnostics at 4096^2 (integer join): 80, 88 and 96
// registers give 24.7, 25.0 and 25.2 GLUPS (80 spills 48 bytes); uncapped it
// takes more than 100 registers and four blocks per SM.
#ifndef OLBM_DF_MAXNREG
#define OLBM_DF_MAXNREG 96
#endif
template <int MODEL, bool DIAG, bool PAIRS>
__global__ void __maxnreg__(OLBM_DF_MAXNREG) step_kernel_df(const double* __restrict__ src, double* __restrict__ dst,
                                                      Geometry g, Coef<typename Column<MODEL, 3, DIAG, PAIRS>::CT> c,
                                                      double* __restrict__ partials, int rows) {
  step_body<MODEL, 3, DIAG, PAIRS>(src, dst, g, c, partials, rows);
}

// The FP64 form is bound by the FP64 pipe. With its products on the integer
// pipes it is capped at 128 registers a thread (four blocks of 128 threads an
// SM, a few bytes spilled): the cap raised the 4096^2 rate from 5.57 to 5.77
// GLUPS when it was set. With every product on the FP64 pipe the rate measured
// the same for caps from 72 (seven blocks, spilling) to 128 registers
// (4751-4762 MLUPS). Launched with at most 512 threads.
#ifndef OLBM_F64_MAXNREG
#define OLBM_F64_MAXNREG 128
#endif
template <int MODEL, bool DIAG>
__global__ void __maxnreg__(OLBM_F64_MAXNREG) step_kernel_f64(const double* __restrict__ src, double* __restrict__ dst, Geometry g,
                                                Coef<double> c, double* __restrict__ partials, int rows) {
  step_body<MODEL, 0, DIAG, false>(src, dst, g, c, partials, rows);
}

}  // namespace olbm

#include "lbm_stream.cuh"

namespace olbm {

// Pipeline shapes per storage form: consumer threads (node pairs; FP64: single
// nodes) and ring slots.
#ifndef OLBM_STREAM_NC16
#define OLBM_STREAM_NC16 256
#endif
#ifndef OLBM_STREAM_STAGES
#define OLBM_STREAM_STAGES 8
#endif
constexpr int kStreamNC32 = 128, kStreamNC16 = OLBM_STREAM_NC16, kStreamStages = OLBM_STREAM_STAGES;
// consumer threads of the two-step tiles (launch kind 2)
#ifndef OLBM_STREAM2_NC16
#define OLBM_STREAM2_NC16 256
#endif
constexpr int kStream2NC32 = 128, kStream2NC16 = OLBM_STREAM2_NC16;
constexpr int kStreamNC64 = 128, kStreamStages64 = 4;
inline int stream_width(int prec) {
  return prec == 0 ? kStreamNC64 : 2 * (prec == 1 ? kStreamNC32 : kStreamNC16);
}

// ------------------------------------------------------------------ diagnostics of the state
// FP64 moments of the pulled populations of node (x, y) of f(x, t): m0 (the sum of
// the stored values), j_x, j_y, with the lattice's 0 and +-1 coefficients taken
// as adds and subtracts (16 operations, as in the collision).
template <int PREC>
__device__ __forceinline__ void pulled_moments(const typename Form<PREC>::S* __restrict__ src, const Geometry& g,
                                               int x, int y, double& m0, double& jx, double& jy) {
  long long o[9];
  pull_offsets(x, y, g, o);
  double f[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = to_double(src[i * g.plane + o[i]]);
  const double s13 = f[1] + f[3], d13 = f[1] - f[3];
  const double s24 = f[2] + f[4], d24 = f[2] - f[4];
  const double s57 = f[5] + f[7], d57 = f[5] - f[7];
  const double s68 = f[6] + f[8], d68 = f[6] - f[8];
  m0 = f[0] + (s13 + s24) + (s57 + s68);
  jx = d13 + (d57 - d68);
  jy = d24 + (d57 + d68);
}

// Pull only (no collision): FP64 moments of f(x, t), block partials as above;
// each thread takes kDiagRows rows of its column, so the block reduction is paid
// once per kDiagRows nodes. The kinetic energy uses the reciprocal of the
// collision (a density outside [2^-126, 2^126) makes it non-finite).
template <int PREC>
__global__ void __launch_bounds__(kNT) diag_kernel(const typename Form<PREC>::S* __restrict__ src, Geometry g,
                                                   double rho_ref, double* __restrict__ partials) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y0 = blockIdx.y * kBY * kDiagRows + threadIdx.y;
  double acc[kNDiag] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (x < g.nx) {
    for (int r = 0; r < kDiagRows; ++r) {
      const int y = y0 + r * kBY;
      if (y >= g.ny) break;
      double m0, jx, jy;
      pulled_moments<PREC>(src, g, x, y, m0, jx, jy);
      if (finite_bits(m0)) {
        acc[0] += m0;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] = fma(0.5 * fma(jx, jx, jy * jy), recip(rho_ref + m0), acc[3]);
      } else {
        acc[4] += 1.0;
      }
    }
  }
  double tot[kNDiag];
  block_sum<kNDiag, kNT>(acc, tot);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double* p = partials + (long long)(blockIdx.y * gridDim.x + blockIdx.x) * kNDiag;
#pragma unroll
    for (int k = 0; k < kNDiag; ++k) p[k] = tot[k];
  }
}

// ------------------------------------------------------------------ init, moments, state copies
// B_i(x) = f^eq_i(rho0(x + c_i), u0(x + c_i)) - rest_i: the buffer whose pull is f^eq(rho0, u0).
// Written as a push (each element once): node x forms its nine f^eq_i from one
// set of per-axis factors and stores them at x - c_i.
template <int PREC>
__global__ void __launch_bounds__(kNT) init_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                                                   const double* __restrict__ uy, Geometry g, double theta,
                                                   double rho_ref, typename Form<PREC>::S* __restrict__ dst) {
  using S = typename Form<PREC>::S;
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  long long o[9];
  pull_offsets(x, y, g, o);
  const long long n = (long long)y * g.nx + x;
  const double r = rho[n], u = ux[n], v = uy[n];
  const double px[3] = {geq_factor(-1, u, theta), geq_factor(0, u, theta), geq_factor(1, u, theta)};
  const double py[3] = {geq_factor(-1, v, theta), geq_factor(0, v, theta), geq_factor(1, v, theta)};
  const double rpx[3] = {r * px[0], r * px[1], r * px[2]};
  // rest values rho_ref W(a) W(b): three distinct products
  const double w0 = 1.0 - theta, wp = 0.5 * theta;
  const double rest[3] = {rho_ref * (w0 * w0), rho_ref * (w0 * wp), rho_ref * (wp * wp)};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int nz = (cx_of(i) != 0) + (cy_of(i) != 0);  // axes with a nonzero velocity component
    dst[i * g.plane + o[i]] = from_double<S>(fma(rpx[cx_of(i) + 1], py[cy_of(i) + 1], -rest[nz]));
  }
}

// (rho, u) of f(x, t) in FP64, unpadded [y][x] output.
template <int PREC>
__global__ void __launch_bounds__(kNT) moments_kernel(const typename Form<PREC>::S* __restrict__ src, Geometry g,
                                                      double rho_ref, double* __restrict__ rho,
                                                      double* __restrict__ ux, double* __restrict__ uy) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  double m0, jx, jy;
  pulled_moments<PREC>(src, g, x, y, m0, jx, jy);
  const double r = rho_ref + m0;
  const double ir = recip(r);  // a density outside [2^-126, 2^126) gives non-finite velocities
  const long long n = (long long)y * g.nx + x;
  rho[n] = r;
  ux[n] = jx * ir;
  uy[n] = jy * ir;
}

// out_i(x) = B_i(x - c_i) + rest_i  (pre-collision f(x, t), FP64, unpadded [i][y][x]).
template <int PREC>
__global__ void __launch_bounds__(kNT) get_state_kernel(const typename Form<PREC>::S* __restrict__ src, Geometry g,
                                                        double theta, double rho_ref, double* __restrict__ out) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  long long o[9];
  pull_offsets(x, y, g, o);
  const long long nodes = (long long)g.nx * g.ny;
  const long long n = (long long)y * g.nx + x;
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i * nodes + n] = to_double(src[i * g.plane + o[i]]) + rest_value(i, theta, rho_ref);
}

// B_i(x - c_i) = in_i(x) - rest_i: the inverse of get_state (each element written once).
template <int PREC>
__global__ void __launch_bounds__(kNT) set_state_kernel(const double* __restrict__ in, Geometry g, double theta,
                                                        double rho_ref, typename Form<PREC>::S* __restrict__ dst) {
  using S = typename Form<PREC>::S;
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  long long o[9];
  pull_offsets(x, y, g, o);
  const long long nodes = (long long)g.nx * g.ny;
  const long long n = (long long)y * g.nx + x;
#pragma unroll
  for (int i = 0; i < 9; ++i) dst[i * g.plane + o[i]] = from_double<S>(in[i * nodes + n] - rest_value(i, theta, rho_ref));
}

// ------------------------------------------------------------------ launchers
inline dim3 grid_of(const Geometry& g) { return dim3((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY); }
inline dim3 diag_grid(const Geometry& g) {
  return dim3((g.nx + kBX - 1) / kBX, (g.ny + kBY * kDiagRows - 1) / (kBY * kDiagRows));
}
// The shifted forms (1, 2) update node pairs (x, x + 1) when nx is even.
inline bool uses_pairs(int prec, const Geometry& g) { return (prec == 1 || prec == 2) && (g.nx % 2) == 0; }
// The pipeline kernel (launch kind 1) applies to the shifted forms and FP64, any nx.
inline bool uses_stream(int prec, const Geometry& g, const LaunchCfg& k) {
  (void)g;
  return (k.kind == 1 && (prec == 0 || prec == 1 || prec == 2)) || (k.kind == 2 && (prec == 1 || prec == 2));
}
// Two-step tiles (kind 2): 2 NC - 2 output columns; any nx.
inline int stream2_width(int prec) { return 2 * (prec == 1 ? kStream2NC32 : kStream2NC16) - 2; }
inline bool step2_applies(int prec, const Geometry& g, const LaunchCfg& k) {
  return k.kind == 2 && (prec == 1 || prec == 2) && g.nx >= 1;
}
inline dim3 step2_grid(const Geometry& g, const LaunchCfg& k, int prec) {
  const int w = stream2_width(prec);
  return dim3((g.nx + w - 1) / w, (g.ny + k.rows - 1) / k.rows);
}
inline dim3 step_grid(const Geometry& g, const LaunchCfg& k, int prec) {
  if (uses_stream(prec, g, k)) {
    const int w = stream_width(prec);
    const int sx = (g.nx + w - 1) / w, sy = (g.ny + k.rows - 1) / k.rows;
    if (k.bx == 0) return dim3(sx, sy);  // one CTA per tile
    const long long tiles = (long long)sx * sy;
    return dim3((unsigned)(k.cap > 0 ? std::min<long long>(tiles, k.cap) : tiles));
  }
  const int cols = uses_pairs(prec, g) ? 2 * k.bx : k.bx;
  return dim3((g.nx + cols - 1) / cols, (g.ny + k.by * k.rows - 1) / (k.by * k.rows));
}

// Launch of a pipeline step kernel with programmatic stream serialisation (see
// pdl_wait): the grid may be scheduled while the previous kernel of the stream
// finishes. OLBM_PDL=0 launches it as an ordinary stream-ordered kernel.
#ifndef OLBM_PDL
#define OLBM_PDL 1
#endif
template <typename... KArgs, typename... Args>
cudaError_t launch_step_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = OLBM_PDL ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <int PREC> struct Launch {
  using S = typename Form<PREC>::S;
  using T = typename Form<PREC>::T;

  template <int MODEL, bool PAIRS>
  static cudaError_t step_p(const StepArgs& a, cudaStream_t st) {
    using CT = typename Column<MODEL, PREC, false, PAIRS>::CT;
    const Coef<CT> c = make_coef<CT>(a.theta, a.tau, a.rho_ref);
    const dim3 block(a.cfg.bx, a.cfg.by);
    const dim3 grid = step_grid(a.g, a.cfg, PREC);
    if constexpr (PREC == 3) {
      if (block.x * block.y > 256) return cudaErrorInvalidConfiguration;
      if (a.diag)
        step_kernel_df<MODEL, true, PAIRS><<<grid, block, 0, st>>>((const S*)a.src, (S*)a.dst, a.g, c, a.partials,
                                                                    a.cfg.rows);
      else
        step_kernel_df<MODEL, false, PAIRS><<<grid, block, 0, st>>>((const S*)a.src, (S*)a.dst, a.g, c, a.partials,
                                                                     a.cfg.rows);
    } else if constexpr (PREC == 0) {
      if (a.diag)
        step_kernel_f64<MODEL, true><<<grid, block, 0, st>>>((const S*)a.src, (S*)a.dst, a.g, c, a.partials,
                                                              a.cfg.rows);
      else
        step_kernel_f64<MODEL, false><<<grid, block, 0, st>>>((const S*)a.src, (S*)a.dst, a.g, c, a.partials,
                                                               a.cfg.rows);
    } else {
      if (a.diag)
        step_kernel<MODEL, PREC, true, PAIRS><<<grid, block, 0, st>>>((const S*)a.src, (S*)a.dst, a.g, c, a.partials,
                                                                       a.cfg.rows);
      else
        step_kernel<MODEL, PREC, false, PAIRS><<<grid, block, 0, st>>>((const S*)a.src, (S*)a.dst, a.g, c,
                                                                        a.partials, a.cfg.rows);
    }
    return cudaGetLastError();
  }

  template <int MODEL, bool DIAG>
  static cudaError_t stream_d(const StepArgs& a, cudaStream_t st) {
    constexpr int NC = PREC == 1 ? kStreamNC32 : kStreamNC16;
    using Shape = StreamShape<PREC, NC, kStreamStages>;
    auto kernel = step_stream_kernel<MODEL, PREC, DIAG, NC, kStreamStages>;
    auto pkernel = step_stream_persistent_kernel<MODEL, PREC, DIAG, NC, kStreamStages>;
    // Per instantiation and device, once: opt in to the large shared-memory
    // carve-out (a per-device attribute) and size the persistent grid (resident
    // CTAs per SM x SMs). Concurrent first calls store the same values.
    constexpr int kMaxDev = 64;
    static int resident[kMaxDev] = {0}, sms_of[kMaxDev] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    if (resident[dev] == 0) {
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, Shape::kSmemBytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pkernel, cudaFuncAttributeMaxDynamicSharedMemorySize, Shape::kSmemBytes);
      int sms = 0, per_sm = 0;
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pkernel, NC + 32, Shape::kSmemBytes);
      if (e != cudaSuccess) return e;
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
      sms_of[dev] = sms;
      resident[dev] = per_sm * sms;
    }
    // bx > 0: a persistent grid of bx CTAs per SM (at most the resident count);
    // bx == 0: one CTA per tile.
    LaunchCfg k = a.cfg;
    k.cap = a.cfg.bx > 0 ? std::min(resident[dev], a.cfg.bx * sms_of[dev]) : 0;
    const dim3 grid = step_grid(a.g, k, PREC);
    if (a.parts_used) *a.parts_used = (long long)grid.x * grid.y;
    const Coef<f32x2> c = make_coef<f32x2>(a.theta, a.tau, a.rho_ref);
    if (a.cfg.bx == 0)
      return launch_step_kernel(kernel, grid, dim3(NC + 32), Shape::kSmemBytes, st, (const S*)a.src, (S*)a.dst, a.g,
                                c, a.partials, a.cfg.rows, a.err);
    if (a.err == nullptr || a.sched == nullptr) return cudaErrorInvalidValue;
    return launch_step_kernel(pkernel, grid, dim3(NC + 32), Shape::kSmemBytes, st, (const S*)a.src, (S*)a.dst, a.g, c,
                              a.partials, a.cfg.rows, a.err, a.sched);
  }

  // FP64 pipeline (launch kind 1, one CTA per tile).
  template <int MODEL, bool DIAG>
  static cudaError_t stream_f64(const StepArgs& a, cudaStream_t st) {
    using Shape = StreamShape<0, kStreamNC64, kStreamStages64>;
    static_assert(Shape::kSmemBytes <= 48 * 1024, "the FP64 ring fits the default shared-memory window");
    if (a.err == nullptr || a.cfg.bx != 0) return cudaErrorInvalidValue;
    const dim3 grid = step_grid(a.g, a.cfg, 0);
    if (a.parts_used) *a.parts_used = (long long)grid.x * grid.y;
    const Coef<double> c = make_coef<double>(a.theta, a.tau, a.rho_ref);
    return launch_step_kernel(step_stream_f64_kernel<MODEL, DIAG, kStreamNC64, kStreamStages64>, grid,
                              dim3(kStreamNC64 + 32), Shape::kSmemBytes, st, (const double*)a.src, (double*)a.dst,
                              a.g, c, a.partials, a.cfg.rows, a.err);
  }

  template <int MODEL>
  static cudaError_t step_m(const StepArgs& a, cudaStream_t st) {
    if constexpr (PREC == 1 || PREC == 2) {
      if (uses_stream(PREC, a.g, a.cfg)) return a.diag ? stream_d<MODEL, true>(a, st) : stream_d<MODEL, false>(a, st);
    }
    if constexpr (PREC == 0) {
      if (uses_stream(PREC, a.g, a.cfg))
        return a.diag ? stream_f64<MODEL, true>(a, st) : stream_f64<MODEL, false>(a, st);
    }
    if constexpr (PREC == 1 || PREC == 2) {
      if (uses_pairs(PREC, a.g)) return step_p<MODEL, true>(a, st);
    }
    return step_p<MODEL, false>(a, st);
  }

  static cudaError_t step(const StepArgs& a, cudaStream_t st) {
    if (!valid_cfg(a.cfg)) return cudaErrorInvalidConfiguration;
    switch (a.model) {
      case 0: return step_m<0>(a, st);
      case 1: return step_m<1>(a, st);
      case 2: return step_m<2>(a, st);
      case 3: return step_m<3>(a, st);
      case 4: return step_m<4>(a, st);
      case 5: return step_m<5>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }

  static cudaError_t diag(const void* src, const Geometry& g, double rho_ref, double* partials, cudaStream_t st) {
    diag_kernel<PREC><<<diag_grid(g), dim3(kBX, kBY), 0, st>>>((const S*)src, g, rho_ref, partials);
    return cudaGetLastError();
  }

  static cudaError_t init(const double* rho, const double* ux, const double* uy, const Geometry& g, double theta,
                          double rho_ref, void* dst, cudaStream_t st) {
    init_kernel<PREC><<<grid_of(g), dim3(kBX, kBY), 0, st>>>(rho, ux, uy, g, theta, rho_ref, (S*)dst);
    return cudaGetLastError();
  }

  static cudaError_t moments(const void* src, const Geometry& g, double rho_ref, double* rho, double* ux,
                             double* uy, cudaStream_t st) {
    moments_kernel<PREC><<<grid_of(g), dim3(kBX, kBY), 0, st>>>((const S*)src, g, rho_ref, rho, ux, uy);
    return cudaGetLastError();
  }

  static cudaError_t get_state(const void* src, const Geometry& g, double theta, double rho_ref, double* out,
                               cudaStream_t st) {
    get_state_kernel<PREC><<<grid_of(g), dim3(kBX, kBY), 0, st>>>((const S*)src, g, theta, rho_ref, out);
    return cudaGetLastError();
  }

  static cudaError_t set_state(const double* in, const Geometry& g, double theta, double rho_ref, void* dst,
                               cudaStream_t st) {
    set_state_kernel<PREC><<<grid_of(g), dim3(kBX, kBY), 0, st>>>(in, g, theta, rho_ref, (S*)dst);
    return cudaGetLastError();
  }
};

}  // namespace olbm

// Defines the C++ entry points of lbm_launch.h for one storage form.
#define OLBM_DEFINE_LAUNCHERS(PREC, SUFFIX)                                                                      \
  namespace olbm {                                                                                               \
  cudaError_t launch_step_##SUFFIX(const StepArgs& a, cudaStream_t st) { return Launch<PREC>::step(a, st); }     \
  cudaError_t launch_diag_##SUFFIX(const void* src, const Geometry& g, double rho_ref, double* partials,         \
                                   cudaStream_t st) {                                                            \
    return Launch<PREC>::diag(src, g, rho_ref, partials, st);                                                    \
  }                                                                                                              \
  cudaError_t launch_init_##SUFFIX(const double* rho, const double* ux, const double* uy, const Geometry& g,     \
                                   double theta, double rho_ref, void* dst, cudaStream_t st) {                   \
    return Launch<PREC>::init(rho, ux, uy, g, theta, rho_ref, dst, st);                                          \
  }                                                                                                              \
  cudaError_t launch_moments_##SUFFIX(const void* src, const Geometry& g, double rho_ref, double* rho,           \
                                      double* ux, double* uy, cudaStream_t st) {                                 \
    return Launch<PREC>::moments(src, g, rho_ref, rho, ux, uy, st);                                              \
  }                                                                                                              \
  cudaError_t launch_get_state_##SUFFIX(const void* src, const Geometry& g, double theta, double rho_ref,        \
                                        double* out, cudaStream_t st) {                                          \
    return Launch<PREC>::get_state(src, g, theta, rho_ref, out, st);                                             \
  }                                                                                                              \
  cudaError_t launch_set_state_##SUFFIX(const double* in, const Geometry& g, double theta, double rho_ref,       \
                                        void* dst, cudaStream_t st) {                                            \
    return Launch<PREC>::set_state(in, g, theta, rho_ref, dst, st);                                              \
  }                                                                                                              \
  }
