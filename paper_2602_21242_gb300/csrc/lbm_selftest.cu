// lbm_selftest.cu -- makes the library's bounded device-side waits run out on
// purpose and reports how the host sees it, so that the timeout paths are
// exercised without faulting or hanging the GPU: each kernel waits on a
// condition that nothing will satisfy, using the same wait routines as the
// pipelined step kernel (mbarrier phase) and the persistent batched kernel
// (grid barrier); each wait gives up after about a second and sets a flag.
#include <chrono>

#include "lbm.h"
#include "lbm_kernels.cuh"

namespace {

// One block waits for an mbarrier phase that needs two arrivals and gets none.
__global__ void stuck_mbarrier_kernel(int* err) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    olbm::mbar_init(&bar, 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  olbm::mbar_wait(&bar, 0u, err);
}

// Two blocks, one of which leaves without arriving: the other waits at the grid barrier.
__global__ void stuck_grid_barrier_kernel(olbm::GridBarrier* b) {
  if (blockIdx.x == 0) return;
  olbm::grid_sync(b, gridDim.x);
}

__global__ void fp64_helpers_kernel(int op, const double* __restrict__ x, long long n, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  double r;
  switch (op) {
    case 0: r = olbm::scaled(v, 0.5f); break;
    case 1: r = olbm::scaled(v, -0.5f); break;
    case 2: r = olbm::scaled(v, 0.25f); break;
    case 3: r = olbm::recip(v); break;
    default: r = olbm::widen_f32(olbm::narrow_trunc(v)); break;
  }
  out[i] = r;
}

}  // namespace

extern "C" int lbm_selftest_fp64(int op, const double* h_x, long long n, double* h_out) {
  if (op < 0 || op > 4 || n < 0 || (n > 0 && (h_x == nullptr || h_out == nullptr))) return LBM_EINVAL;
  if (n == 0) return LBM_OK;
  double* d = nullptr;
  const size_t bytes = sizeof(double) * (size_t)n;
  if (cudaMalloc(&d, 2 * bytes) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ENOMEM;
  }
  cudaError_t e = cudaMemcpy(d, h_x, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    fp64_helpers_kernel<<<(unsigned)((n + 255) / 256), 256>>>(op, d, n, d + n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h_out, d + n, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_selftest_timeout(int which, double* h_seconds) {
  if (which != 0 && which != 1) return LBM_EINVAL;
  int* d = nullptr;
  const size_t bytes = which == 0 ? sizeof(int) : sizeof(olbm::GridBarrier);
  if (cudaMalloc(&d, bytes) != cudaSuccess) return LBM_ENOMEM;
  cudaMemset(d, 0, bytes);
  const auto t0 = std::chrono::steady_clock::now();
  if (which == 0)
    stuck_mbarrier_kernel<<<1, 32>>>(d);
  else
    stuck_grid_barrier_kernel<<<2, 32>>>(reinterpret_cast<olbm::GridBarrier*>(d));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int flag = 0;
  if (e == cudaSuccess)
    e = cudaMemcpy(&flag, which == 0 ? d : &reinterpret_cast<olbm::GridBarrier*>(d)->err, sizeof(int),
                   cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (h_seconds) *h_seconds = secs;
  if (e != cudaSuccess) return LBM_ECUDA;
  return flag ? LBM_ETIMEOUT : LBM_OK;
}

namespace {

// The integer-pipe binary64 sum and product next to the FP64 instructions.
__global__ void fp64_emu_kernel(int op, const double* __restrict__ a, const double* __restrict__ b, long long n,
                                double* __restrict__ emu, double* __restrict__ fp64) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (op == 0) {
    emu[i] = olbm::emu::add64(a[i], b[i]);
    fp64[i] = __dadd_rn(a[i], b[i]);
  } else {
    emu[i] = olbm::emu::mul64(a[i], b[i]);
    fp64[i] = __dmul_rn(a[i], b[i]);
  }
}

template <int MODEL>
__global__ void collide_f64_kernel(const double* __restrict__ fin, long long n, olbm::Coef<double> c, int mode,
                                   double* __restrict__ out_emu, double* __restrict__ out_ref) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[9];
  olbm::d64f g[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) f[k] = fin[i * 9 + k], g[k] = olbm::d64f(f[k]);
  double mom[5], momr[5];
  int md = mode;  // the products the collision starts with (see olbm::collide)
  olbm::collide<MODEL, false, double>(
      f, c,
      [&](const olbm::NodeMoments<double>& m) {
        mom[0] = m.m0, mom[1] = m.jx, mom[2] = m.jy, mom[3] = m.ux, mom[4] = m.uy;
      },
      olbm::KeepInputs(), &md);
  const olbm::Coef<olbm::d64f> cr = olbm::coef_cast<olbm::d64f>(c);
  olbm::collide_form<MODEL, false, olbm::d64f>(g, cr, [&](const olbm::NodeMoments<olbm::d64f>& m) {
    momr[0] = m.m0.v, momr[1] = m.jx.v, momr[2] = m.jy.v, momr[3] = m.ux.v, momr[4] = m.uy.v;
  });
#pragma unroll
  for (int k = 0; k < 9; ++k) out_emu[i * 14 + k] = f[k], out_ref[i * 14 + k] = g[k].v;
#pragma unroll
  for (int k = 0; k < 5; ++k) out_emu[i * 14 + 9 + k] = mom[k], out_ref[i * 14 + 9 + k] = momr[k];
}

}  // namespace

extern "C" int lbm_selftest_fp64_emu(int op, const double* h_a, const double* h_b, long long n, double* h_emu,
                                     double* h_fp64) {
  if ((op != 0 && op != 1) || n < 0 ||
      (n > 0 && (h_a == nullptr || h_b == nullptr || h_emu == nullptr || h_fp64 == nullptr)))
    return LBM_EINVAL;
  if (n == 0) return LBM_OK;
  double* d = nullptr;
  const size_t bytes = sizeof(double) * (size_t)n;
  if (cudaMalloc(&d, 4 * bytes) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ENOMEM;
  }
  cudaError_t e = cudaMemcpy(d, h_a, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d + n, h_b, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    fp64_emu_kernel<<<(unsigned)((n + 255) / 256), 256>>>(op, d, d + n, n, d + 2 * n, d + 3 * n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h_emu, d + 2 * n, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h_fp64, d + 3 * n, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_selftest_collide_f64(int model, int mode, double theta, double tau, const double* h_f,
                                        long long n, double* h_emu, double* h_ref) {
  if (model < LBM_LBGK || model > LBM_LBGK_POLY || mode < 0 || mode > 2 || n < 0 || !(theta > 0.0 && theta < 1.0) ||
      !(tau > 0.5) ||
      (n > 0 && (h_f == nullptr || h_emu == nullptr || h_ref == nullptr)))
    return LBM_EINVAL;
  if (n == 0) return LBM_OK;
  double* d = nullptr;
  const size_t in_bytes = sizeof(double) * 9 * (size_t)n, out_bytes = sizeof(double) * 14 * (size_t)n;
  if (cudaMalloc(&d, in_bytes + 2 * out_bytes) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ENOMEM;
  }
  double* d_emu = d + 9 * n;
  double* d_ref = d_emu + 14 * n;
  const olbm::Coef<double> c = olbm::make_coef<double>(theta, tau, 1.0);
  cudaError_t e = cudaMemcpy(d, h_f, in_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const unsigned grid = (unsigned)((n + 127) / 128);
    switch (model) {
      case 0: collide_f64_kernel<0><<<grid, 128>>>(d, n, c, mode, d_emu, d_ref); break;
      case 1: collide_f64_kernel<1><<<grid, 128>>>(d, n, c, mode, d_emu, d_ref); break;
      case 2: collide_f64_kernel<2><<<grid, 128>>>(d, n, c, mode, d_emu, d_ref); break;
      case 3: collide_f64_kernel<3><<<grid, 128>>>(d, n, c, mode, d_emu, d_ref); break;
      case 4: collide_f64_kernel<4><<<grid, 128>>>(d, n, c, mode, d_emu, d_ref); break;
      default: collide_f64_kernel<5><<<grid, 128>>>(d, n, c, mode, d_emu, d_ref); break;
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h_emu, d_emu, out_bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h_ref, d_ref, out_bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
