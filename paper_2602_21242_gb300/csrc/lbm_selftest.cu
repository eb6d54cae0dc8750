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
