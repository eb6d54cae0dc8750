// lbm_noalloc.cu -- lbm_step_noalloc: one fused FP64 step with diagnostics that
// allocates no device memory.
//
// Who needs it: code that must not call cudaMalloc/cudaFree -- a caller whose
// device memory all comes from its own pool or arena (so the library may not
// take more behind its back), or a caller in a latency-critical loop where an
// allocation's implicit synchronisation would stall the GPU. The regular entry
// points allocate per-lattice buffers in lbm_create; this one
// takes every input and output from the caller and keeps its only scratch (the
// per-block diagnostics partial sums) in a fixed array in the library's device
// image.
//
// The scratch array below is static device memory: every GPU that loads the
// library holds it until the process exits, and all calls on a device share
// it. Each call overwrites the partials it reads (every block writes its own
// five sums before the final reduction reads them), so nothing needs clearing
// between calls, but two calls whose work overlaps on one device (for example
// on different streams) race on it.
#include <mutex>

#include "lbm.h"
#include "lbm_kernels.cuh"

namespace {

// Capacity: 8192 thread blocks x 5 partial sums (320 KiB).
constexpr int kNoAllocMaxBlocks = 8192;
__device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * 5];

// Device address of g_noalloc_partials, resolved once per device. In host code
// the symbol's name is only a host-side stand-in, so kernels get this address.
constexpr int kMaxDevices = 128;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_lock;

int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
  std::lock_guard<std::mutex> guard(g_scratch_lock);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || p == nullptr) return LBM_ECUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return LBM_OK;
}

// Final fixed-order sum of the partials into the caller's 5 doubles.
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) noalloc_sum_kernel(const double* __restrict__ partials, int nparts,
                                                                  double* __restrict__ out5) {
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < nparts; j += kSumThreads)
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] += partials[(long long)j * 5 + k];
  double tot[5];
  olbm::block_sum<5, kSumThreads>(v, tot);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) out5[k] = tot[k];  // FP64 storage: no reference density to add
  }
}

template <int MODEL>
cudaError_t launch(const olbm::Geometry& g, const olbm::Coef<double>& c, const double* src, double* dst,
                   double* partials, const olbm::LaunchCfg& k, cudaStream_t st) {
  const dim3 grid = olbm::step_grid(g, k, 0), block(k.bx, k.by);
  olbm::step_kernel<MODEL, 0, true, false><<<grid, block, 0, st>>>(src, dst, g, c, partials, k.rows);
  return cudaGetLastError();
}

}  // namespace

extern "C" int lbm_step_noalloc(int nx, int ny, double theta, double tau, int model, const double* d_src,
                                double* d_dst, double* d_diag5, void* stream) {
  long long pitch = 0, plane = 0, bytes = 0;
  if (lbm_layout(nx, ny, LBM_F64, &pitch, &plane, &bytes) != LBM_OK)
    return olbm::set_thread_error(LBM_EINVAL, "lbm_step_noalloc: invalid size %d x %d", nx, ny);
  if (!(theta > 0.0 && theta < 1.0) || !(tau > 0.5) || model < LBM_LBGK || model > LBM_OREG_COMPLETE_NEQ)
    return olbm::set_thread_error(LBM_EINVAL, "lbm_step_noalloc: theta, tau or model out of range");
  if (!d_src || !d_dst || !d_diag5 || d_src == d_dst)
    return olbm::set_thread_error(LBM_EINVAL, "lbm_step_noalloc: NULL or aliased buffers");
  const olbm::Geometry g{nx, ny, pitch, plane};
  // 32 x 8 threads per block; rows per thread grows until the grid fits the scratch array.
  olbm::LaunchCfg k;
  k.bx = 32;
  k.by = 8;
  k.rows = 4;
  while (olbm::step_blocks(g, k, LBM_F64) > kNoAllocMaxBlocks && k.rows < 64) k.rows *= 2;
  const long long nparts = olbm::step_blocks(g, k, LBM_F64);
  if (nparts > kNoAllocMaxBlocks)
    return olbm::set_thread_error(LBM_EINVAL,
                                  "lbm_step_noalloc: a %d x %d lattice needs %lld thread blocks, more than the %d "
                                  "the fixed scratch holds (32 x 8 threads, up to 64 rows per thread)",
                                  nx, ny, nparts, kNoAllocMaxBlocks);
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != LBM_OK)
    return olbm::set_thread_error(LBM_ECUDA, "lbm_step_noalloc: cannot resolve the scratch array on this device");
  const olbm::Coef<double> c = olbm::make_coef<double>(theta, tau, 0.0);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (model) {
    case 0: e = launch<0>(g, c, d_src, d_dst, scratch, k, st); break;
    case 1: e = launch<1>(g, c, d_src, d_dst, scratch, k, st); break;
    case 2: e = launch<2>(g, c, d_src, d_dst, scratch, k, st); break;
    case 3: e = launch<3>(g, c, d_src, d_dst, scratch, k, st); break;
    default: e = launch<4>(g, c, d_src, d_dst, scratch, k, st); break;
  }
  if (e == cudaSuccess) {
    noalloc_sum_kernel<<<1, kSumThreads, 0, st>>>(scratch, (int)nparts, d_diag5);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return olbm::set_thread_error(LBM_ECUDA, "lbm_step_noalloc launch: %s", cudaGetErrorString(e));
  return LBM_OK;
}
