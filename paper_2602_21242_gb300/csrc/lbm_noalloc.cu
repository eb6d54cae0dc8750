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
#include <cstdint>
#include <mutex>

#include "lbm.h"
#include "lbm_kernels.cuh"

namespace {

// Capacity: 8192 thread blocks x 5 partial sums (320 KiB).
constexpr int kNoAllocMaxBlocks = 8192;
__device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * 5];

// Device address of g_noalloc_partials, resolved once per device and CUDA
// context. In host code the symbol's name is only a host-side stand-in, so
// kernels get this address. A cudaDeviceReset (or the release and re-creation
// of the primary context) reloads the library's device image, and the array may
// then lie elsewhere: each entry remembers the unique id of the context it was
// resolved in (cuCtxGetId, reached through the runtime's driver entry points so
// that the library needs no link-time dependency on the driver library) and is
// resolved again when the current context's id differs. Where those entry
// points are missing the address is resolved on every call
// (cudaGetSymbolAddress allocates nothing).
constexpr int kMaxDevices = 128;
struct ScratchEntry {
  double* addr = nullptr;
  unsigned long long ctx_id = 0;
};
ScratchEntry g_scratch[kMaxDevices];
std::mutex g_scratch_lock;

using CtxGetCurrentFn = int (*)(void** ctx);                       // CUresult cuCtxGetCurrent(CUcontext*)
using CtxGetIdFn = int (*)(void* ctx, unsigned long long* ctx_id);  // CUresult cuCtxGetId(CUcontext, ...)
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
std::once_flag g_driver_once;

void load_driver_entry_points() {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess && p)
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(p);
  p = nullptr;
  q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess && p)
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(p);
  cudaGetLastError();  // a failed lookup leaves no sticky error behind
}

// Unique id of the current CUDA context, 0 if it cannot be read.
unsigned long long current_context_id() {
  std::call_once(g_driver_once, load_driver_entry_points);
  if (!g_ctx_get_current || !g_ctx_get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != 0 || ctx == nullptr || g_ctx_get_id(ctx, &id) != 0) return 0;
  return id;
}

int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
  // cudaGetDevice does not create the context; the symbol lookup below does,
  // so the id is read again after it when the first read found no context.
  unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> guard(g_scratch_lock);
  ScratchEntry& e = g_scratch[dev];
  if (e.addr == nullptr || id == 0 || e.ctx_id != id) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (err != cudaSuccess || p == nullptr) return LBM_ECUDA;
    if (id == 0) id = current_context_id();
    e.addr = static_cast<double*>(p);
    e.ctx_id = id;
  }
  *out = e.addr;
  return LBM_OK;
}

// [a, a + na) and [b, b + nb) share a byte.
bool overlaps(const void* a, long long na, const void* b, long long nb) {
  const uintptr_t pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
  return pa < pb + (uintptr_t)nb && pb < pa + (uintptr_t)na;
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
  if (!(theta > 0.0 && theta < 1.0) || !(tau > 0.5) || model < LBM_LBGK || model > LBM_LBGK_POLY)
    return olbm::set_thread_error(LBM_EINVAL, "lbm_step_noalloc: theta, tau or model out of range");
  if (!d_src || !d_dst || !d_diag5)
    return olbm::set_thread_error(LBM_EINVAL, "lbm_step_noalloc: NULL buffer");
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
  // The kernels take the buffers as __restrict__: no byte may be shared.
  const long long diag_bytes = 5 * (long long)sizeof(double);
  if (overlaps(d_src, bytes, d_dst, bytes) || overlaps(d_diag5, diag_bytes, d_src, bytes) ||
      overlaps(d_diag5, diag_bytes, d_dst, bytes))
    return olbm::set_thread_error(LBM_EINVAL, "lbm_step_noalloc: d_src, d_dst and d_diag5 overlap");
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
    case 4: e = launch<4>(g, c, d_src, d_dst, scratch, k, st); break;
    default: e = launch<5>(g, c, d_src, d_dst, scratch, k, st); break;
  }
  if (e == cudaSuccess) {
    noalloc_sum_kernel<<<1, kSumThreads, 0, st>>>(scratch, (int)nparts, d_diag5);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return olbm::set_thread_error(LBM_ECUDA, "lbm_step_noalloc launch: %s", cudaGetErrorString(e));
  return LBM_OK;
}
