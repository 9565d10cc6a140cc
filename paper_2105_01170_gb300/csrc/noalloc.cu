// Allocation-free entry point: the batched per-slice Jacobi SVD with its
// scratch memory in a fixed, statically allocated device array.
//
// Why: some callers cannot call cudaMalloc at the point where they need the
// work done -- for example the execution callback of an inference-engine
// plugin, which must not allocate, or a real-time loop whose device memory is
// budgeted once at start-up by another allocator.  sma_create allocates the
// handle's workspaces, so those callers cannot use the handle API.  This
// entry point takes only caller-owned inputs and outputs and uses a
// file-scope __device__ array for the block-mode working copy and the status
// word.  The array exists on every GPU that loads the library, for the
// lifetime of the process.
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB per device
constexpr size_t kStatusBytes = 256;                // status word slot
constexpr int kMaxDevices = 64;

// Device scratch: [status int | pad to 256 B | fp32 block-mode workspace].
static __device__ __align__(256) unsigned char g_sma_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};
void* g_scratch_ctx[kMaxDevices] = {nullptr};   // the context the address belongs to

// cuCtxGetCurrent through the runtime's driver entry point (no link-time
// dependency on the driver library, so the library still loads on a host
// without a GPU).
using CtxGetCurrent = int (*)(void**);
CtxGetCurrent ctx_get_current() {
  static CtxGetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      f = nullptr;
    cudaGetLastError();
    return reinterpret_cast<CtxGetCurrent>(f);
  }();
  return fn;
}

// Device address of g_sma_scratch on the current device, looked up once per
// device and context (the host-side symbol is only a stand-in, never a
// device address).  The context is kept beside the address: after
// cudaDeviceReset the device's primary context is a new one, the array is
// mapped again at a new address, and the lookup is repeated.
sma_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SMA_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return SMA_ERR_UNSUPPORTED;
  const CtxGetCurrent get = ctx_get_current();
  if (!get) return SMA_ERR_CUDA;
  void* ctx = nullptr;   // null while the runtime has not made a context current yet
  if (get(&ctx) != 0) return SMA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!ctx || !g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    // the lookup itself makes the device's primary context current
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sma_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return SMA_ERR_CUDA;
    }
    if (get(&ctx) != 0 || !ctx) return SMA_ERR_CUDA;
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_addr[dev];
  return SMA_OK;
}

}  // namespace

extern "C" {

sma_status sma_slice_svd_noalloc(const float* X, int32_t m, int32_t n, int32_t p, float* W,
                                 float* V, double* sigma, int32_t* sweeps, int32_t* status,
                                 int32_t max_sweeps, void* stream) {
  if (!X || !W || !V || !sigma || m <= 0 || n <= 0 || p <= 0) return SMA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* base = nullptr;
  sma_status s = scratch_address(&base);
  if (s != SMA_OK) return s;
  int dev = 0, max_smem = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return SMA_ERR_CUDA;
  }
  const sma::JacobiPlan pl = sma::jacobi_plan<float>(m, n, max_smem);
  if (pl.smem == 0) return SMA_ERR_ARG;   // one stacked column pair exceeds shared memory
  const int64_t per_slice = pl.block_mode ? (int64_t)(pl.mm + pl.rc) * pl.rc : 0;
  const int64_t capacity = (int64_t)((kScratchBytes - kStatusBytes) / sizeof(float));
  if (per_slice > capacity) return SMA_ERR_ARG;  // one slice's working copy exceeds 8 MiB
  const int chunk = per_slice > 0 ? (int)(capacity / per_slice < p ? capacity / per_slice : p) : p;
  int* d_status = static_cast<int*>(base);
  float* d_work = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + kStatusBytes);
  // the status word accumulates with atomicOr: clear what the last call left
  if (cudaMemsetAsync(d_status, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return SMA_ERR_CUDA;
  }
  const int64_t mn = (int64_t)m * n;
  for (int c0 = 0; c0 < p; c0 += chunk) {
    const int cnt = (p - c0) < chunk ? (p - c0) : chunk;
    sma::JacobiParams<float> J;
    J.src = X + c0 * mn; J.src_bs = mn; J.m = m; J.n = n;
    J.mm = pl.mm; J.rc = pl.rc; J.trans = pl.trans; J.ldS = pl.ldS; J.bcols = pl.bcols;
    J.g = pl.g; J.sort_n = pl.sort_n; J.tile = pl.tile;
    J.max_sweeps = max_sweeps > 0 ? max_sweeps : 30;
    J.tol = 4.0 * std::sqrt((double)pl.mm) * sma::Eps<float>::v;
    J.W = pl.block_mode ? d_work : nullptr; J.W_bs = per_slice;
    J.U = W + c0 * (int64_t)pl.mm * pl.rc; J.U_bs = (int64_t)pl.mm * pl.rc;
    J.V = V + c0 * (int64_t)pl.rc * pl.rc; J.V_bs = (int64_t)pl.rc * pl.rc;
    J.sigma = sigma + c0 * (int64_t)pl.rc;
    J.sweeps = sweeps ? sweeps + c0 : nullptr;
    J.status = d_status;
    if (sma::jacobi_svd<float>(J, cnt, pl.threads, pl.smem, st) != cudaSuccess) {
      cudaGetLastError();
      return SMA_ERR_CUDA;
    }
  }
  if (status && cudaMemcpyAsync(status, d_status, sizeof(int), cudaMemcpyDeviceToDevice, st) !=
                    cudaSuccess) {
    cudaGetLastError();
    return SMA_ERR_CUDA;
  }
  return SMA_OK;
}

}  // extern "C"
