// k_noalloc.cu -- W^T W for callers that cannot allocate device memory.
//
// aunmf_gram_w (the handle-based entry point) keeps its per-block partial
// Gram matrices in a workspace that the handle grows with cudaMalloc.  Some
// callers cannot allow that: code that runs while another framework's pool
// owns the device memory (a cudaMalloc there can fail or break the pool's
// accounting), or code on a fixed memory budget that must not grow at run
// time.  aunmf_gram_w_noalloc computes the same Gram matrix with the partials
// in a fixed, file-scope device array instead, and allocates nothing.
//
// The array is g_gram_scratch below: kNoAllocBlocks partial k x k matrices
// for k <= kNoAllocKMax, i.e. 256 * 64 * 64 floats = 4 MiB, which every GPU
// that loads this library holds until the process exits.
#include <cuda.h>

#include <mutex>

#include "internal.cuh"

namespace aunmf {
namespace {

constexpr int kNoAllocKMax = 64;
constexpr int kNoAllocBlocks = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_gram_scratch[kNoAllocBlocks * kNoAllocKMax * kNoAllocKMax];

std::mutex g_scratch_mu;
// device address of g_gram_scratch per device, and the id of the CUDA
// context it was looked up in (a device reset creates a new context, in
// which the module and its array are loaded again at another address)
float *g_scratch_dev[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Id of the current context (0 if the driver cannot tell).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
    cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array on the current device.  The symbol's
// name in host code is only a host-side stand-in; the address a kernel may
// use comes from cudaGetSymbolAddress, looked up with that device current
// once per device and context (again after a device reset).
float *scratch_for_current_device(int *status) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    *status = AUNMF_E_CUDA;
    return nullptr;
  }
  if (dev >= kMaxDevices) {
    *status = AUNMF_E_UNSUPPORTED;
    return nullptr;
  }
  const unsigned long long ctx = current_context_id();  // 0: no context yet
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      *status = AUNMF_E_CUDA;
      return nullptr;
    }
    g_scratch_dev[dev] = static_cast<float *>(p);
    // the lookup has made the runtime's context current if it was not yet
    g_scratch_ctx[dev] = current_context_id();
  }
  *status = AUNMF_OK;
  return g_scratch_dev[dev];
}

}  // namespace
}  // namespace aunmf

extern "C" int aunmf_gram_w_noalloc(const float *W, int64_t m, int k, float *G, void *stream) {
  using namespace aunmf;
  if (!W || !G || m < 1 || k < 1) return AUNMF_E_INVAL;
  if (k > kNoAllocKMax) return AUNMF_E_INVAL;  // beyond the fixed scratch array
  int status = AUNMF_OK;
  float *scratch = scratch_for_current_device(&status);
  if (!scratch) return status;
  // at most kNoAllocBlocks partials; each call overwrites every partial it
  // reads, so nothing has to be cleared between calls
  const cudaError_t e = launch_gram(W, m, k, k, G, scratch, kNoAllocBlocks,
                                    reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? AUNMF_OK : AUNMF_E_CUDA;
}
