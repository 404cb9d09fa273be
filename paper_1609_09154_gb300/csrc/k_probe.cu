// k_probe.cu -- the gather roof of the sparse products (a measurement, not a
// step of the method).
//
// Each nonzero of a sparse product (Sec. 5.2.1) gathers one k-vector of the
// fixed factor, a row at a data-dependent address.  With 200-byte rows
// (k = 50) spread over a 100-500 MB factor, those gathers, served from L2 or
// from HBM through it, bound the products: the algorithmic HBM bytes are
// not the limit.  This kernel times the gathers alone for the same index
// stream: every index's row is loaded once, with the widest loads (a
// half-warp per row, 16 bytes a lane, over rows padded to a multiple of 4
// floats), summed into a register that is never stored, and nothing else is
// done.  The products' time over this kernel's is the fraction of the roof
// they reach.
#include "internal.cuh"

namespace aunmf {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeWarps = kProbeThreads / kWarp;

__global__ void __launch_bounds__(kProbeThreads)
    k_probe_gather(const int32_t *__restrict__ idx, int64_t n, const float *__restrict__ X,
                   int k, int64_t ld4, float *__restrict__ sink) {
  const int lane = threadIdx.x & 31, q = lane & 15, hb = lane >> 4;
  const int64_t w0 = (int64_t)blockIdx.x * kProbeWarps + (threadIdx.x >> 5);
  const int64_t ws = (int64_t)gridDim.x * kProbeWarps;
  const bool act = 4 * q < k;
  const float4 *X4 = reinterpret_cast<const float4 *>(X);
  float acc = 0.f;
  const int64_t nb = (n + 31) / 32;
  for (int64_t b = w0; b < nb; b += ws) {
    const int64_t e = b * 32 + lane;
    const int my = e < n ? __ldg(&idx[e]) : -1;
#pragma unroll
    for (int j0 = 0; j0 < 32; j0 += 8) {
      float4 g[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = __shfl_sync(0xffffffffu, my, j0 + 2 * u + hb);
        g[u] = (act && c >= 0) ? __ldg(&X4[(int64_t)c * ld4 + q]) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc += (g[u].x + g[u].y) + (g[u].z + g[u].w);
    }
  }
  if (acc == -1.f) sink[0] = acc;  // never true (nonnegative data): keeps the loads
}

}  // namespace
}  // namespace aunmf

extern "C" int aunmf_probe_gather(const int32_t *idx, int64_t n, const float *X, int64_t rows,
                                  int k, int64_t ld, float *sink, void *stream) {
  using namespace aunmf;
  if (!idx || !X || !sink || n < 0 || rows < 1 || k < 1 || k > 64 || ld < k || ld % 4 != 0)
    return AUNMF_E_INVAL;
  if (reinterpret_cast<uintptr_t>(X) % 16 != 0) return AUNMF_E_INVAL;
  if (n == 0) return AUNMF_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 152;
  const int64_t warps = (n + 31) / 32;
  int64_t nb = (warps + kProbeWarps - 1) / kProbeWarps;
  if (nb > (int64_t)sms * 16) nb = (int64_t)sms * 16;
  k_probe_gather<<<(unsigned)nb, kProbeThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      idx, n, X, k, ld / 4, sink);
  g_launches += 1;
  return cudaGetLastError() == cudaSuccess ? AUNMF_OK : AUNMF_E_CUDA;
}
