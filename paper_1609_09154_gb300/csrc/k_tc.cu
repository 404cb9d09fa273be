// k_tc.cu -- tensor-core products (placeholder until the tcgen05 kernels land).
#include "internal.cuh"
#include "tc.cuh"

namespace aunmf {
namespace tc {
int check(int64_t, int64_t, int64_t, int, int, const float *) { return AUNMF_E_UNSUPPORTED; }
size_t factor_elems(int64_t rows, int k) { return (size_t)rows * k; }
cudaError_t launch_to_bf16(const float *, int64_t, int64_t, int64_t, uint16_t *, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_aht_tc(const float *, const uint16_t *, int64_t, int64_t, int64_t,
                          const float *, uint16_t *, int, int, float *, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_wta_tc(const float *, const uint16_t *, int64_t, int64_t, int64_t,
                          const float *, uint16_t *, int, int, float *, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace tc
}  // namespace aunmf
