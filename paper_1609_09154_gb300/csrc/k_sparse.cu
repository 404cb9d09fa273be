// k_sparse.cu -- sparse (CSR) products (placeholder until the SpMM kernels land).
#include "internal.cuh"

namespace aunmf {
cudaError_t launch_aht_csr(const int64_t *, const int32_t *, const float *, int64_t,
                           const float *, int, float *, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_wta_csr(const int64_t *, const int32_t *, const float *, int64_t, int64_t,
                           const float *, int, float *, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace aunmf
