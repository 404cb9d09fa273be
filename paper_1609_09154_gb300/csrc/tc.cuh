// tc.cuh -- tensor-core (tcgen05) products with A: declarations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace aunmf {
namespace tc {

// AUNMF_OK if the tensor-core path takes (m, n, lda, k, prec, A), else a status.
int check(int64_t m, int64_t n, int64_t lda, int k, int prec, const float *A);
// Elements of a BF16 factor copy (rows x k, padded as the kernels need).
size_t factor_elems(int64_t rows, int k);
// BF16 copy of A (m x n, lda) into out (m x n, ld n).
cudaError_t launch_to_bf16(const float *A, int64_t m, int64_t n, int64_t lda, uint16_t *out,
                           cudaStream_t s);
// P_W (m x k) = A Ht, P_Ht (n x k) = A^T W on tensor cores.
cudaError_t launch_aht_tc(const float *A, const uint16_t *Abf, int64_t m, int64_t n, int64_t lda,
                          const float *Ht, uint16_t *Htbf, int k, int prec, float *P,
                          cudaStream_t s);
cudaError_t launch_wta_tc(const float *A, const uint16_t *Abf, int64_t m, int64_t n, int64_t lda,
                          const float *W, uint16_t *Wbf, int k, int prec, float *P,
                          cudaStream_t s);

}  // namespace tc
}  // namespace aunmf
