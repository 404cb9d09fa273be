// k_validate.cu -- optional input checks of a run (aunmf_options.validate):
// the problem of Sec. 2 ("original NMF") is posed for A >= 0, and the
// updates of Sec. 4 keep W, H >= 0 only from a nonnegative start.  Each
// kernel ORs a bit into *flag for what it finds and reads nothing outside
// the arrays it is given; the host reads the flag before any other kernel
// touches the input (a malformed CSR structure must not reach the kernels
// that index with it).
#include <math.h>

#include "internal.cuh"

namespace aunmf {
namespace {

__device__ __forceinline__ bool bad_value(float v) { return !(v >= 0.f) || isinf(v); }

// A (m x n, ld lda) dense: any entry negative, NaN or infinite
__global__ void k_check_dense(const float *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                              int *flag) {
  bool bad = false;
  for (int64_t r = blockIdx.x; r < m; r += gridDim.x)
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) bad |= bad_value(A[r * lda + c]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, kValidateValues);
}

__global__ void k_check_vec(const float *__restrict__ v, int64_t len, int *flag, int bit) {
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (int64_t)gridDim.x * blockDim.x)
    bad |= bad_value(v[e]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, bit);
}

// CSR structure, a warp per row: rowptr[0] = 0, rowptr[m] = nnz,
// rowptr[r] <= rowptr[r + 1] within [0, nnz], and the row's column indices
// in [0, n) and strictly increasing.  A row whose bounds are out of range
// is flagged and its indices are not read.
__global__ void k_check_csr(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                            int64_t m, int64_t n, int64_t nnz, int *flag) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  bool bad = false;
  if (w0 == 0 && lane == 0) bad |= rowptr[0] != 0 || rowptr[m] != nnz;
  for (int64_t r = w0; r < m; r += nw) {
    const int64_t p0 = rowptr[r], p1 = rowptr[r + 1];
    if (p0 < 0 || p1 < p0 || p1 > nnz) {
      bad = true;
      continue;
    }
    for (int64_t e = p0 + lane; e < p1; e += 32) {
      const int32_t c = colidx[e];
      bad |= c < 0 || (int64_t)c >= n;
      if (e > p0) bad |= colidx[e - 1] >= c;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, kValidateStructure);
}

unsigned grid_for(int64_t work) {
  int64_t nb = (work + 255) / 256;
  if (nb > 152 * 8) nb = 152 * 8;
  return (unsigned)(nb > 0 ? nb : 1);
}

}  // namespace

cudaError_t launch_validate_dense(const float *A, int64_t m, int64_t n, int64_t lda, int *flag,
                                  cudaStream_t s) {
  const unsigned nb = (unsigned)(m < 152 * 8 ? m : 152 * 8);
  k_check_dense<<<nb, 256, 0, s>>>(A, m, n, lda, flag);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_validate_vec(const float *v, int64_t len, int bit, int *flag, cudaStream_t s) {
  if (len <= 0) return cudaSuccess;
  k_check_vec<<<grid_for(len), 256, 0, s>>>(v, len, flag, bit);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_validate_csr(const int64_t *rowptr, const int32_t *colidx, const float *val,
                                int64_t m, int64_t n, int64_t nnz, int *flag, cudaStream_t s) {
  k_check_csr<<<grid_for(32 * m), 256, 0, s>>>(rowptr, colidx, m, n, nnz, flag);
  g_launches += 1;
  return launch_validate_vec(val, nnz, kValidateValues, flag, s);
}

}  // namespace aunmf
