// k_sparse.cu -- sparse A (Sec. 5.2.1: the products cost 4 nnz(A) k flops).
//
//   P_W  = A Ht     : CSR SpMM, one warp per row of A; lane l accumulates the
//                     entries j = l, l+32, ... of the output row while the warp
//                     walks the row's nonzeros and gathers rows of Ht (n x k).
//   P_Ht = A^T W    : the same kernel over the CSC form of A (the CSR form of
//                     A^T), gathering rows of W (m x k).
// The CSC copy is built once per run on the device (k_csc.cu).
#include "internal.cuh"

namespace aunmf {
namespace {

constexpr int kSpThreads = 256;
constexpr int kSpWarps = kSpThreads / kWarp;

// Y (rows x k) = S (rows x ncols, CSR ptr/idx/val) * X (ncols x k).
template <int KT>
__global__ void __launch_bounds__(kSpThreads)
    k_spmm(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
           const float *__restrict__ val, int64_t rows, const float *__restrict__ X, int k,
           float *__restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * kSpWarps + (threadIdx.x >> 5);
  const int64_t ws = (int64_t)gridDim.x * kSpWarps;
  for (int64_t r = w0; r < rows; r += ws) {
    float acc[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) acc[t] = 0.f;
    const int64_t e0 = ptr[r], e1 = ptr[r + 1];
    for (int64_t eb = e0; eb < e1; eb += 32) {
      // stage 32 nonzeros of the row in registers, then broadcast them
      const int64_t e = eb + lane;
      const int my_c = e < e1 ? __ldg(&idx[e]) : 0;
      const float my_v = e < e1 ? __ldg(&val[e]) : 0.f;
      const int cnt = (int)min((int64_t)32, e1 - eb);
      int j = 0;
      for (; j + 4 <= cnt; j += 4) {
        int c[4];
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          c[u] = __shfl_sync(0xffffffffu, my_c, j + u);
          v[u] = __shfl_sync(0xffffffffu, my_v, j + u);
        }
        float g[4][KT];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int t = 0; t < KT; ++t) {
            const int col = lane + 32 * t;
            g[u][t] = col < k ? __ldg(&X[(int64_t)c[u] * k + col]) : 0.f;
          }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int t = 0; t < KT; ++t) acc[t] = fmaf(v[u], g[u][t], acc[t]);
      }
      for (; j < cnt; ++j) {
        const int c = __shfl_sync(0xffffffffu, my_c, j);
        const float v = __shfl_sync(0xffffffffu, my_v, j);
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          const int col = lane + 32 * t;
          if (col < k) acc[t] = fmaf(v, __ldg(&X[(int64_t)c * k + col]), acc[t]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int col = lane + 32 * t;
      if (col < k) Y[r * k + col] = acc[t];
    }
  }
}

cudaError_t spmm(const int64_t *ptr, const int32_t *idx, const float *val, int64_t rows,
                 const float *X, int k, float *Y, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  int64_t nb = (rows + kSpWarps - 1) / kSpWarps;
  if (nb > 152 * 16) nb = 152 * 16;
  const int kt = (k + 31) / 32;
  switch (kt) {
    case 1: k_spmm<1><<<(unsigned)nb, kSpThreads, 0, s>>>(ptr, idx, val, rows, X, k, Y); break;
    case 2: k_spmm<2><<<(unsigned)nb, kSpThreads, 0, s>>>(ptr, idx, val, rows, X, k, Y); break;
    case 3: k_spmm<3><<<(unsigned)nb, kSpThreads, 0, s>>>(ptr, idx, val, rows, X, k, Y); break;
    case 4: k_spmm<4><<<(unsigned)nb, kSpThreads, 0, s>>>(ptr, idx, val, rows, X, k, Y); break;
    case 5: case 6: case 7:
    case 8: k_spmm<8><<<(unsigned)nb, kSpThreads, 0, s>>>(ptr, idx, val, rows, X, k, Y); break;
    default: k_spmm<16><<<(unsigned)nb, kSpThreads, 0, s>>>(ptr, idx, val, rows, X, k, Y); break;
  }
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_aht_csr(const int64_t *rowptr, const int32_t *colidx, const float *val,
                           int64_t m, const float *Ht, int k, float *P, cudaStream_t s) {
  return spmm(rowptr, colidx, val, m, Ht, k, P, s);
}

cudaError_t launch_wta_csc(const int64_t *colptr, const int32_t *rowidx, const float *cval,
                           int64_t n, const float *W, int k, float *P, cudaStream_t s) {
  return spmm(colptr, rowidx, cval, n, W, k, P, s);
}


}  // namespace aunmf
