// k_sparse.cu -- sparse A (Sec. 5.2.1: the products cost 4 nnz(A) k flops).
//
//   P_W  = A Ht     : CSR SpMM, one warp per row of A; lane l accumulates the
//                     entries j = l, l+32, ... of the output row while the warp
//                     walks the row's nonzeros and gathers rows of Ht (n x k).
//   P_Ht = A^T W    : the same kernel over the CSC form of A (the CSR form of
//                     A^T), gathering rows of W (m x k).
// The CSC copy is built once per run on the device: column counts, an
// exclusive scan, a scatter, and a ranking pass that orders every column's
// entries by row index (so the result does not depend on the scatter order).
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

// ---------------------------------------------------------------- CSR -> CSC
__global__ void k_count_cols(const int32_t *__restrict__ idx, int64_t nnz, int *__restrict__ cnt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[idx[e]], 1);
}

// Exclusive scan of cnt[0..n) into ptr[0..n] (single block, chunked).
__global__ void k_scan(const int *__restrict__ cnt, int64_t n, int64_t *__restrict__ ptr) {
  __shared__ long long part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t chunk = (n + T - 1) / T;
  const int64_t b = (int64_t)t * chunk, e = min(n, b + chunk);
  long long s = 0;
  for (int64_t i = b; i < e; ++i) s += cnt[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    long long run = 0;
    for (int i = 0; i < T; ++i) {
      const long long v = part[i];
      part[i] = run;
      run += v;
    }
  }
  __syncthreads();
  long long run = part[t];
  for (int64_t i = b; i < e; ++i) {
    ptr[i] = run;
    run += cnt[i];
  }
  if (e == n && b < n) ptr[n] = run;
  if (n == 0 && t == 0) ptr[0] = 0;
}

// Scatter every nonzero (r, c, v) to a free slot of column c (any order).
__global__ void k_scatter(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ idx,
                          const float *__restrict__ val, int64_t m,
                          const int64_t *__restrict__ colptr, int *__restrict__ cursor,
                          int32_t *__restrict__ rowidx, float *__restrict__ cval) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t ws = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < m; r += ws)
    for (int64_t e = rowptr[r] + lane; e < rowptr[r + 1]; e += 32) {
      const int c = idx[e];
      const int64_t pos = colptr[c] + atomicAdd(&cursor[c], 1);
      rowidx[pos] = (int32_t)r;
      cval[pos] = val[e];
    }
}

// Order each column's entries by row: the entry with row index r moves to
// slot (number of entries of the column with a smaller row index).  Row
// indices within a column are distinct.  One warp per column.
__global__ void k_rank_cols(const int64_t *__restrict__ colptr, int64_t n,
                            const int32_t *__restrict__ rin, const float *__restrict__ vin,
                            int32_t *__restrict__ rout, float *__restrict__ vout) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t ws = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = w0; c < n; c += ws) {
    const int64_t b = colptr[c], e = colptr[c + 1];
    for (int64_t i = b + lane; i < e; i += 32) {
      const int32_t ri = rin[i];
      int64_t rank = 0;
      for (int64_t j = b; j < e; ++j) rank += (rin[j] < ri);
      rout[b + rank] = ri;
      vout[b + rank] = vin[i];
    }
  }
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

size_t csc_scratch_bytes(int64_t n, int64_t nnz) {
  return sizeof(int) * (size_t)n + sizeof(int32_t) * (size_t)nnz + sizeof(float) * (size_t)nnz + 256;
}

cudaError_t launch_csr_to_csc(const int64_t *rowptr, const int32_t *colidx, const float *val,
                              int64_t m, int64_t n, int64_t nnz, int64_t *colptr, int32_t *rowidx,
                              float *cval, void *scratch, cudaStream_t s) {
  int *cnt = reinterpret_cast<int *>(scratch);
  int32_t *r_tmp = reinterpret_cast<int32_t *>(cnt + n);
  float *v_tmp = reinterpret_cast<float *>(r_tmp + nnz);
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * n, s);
  if (e != cudaSuccess) return e;
  int64_t nb = (nnz + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  if (nb < 1) nb = 1;
  k_count_cols<<<(unsigned)nb, 256, 0, s>>>(colidx, nnz, cnt);
  k_scan<<<1, 1024, 0, s>>>(cnt, n, colptr);
  e = cudaMemsetAsync(cnt, 0, sizeof(int) * n, s);
  if (e != cudaSuccess) return e;
  int64_t nbw = (m * 32 + 255) / 256;
  if (nbw > 152 * 16) nbw = 152 * 16;
  if (nbw < 1) nbw = 1;
  k_scatter<<<(unsigned)nbw, 256, 0, s>>>(rowptr, colidx, val, m, colptr, cnt, r_tmp, v_tmp);
  int64_t nbc = (n * 32 + 255) / 256;
  if (nbc > 152 * 16) nbc = 152 * 16;
  if (nbc < 1) nbc = 1;
  k_rank_cols<<<(unsigned)nbc, 256, 0, s>>>(colptr, n, r_tmp, v_tmp, rowidx, cval);
  g_launches += 4;
  return cudaGetLastError();
}

}  // namespace aunmf
