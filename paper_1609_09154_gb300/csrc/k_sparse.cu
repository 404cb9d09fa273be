// k_sparse.cu -- sparse A (Sec. 5.2.1: the products cost 4 nnz(A) k flops).
//
//   P_W  = A Ht     : CSR SpMM, one warp per row of A; lane l accumulates the
//                     entries j = l, l+32, ... of the output row while the warp
//                     walks the row's nonzeros and gathers rows of Ht (n x k).
//   P_Ht = A^T W    : the same kernel over the CSC form of A (the CSR form of
//                     A^T), gathering rows of W (m x k).
// The CSC copy is built once per run on the device (k_csc.cu).
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace aunmf {
namespace {

constexpr int kSpThreads = 256;
constexpr int kSpWarps = kSpThreads / kWarp;
constexpr int64_t kChunkNz = 2048;  // nonzeros per warp on a long row

// acc[t] (lane's entries j = lane + 32 t) += sum over nonzeros e in [e0, e1)
// of val[e] X[idx[e], j]: the warp stages 32 nonzeros in registers, then
// broadcasts them and gathers the k-vectors of X (ncols rows), four at a
// time.  (ncols is read only by the checked build.)
template <int KT>
__device__ __forceinline__ void spmm_range(const int32_t *__restrict__ idx,
                                           const float *__restrict__ val,
                                           const float *__restrict__ X, int64_t ncols, int k,
                                           int64_t e0, int64_t e1, float (&acc)[KT], int lane) {
  (void)ncols;
  for (int64_t eb = e0; eb < e1; eb += 32) {
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
          g[u][t] = (col < k && AUNMF_BOUND((uint64_t)c[u] < (uint64_t)ncols,
                                            AUNMF_CHECK_SPMM_COLUMN))
                        ? __ldg(&X[(int64_t)c[u] * k + col])
                        : 0.f;
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
        if (col < k && AUNMF_BOUND((uint64_t)c < (uint64_t)ncols, AUNMF_CHECK_SPMM_COLUMN))
          acc[t] = fmaf(v, __ldg(&X[(int64_t)c * k + col]), acc[t]);
      }
    }
  }
}

// Y (rows x k) = S (rows x ncols, CSR ptr/idx/val, nnz nonzeros) * X
// (ncols x k), a warp per row.  Rows longer than `skip_above` (> 0) are left
// to the chunked kernels below.
template <int KT>
__global__ void __launch_bounds__(kSpThreads)
    k_spmm(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
           const float *__restrict__ val, int64_t rows, int64_t ncols, int64_t nnz,
           const float *__restrict__ X, int k, float *__restrict__ Y, int64_t skip_above) {
  (void)nnz;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * kSpWarps + (threadIdx.x >> 5);
  const int64_t ws = (int64_t)gridDim.x * kSpWarps;
  for (int64_t r = w0; r < rows; r += ws) {
    const int64_t e0 = ptr[r], e1 = ptr[r + 1];
    if (skip_above > 0 && e1 - e0 > skip_above) continue;
    if (!AUNMF_BOUND(e0 >= 0 && e0 <= e1 && e1 <= nnz, AUNMF_CHECK_SPMM_RANGE)) continue;
    float acc[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) acc[t] = 0.f;
    spmm_range<KT>(idx, val, X, ncols, k, e0, e1, acc, lane);
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int col = lane + 32 * t;
      if (col < k) Y[r * k + col] = acc[t];
    }
  }
}

// Long rows (a power-law hub can hold 10^6 nonzeros, which one warp would
// walk alone while the rest of the GPU idles): chunk c of the sorted list of
// long rows covers kChunkNz nonzeros of row lrow[i], chunk0[i] <= c <
// chunk0[i + 1]; a warp per chunk writes its partial sums, and a warp per
// long row adds its chunks in chunk order (so results do not depend on
// scheduling).
template <int KT>
__global__ void __launch_bounds__(kSpThreads)
    k_spmm_chunks(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                  const float *__restrict__ val, int64_t rows, int64_t ncols, int64_t nnz,
                  const float *__restrict__ X, int k, const int64_t *__restrict__ lrow,
                  const int64_t *__restrict__ chunk0, int64_t nlong, int64_t nchunks,
                  float *__restrict__ part) {
  (void)rows;
  (void)nnz;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * kSpWarps + (threadIdx.x >> 5);
  const int64_t ws = (int64_t)gridDim.x * kSpWarps;
  for (int64_t c = w0; c < nchunks; c += ws) {
    int64_t lo = 0, hi = nlong - 1;  // last i with chunk0[i] <= c
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (chunk0[mid] <= c) lo = mid; else hi = mid - 1;
    }
    const int64_t r = lrow[lo];
    if (!AUNMF_BOUND(r >= 0 && r < rows, AUNMF_CHECK_SPMM_RANGE)) continue;
    const int64_t e0 = ptr[r] + (c - chunk0[lo]) * kChunkNz;
    const int64_t e1 = min(ptr[r + 1], e0 + kChunkNz);
    if (!AUNMF_BOUND(e0 >= 0 && e0 <= e1 && e1 <= nnz, AUNMF_CHECK_SPMM_RANGE)) continue;
    float acc[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) acc[t] = 0.f;
    spmm_range<KT>(idx, val, X, ncols, k, e0, e1, acc, lane);
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int col = lane + 32 * t;
      if (col < k) part[c * k + col] = acc[t];
    }
  }
}

template <int KT>
__global__ void __launch_bounds__(kSpThreads)
    k_spmm_long_sum(const int64_t *__restrict__ lrow, const int64_t *__restrict__ chunk0,
                    int64_t nlong, const float *__restrict__ part, int k, float *__restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * kSpWarps + (threadIdx.x >> 5);
  const int64_t ws = (int64_t)gridDim.x * kSpWarps;
  for (int64_t i = w0; i < nlong; i += ws) {
    float acc[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) acc[t] = 0.f;
    for (int64_t c = chunk0[i]; c < chunk0[i + 1]; ++c)
#pragma unroll
      for (int t = 0; t < KT; ++t) {
        const int col = lane + 32 * t;
        if (col < k) acc[t] += part[c * k + col];
      }
    const int64_t r = lrow[i];
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int col = lane + 32 * t;
      if (col < k) Y[r * k + col] = acc[t];
    }
  }
}

// len[i] = nonzeros of row list[i].
__global__ void k_long_lens(const int64_t *__restrict__ ptr, const int64_t *__restrict__ list,
                            int64_t n, int64_t *__restrict__ len) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    len[i] = ptr[list[i] + 1] - ptr[list[i]];
}

// Appends the rows longer than thr to list (unordered; the caller sorts).
__global__ void k_find_long(const int64_t *__restrict__ ptr, int64_t rows, int64_t thr,
                            int64_t *__restrict__ list, unsigned long long *count,
                            int64_t capacity) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x)
    if (ptr[r + 1] - ptr[r] > thr) {
      const unsigned long long at = atomicAdd(count, 1ull);
      if ((int64_t)at < capacity) list[at] = r;
    }
}

int sp_blocks(int64_t warps) {
  int64_t nb = (warps + kSpWarps - 1) / kSpWarps;
  if (nb > 152 * 16) nb = 152 * 16;
  return nb < 1 ? 1 : (int)nb;
}

#define AUNMF_SP_SWITCH(KTV, CALL) \
  switch (KTV) {                   \
    case 1: CALL(1); break;        \
    case 2: CALL(2); break;        \
    case 3: CALL(3); break;        \
    case 4: CALL(4); break;        \
    case 5: case 6: case 7:        \
    case 8: CALL(8); break;        \
    default: CALL(16); break;      \
  }

cudaError_t spmm(const int64_t *ptr, const int32_t *idx, const float *val, int64_t rows,
                 int64_t ncols, int64_t nnz, const float *X, int k, float *Y,
                 const SpLongRows *lr, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  const int kt = (k + 31) / 32;
  const bool split = lr && lr->nlong > 0;
  const int64_t skip = split ? kLongRowNz : 0;
  const int nb = sp_blocks(rows);
#define AUNMF_SP_MAIN(KT) \
  k_spmm<KT><<<nb, kSpThreads, 0, s>>>(ptr, idx, val, rows, ncols, nnz, X, k, Y, skip)
  AUNMF_SP_SWITCH(kt, AUNMF_SP_MAIN)
#undef AUNMF_SP_MAIN
  g_launches += 1;
  if (split) {
    const int nbc = sp_blocks(lr->nchunks), nbl = sp_blocks(lr->nlong);
#define AUNMF_SP_CH(KT)                                                                  \
  k_spmm_chunks<KT><<<nbc, kSpThreads, 0, s>>>(ptr, idx, val, rows, ncols, nnz, X, k,      \
                                               lr->row, lr->chunk0, lr->nlong, lr->nchunks, \
                                               lr->part);                                \
  k_spmm_long_sum<KT><<<nbl, kSpThreads, 0, s>>>(lr->row, lr->chunk0, lr->nlong, lr->part, k, Y)
    AUNMF_SP_SWITCH(kt, AUNMF_SP_CH)
#undef AUNMF_SP_CH
    g_launches += 2;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_aht_csr(const int64_t *rowptr, const int32_t *colidx, const float *val,
                           int64_t m, int64_t n, int64_t nnz, const float *Ht, int k, float *P,
                           const SpLongRows *lr, cudaStream_t s) {
  return spmm(rowptr, colidx, val, m, n, nnz, Ht, k, P, lr, s);
}

cudaError_t launch_wta_csc(const int64_t *colptr, const int32_t *rowidx, const float *cval,
                           int64_t n, int64_t m, int64_t nnz, const float *W, int k, float *P,
                           const SpLongRows *lr, cudaStream_t s) {
  return spmm(colptr, rowidx, cval, n, m, nnz, W, k, P, lr, s);
}

int64_t long_rows_capacity(int64_t nnz) { return nnz / kLongRowNz + 1; }

// The long rows of a CSR (or CSC) row-pointer array, sorted, with their chunk
// prefix: a device pass finds them (list, count), the host sorts the short
// list and forms the prefix, which goes back to the device.  Synchronises.
cudaError_t find_long_rows(const int64_t *ptr, int64_t rows, int64_t nnz, int64_t *list,
                           int64_t *chunk0, unsigned long long *count, SpLongRows *lr,
                           cudaStream_t s) {
  lr->nlong = lr->nchunks = 0;
  lr->row = list;
  lr->chunk0 = chunk0;
  if (rows == 0) return cudaSuccess;
  const int64_t cap = long_rows_capacity(nnz);
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  int64_t nb = (rows + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  k_find_long<<<(unsigned)nb, 256, 0, s>>>(ptr, rows, kLongRowNz, list, count, cap);
  g_launches += 1;
  unsigned long long n = 0;
  if ((e = cudaMemcpyAsync(&n, count, sizeof(n), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  if (n == 0) return cudaSuccess;
  if ((int64_t)n > cap) return cudaErrorInvalidValue;  // cannot happen: each has > kLongRowNz
  std::vector<int64_t> h(n), len(n), c0(n + 1, 0);
  if ((e = cudaMemcpy(h.data(), list, sizeof(int64_t) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return e;
  std::sort(h.begin(), h.end());
  if ((e = cudaMemcpy(list, h.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  k_long_lens<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ptr, list, (int64_t)n, chunk0);
  g_launches += 1;
  if ((e = cudaMemcpyAsync(len.data(), chunk0, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  for (size_t i = 0; i < n; ++i) c0[i + 1] = c0[i] + (len[i] + kChunkNz - 1) / kChunkNz;
  if ((e = cudaMemcpy(chunk0, c0.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return e;
  lr->nlong = (int64_t)n;
  lr->nchunks = c0[n];
  return cudaSuccess;
}


}  // namespace aunmf
