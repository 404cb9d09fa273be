// k_csc.cu -- the CSC form of a sparse A (CSR in, CSC out), built once per
// run for the W^T A product (Sec. 5.2.1).
//
// The nonzeros' positions are sorted by column with a stable radix sort
// (CUB); the CSR order is row-major, so the entries of every column come out
// in row order, whatever the column's length.  Row indices and values are
// then gathered through the sorted positions, and the column pointers are
// read off the sorted keys (the first position of each column), so no step
// uses atomics: a column with a million entries (a power-law hub) costs no
// more than a million columns of one.
#include <cub/device/device_radix_sort.cuh>

#include "internal.cuh"

namespace aunmf {
namespace {

constexpr int kCscThreads = 256;

int grid_for(int64_t items, int per_sm) {
  int64_t nb = (items + kCscThreads - 1) / kCscThreads;
  if (nb > 152LL * per_sm) nb = 152LL * per_sm;
  return nb < 1 ? 1 : (int)nb;
}

// rows[e] = r for the nonzeros e of row r (a warp per row).
__global__ void k_rows_of(const int64_t *__restrict__ rowptr, int64_t m, int64_t nnz,
                          int32_t *__restrict__ rows) {
  (void)nnz;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t ws = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < m; r += ws)
    for (int64_t e = rowptr[r] + lane; e < rowptr[r + 1]; e += 32)
      if (AUNMF_BOUND(e >= 0 && e < nnz, AUNMF_CHECK_CSC)) rows[e] = (int32_t)r;
}

__global__ void k_iota(int32_t *__restrict__ p, int64_t nnz) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    p[e] = (int32_t)e;
}

// rowidx[q] = rows[pos[q]], cval[q] = val[pos[q]]; colptr[c] = the first q
// with key[q] >= c (c = 0..n): position q starts the columns key[q-1]+1 ..
// key[q] (from 0 at q = 0), and colptr[c] = nnz for the columns after the
// last key.
__global__ void k_csc_fill(const int32_t *__restrict__ key, const int32_t *__restrict__ pos,
                           const int32_t *__restrict__ rows, const float *__restrict__ val,
                           int64_t nnz, int64_t n, int64_t *__restrict__ colptr,
                           int32_t *__restrict__ rowidx, float *__restrict__ cval) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = pos[q];
    const int64_t c1 = key[q];
    if (!AUNMF_BOUND(e >= 0 && e < nnz && c1 >= 0 && c1 < n, AUNMF_CHECK_CSC)) continue;
    rowidx[q] = rows[e];
    cval[q] = val[e];
    const int64_t c0 = q == 0 ? 0 : (int64_t)key[q - 1] + 1;
    for (int64_t c = c0; c <= c1; ++c) colptr[c] = q;
  }
}

__global__ void k_colptr_tail(const int32_t *__restrict__ key, int64_t nnz, int64_t n,
                              int64_t *__restrict__ colptr) {
  const int64_t c0 = nnz > 0 ? (int64_t)key[nnz - 1] + 1 : 0;
  for (int64_t c = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= n;
       c += (int64_t)gridDim.x * blockDim.x)
    colptr[c] = nnz;
}

int key_bits(int64_t n) {
  int b = 1;
  while (b < 31 && (1LL << b) < n) ++b;
  return b;
}

size_t sort_temp_bytes(int64_t nnz, int64_t n) {
  size_t t = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, t, static_cast<const int32_t *>(nullptr),
                                  static_cast<int32_t *>(nullptr),
                                  static_cast<const int32_t *>(nullptr),
                                  static_cast<int32_t *>(nullptr), (int)nnz, 0, key_bits(n));
  return t;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Scratch: sorted keys, positions in and out, the row of every nonzero, and
// the sort's temporary storage (4 nnz int32 arrays + the CUB buffer).
size_t csc_scratch_bytes(int64_t n, int64_t nnz) {
  return 4 * al256(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1)) + al256(sort_temp_bytes(nnz, n)) +
         256;
}

cudaError_t launch_csr_to_csc(const int64_t *rowptr, const int32_t *colidx, const float *val,
                              int64_t m, int64_t n, int64_t nnz, int64_t *colptr, int32_t *rowidx,
                              float *cval, void *scratch, cudaStream_t s) {
  if (nnz > 0x7fffffffLL || n > 0x7fffffffLL) return cudaErrorInvalidValue;
  char *p = static_cast<char *>(scratch);
  const size_t arr = al256(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  int32_t *key = reinterpret_cast<int32_t *>(p);
  int32_t *pos_in = reinterpret_cast<int32_t *>(p + arr);
  int32_t *pos = reinterpret_cast<int32_t *>(p + 2 * arr);
  int32_t *rows = reinterpret_cast<int32_t *>(p + 3 * arr);
  void *temp = p + 4 * arr;
  size_t temp_bytes = sort_temp_bytes(nnz, n);
  if (nnz > 0) {
    k_iota<<<grid_for(nnz, 16), kCscThreads, 0, s>>>(pos_in, nnz);
    k_rows_of<<<grid_for(m * 32, 16), kCscThreads, 0, s>>>(rowptr, m, nnz, rows);
    cudaError_t e = cub::DeviceRadixSort::SortPairs(temp, temp_bytes, colidx, key, pos_in, pos,
                                                    (int)nnz, 0, key_bits(n), s);
    if (e != cudaSuccess) return e;
    k_csc_fill<<<grid_for(nnz, 16), kCscThreads, 0, s>>>(key, pos, rows, val, nnz, n, colptr,
                                                          rowidx, cval);
    g_launches += 3;
  }
  k_colptr_tail<<<grid_for(n + 1, 4), kCscThreads, 0, s>>>(key, nnz, n, colptr);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace aunmf
