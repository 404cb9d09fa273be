// internal.cuh -- declarations shared by the library's translation units.
// Nothing here is part of the C ABI (that is include/aunmf.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/aunmf.h"

namespace aunmf {

constexpr int kWarp = 32;

// Kernels enqueued by this thread since the counter was last read; every
// launcher adds the number of kernels it launches.
extern thread_local long long g_launches;

// Bounded device waits and the test hook that makes them run out
// (aunmf_test_inject).  site(): the injection now set (AUNMF_INJECT_*);
// wait_cycles(): SM clocks a bounded wait may spin before it gives up,
// ~2 s unless the hook set a shorter limit.
namespace fault {
constexpr long long kDefaultWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
int site();
long long wait_cycles();
}  // namespace fault

// Optional input checks (aunmf_options.validate): each ORs its bit into
// *flag.  Values: an entry of A negative, NaN or infinite; structure: a CSR
// row pointer out of order or range, or a column index out of [0, n) or not
// increasing within its row; factors: an entry of W0 or H0 negative, NaN or
// infinite.
constexpr int kValidateValues = 1, kValidateStructure = 2, kValidateFactors = 4;
cudaError_t launch_validate_dense(const float *A, int64_t m, int64_t n, int64_t lda, int *flag,
                                  cudaStream_t s);
cudaError_t launch_validate_vec(const float *v, int64_t len, int bit, int *flag, cudaStream_t s);
cudaError_t launch_validate_csr(const int64_t *rowptr, const int32_t *colidx, const float *val,
                                int64_t m, int64_t n, int64_t nnz, int *flag, cudaStream_t s);

// Checked build (-DAUNMF_CHECK, libaunmf_check.so): AUNMF_BOUND(ok, site)
// tests an index condition in device code.  When it fails it records `site`
// (an AUNMF_CHECK_* code; the first one per translation unit) in a device
// word and yields false, so the caller skips the access instead of
// faulting.  In the normal build it is the constant true, and `ok` is not
// evaluated.  Each unit registers a reader of its word at load time;
// aunmf_check_status() calls them (no readers: the normal build).
void register_check_reader(int (*reader)());
#ifdef AUNMF_CHECK
namespace {
__device__ int g_check_site;
__device__ __noinline__ bool check_fail(int site) {
  atomicCAS(&g_check_site, 0, site);
  return false;
}
int read_check_site() {
  int v = 0;
  const int z = 0;
  if (cudaMemcpyFromSymbol(&v, g_check_site, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaMemcpyToSymbol(g_check_site, &z, sizeof(int));
  return v;
}
[[maybe_unused]] const int g_check_registered = (register_check_reader(read_check_site), 0);
}  // namespace
#define AUNMF_BOUND(ok, site) ((ok) ? true : check_fail(site))
#else
#define AUNMF_BOUND(ok, site) true
#endif

// Device-side error/diagnostic counters, one block of int64 in the workspace.
struct DevCounters {
  long long bpp_pivots;
  long long bpp_nonconv;
  long long bpp_numeric;
  long long nonfinite;
  long long iter;      // index of the next relres slot
  long long bpp_redo;  // right-hand sides re-solved by the direct fallback
  long long pad[2];
};

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `s` and return cudaGetLastError().

// hi + lo += a * b with the product formed exactly (FMA gives its rounding
// error) and the sum's rounding error kept (Knuth's two-sum): a pair of FP32
// numbers carrying ~48 bits, at a few FP32 operations per term.
// The _rn intrinsics keep the compiler from contracting a product and a sum
// into one FMA, which would break the error terms.
__device__ __forceinline__ void two_fma_acc(float a, float b, float &hi, float &lo) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float z = __fsub_rn(s, hi);
  const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(p, z));
  lo = __fadd_rn(lo, __fadd_rn(t, e));
  hi = s;
}

// Gram: partial[b] = sum over rows of block b of X^T X (X rows x k, row-major,
// leading dimension ldx); then G = sum_b partial[b] in FP64, fixed order.
// err: the device error flag for the bounded waits of the wide-rank form
// (k >= 96, which runs the TMA-fed product kernel on X^T X); null keeps the
// k_gram_part form.
cudaError_t launch_gram(const float *X, int64_t rows, int k, int64_t ldx, float *G,
                        float *partials, int max_blocks, cudaStream_t s, int *err = nullptr);
int gram_partial_blocks(int64_t rows, int max_blocks);
// The same Gram with every product formed exactly in FP64 (FP32 x FP32 fits a
// double) and summed in FP64: G64 (k x k, FP64) for the BPP solves, and G32 =
// G64 rounded to FP32 (may be null).  partials: max_blocks * k * k doubles.
cudaError_t launch_gram_d(const float *X, int64_t rows, int k, int64_t ldx, double *G64,
                          float *G32, double *partials, int max_blocks, cudaStream_t s);
// G64 = G32 widened (k x k).
cudaError_t launch_widen(const float *G32, int k, double *G64, cudaStream_t s);

// SIMT FP32 products.
//   aht: P_W (m x k, ld k) = A (m x n, lda) * Ht (n x k, ld k)
//   wta: P_Ht (n x k, ld k) = A^T (n x m) * W (m x k, ld k)
// parts: simt_parts_bytes(max(m, n), k) bytes for the K-split partials and a
// copy of the factor with rows padded to 4 floats (null: no split, and the
// TMA-fed form is not used).  err: the device error flag that the TMA-fed
// form's bounded waits raise (null: that form is not used).
size_t simt_parts_bytes(int64_t rows, int k);
cudaError_t launch_aht_simt(const float *A, int64_t m, int64_t n, int64_t lda, const float *Ht,
                            int k, float *P, float *parts, int *err, cudaStream_t s);
cudaError_t launch_wta_simt(const float *A, int64_t m, int64_t n, int64_t lda, const float *W,
                            int k, float *P, float *parts, int *err, cudaStream_t s);

// Sparse products (FP32).  P_W (m x k) = A Ht from CSR; P_Ht (n x k) = A^T W
// from the CSC form (colptr[n+1], rowidx[nnz], cval[nnz]) built by
// launch_csr_to_csc (scratch: csc_scratch_bytes(n, nnz) bytes).
// Rows (of the CSR, or of the CSC: columns of A) with more than kLongRowNz
// nonzeros, which the products split into chunks over many warps: the sorted
// row list, its chunk prefix, and chunk partial sums (nchunks x k floats);
// nlong = 0: none (or lr == null).
constexpr int64_t kLongRowNz = 4096;
struct SpLongRows {
  int64_t nlong = 0, nchunks = 0;
  const int64_t *row = nullptr;
  const int64_t *chunk0 = nullptr;
  float *part = nullptr;
};
// (n, m and nnz bound the gathered indices in the checked build.)
cudaError_t launch_aht_csr(const int64_t *rowptr, const int32_t *colidx, const float *val,
                           int64_t m, int64_t n, int64_t nnz, const float *Ht, int k, float *P,
                           const SpLongRows *lr, cudaStream_t s);
cudaError_t launch_wta_csc(const int64_t *colptr, const int32_t *rowidx, const float *cval,
                           int64_t n, int64_t m, int64_t nnz, const float *W, int k, float *P,
                           const SpLongRows *lr, cudaStream_t s);
// list: long_rows_capacity(nnz) int64; chunk0: capacity + 1 int64; count: one
// counter.  Fills lr (its part stays null: the caller allocates nchunks x k
// floats).  Synchronises the stream.
int64_t long_rows_capacity(int64_t nnz);
cudaError_t find_long_rows(const int64_t *ptr, int64_t rows, int64_t nnz, int64_t *list,
                           int64_t *chunk0, unsigned long long *count, SpLongRows *lr,
                           cudaStream_t s);
size_t csc_scratch_bytes(int64_t n, int64_t nnz);
cudaError_t launch_csr_to_csc(const int64_t *rowptr, const int32_t *colidx, const float *val,
                              int64_t m, int64_t n, int64_t nnz, int64_t *colptr, int32_t *rowidx,
                              float *cval, void *scratch, cudaStream_t s);

// Transpose: out (cols x rows) = in (rows x cols)^T, both row-major, dense ld.
cudaError_t launch_transpose(const float *in, int64_t rows, int64_t cols, float *out,
                             cudaStream_t s);

// Local updates on row-major X (rows x k) given P (rows x k) and G (k x k).
cudaError_t launch_mu(float *X, const float *P, const float *G, int64_t rows, int k, float eps,
                      cudaStream_t s);
// unit: Eq. halsupdate as printed (no division by G_ii).
cudaError_t launch_hals(float *X, const float *P, const float *G, int64_t rows, int k,
                        cudaStream_t s, bool unit = false);
// The W sweep of Eq. halsupdate as printed (no division by (HH^T)_ii, each
// column normalised before the next is updated), one cooperative launch.
// part: 2 * printed_sweep_blocks() doubles; bar: one counter (zeroed here);
// err: set when a grid barrier waits too long.
int printed_sweep_blocks();
cudaError_t launch_hals_w_printed(float *W, const float *P, const float *G, int64_t rows, int k,
                                  double *part, unsigned *bar, int *err, cudaStream_t s);
// Projected gradient of 0.5 ||A - WH||^2: pgrad_blocks() FP64 partials of
// sum p^2 over rows of X, p = (X G - P)_rj where X_rj > 0, else min(0, .);
// then out[ctr->iter] = sqrt(sum of n partials).
int pgrad_blocks();
cudaError_t launch_pgrad_partial(const float *X, const float *P, const float *G, int64_t rows,
                                 int k, double *part, cudaStream_t s);
cudaError_t launch_pgrad_final(const double *part, int n, const DevCounters *ctr, double *out,
                               cudaStream_t s);
// HALS normalisation: s_i = sqrt(GW_ii); X(:, i) /= s_i; Y(:, i) *= s_i (Y = Ht,
// may be null, rows_y rows); GW_ij /= s_i s_j.  Zero norms leave column i as is.
cudaError_t launch_hals_normalise(float *X, int64_t rows_x, float *Y, int64_t rows_y, float *GW,
                                  int k, cudaStream_t s);
// BPP: X(r, :) = argmin_{x>=0} ||C x - b|| given G = C^T C (FP64) and
// R(r, :) = C^T b, in FP64.  warm != 0 starts each row from the support of
// X's current row.  scratch: bpp_scratch_bytes(k, rows) bytes of device
// memory (G^{-1} and a per-row flag for the direct fallback).
size_t bpp_scratch_bytes(int k, int64_t rows);
cudaError_t launch_bpp(const double *G, const float *R, int64_t rows, int k, float *X,
                       int max_pivots, int warm, DevCounters *ctr, void *scratch, cudaStream_t s);

// Reductions for the relative residual.
// sum of squares of A (dense) or of val (CSR) into *out (device double).
cudaError_t launch_norm2(const float *A, int64_t m, int64_t n, int64_t lda, double *partials,
                         int nparts, double *out, cudaStream_t s);
cudaError_t launch_norm2_vec(const float *v, int64_t len, double *partials, int nparts,
                             double *out, cudaStream_t s);
// relres[ctr->iter++] = sqrt(max(0, n2a - 2 <P, Ht> + <GW, GH>) / n2a); also
// copies the value to *last.
cudaError_t launch_relres(const float *P, const float *Ht, int64_t len, const float *GW,
                          const float *GH, int k, const double *n2a, double *partials,
                          int nparts, double *relres_dev, DevCounters *ctr, double *last,
                          cudaStream_t s);

// 0.5 ||A - W H||^2 = 0.5 (n2a - 2 <P, Ht> + <GW, GH>) into *loss (device).
cudaError_t launch_loss(const float *P, const float *Ht, int64_t len, const float *GW,
                        const float *GH, int k, const double *n2a, double *partials, int nparts,
                        double *loss, cudaStream_t s);
// out = g (X G - P), X and P rows x k, G k x k, g = *gscale (NULL: 1).
cudaError_t launch_xg_minus_p(const float *X, const float *P, const float *G, int64_t rows, int k,
                              const float *gscale, float *out, cudaStream_t s);

// Copy with a different leading dimension (rows x cols).
cudaError_t launch_copy2d(const float *in, int64_t ld_in, float *out, int64_t ld_out,
                          int64_t rows, int64_t cols, cudaStream_t s);

}  // namespace aunmf
