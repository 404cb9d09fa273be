// batched.cuh -- descriptors and launchers of the batched AU-NMF kernels
// (k_batched.cu), used by aunmf_run_batched.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace aunmf {
namespace batched {

constexpr int kMaxK = 64;  // rank limit of batched problems (BPP's limit)

// One problem of the batch: its input, factors and workspace (device
// pointers; the descriptor array lives in device memory).
struct BInst {
  int64_t m, n;
  int k;
  int nr;                 // residual partial slots
  const float *A;         // m x n, lda
  int64_t lda;
  float *W;               // m x k (the caller's output array)
  float *Ht, *PW, *PHt;   // n x k, m x k, n x k
  double *GH, *GW;        // k x k, FP64 (products formed exactly, FP64 sums)
  double *gpart_w, *gpart_h;
  int ngw, ngh;           // Gram partial slots for the m rows of W / n rows of Ht
  void *Ax, *At, *Hk, *Wt;  // rounded copies of A, A^T; split factor copies
  int64_t ldx, ldat, ldh, ldw;
  double *Q;              // G^{-1} of the current update as an FP32 pair (2 k^2 floats)
  double *Lq;             // its Cholesky factor (k x k), 1 / diag (k), column sums of |Q| (k)
  int *q_ok;              // [0]: Q usable; [1]: the factorisation succeeded
  uint8_t *redo;          // rows flagged for the direct BPP fallback
  double *n2a;            // {||A||^2, 2 <round(A) - A, A>}
  double *rpart;          // residual partials
  double *relres;         // per-iteration relative residual (device)
};

// A range of one problem's rows (or elements) handled by one block.
struct Item {
  int p;
  int chunk;  // partial slot of the range
  int64_t r0, r1;
};

cudaError_t launch_prepare(const BInst *P, const int64_t *tile_prefix, int count, int64_t tiles,
                           bool bf16, double *tile_sq, cudaStream_t s);
cudaError_t launch_init(const BInst *P, const float *const *H0, const int64_t *row_prefix,
                        int count, int64_t total, cudaStream_t s);
cudaError_t launch_finish(const BInst *P, float *const *H, const int64_t *row_prefix, int count,
                          int64_t total, cudaStream_t s);
cudaError_t launch_split_transpose(const BInst *P, const int64_t *tile_prefix, int count,
                                   int64_t tiles, int side, bool bf16, cudaStream_t s);
cudaError_t launch_gram(const BInst *P, const Item *items, int nitems, int count, int side,
                        cudaStream_t s);
// cold: every solve starts from x = 0 (aunmf_options.bpp_cold_start)
cudaError_t launch_bpp(const BInst *P, const Item *items, int nitems, int count, int side,
                       int kmax, int max_piv, int cold, DevCounters *ctr, int wpb, cudaStream_t s);
int bpp_max_warps(int kmax);
cudaError_t launch_relres(const BInst *P, const Item *items, int nitems, int count,
                          DevCounters *ctr, int iters, cudaStream_t s);

}  // namespace batched
}  // namespace aunmf
