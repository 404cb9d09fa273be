// tc.cuh -- tensor-core (tcgen05) products with A: host-side launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace aunmf {
namespace tc {

// AUNMF_OK if the tensor-core path takes (m, n, k, prec), else a status.
int check(int64_t m, int64_t n, int64_t lda, int k, int prec, const float *A);
// Leading dimension (elements) of the library's K-major copies: a multiple of 8
// so that every row starts on a 16-byte boundary for TMA (FP32 and BF16).
int64_t copy_ld(int64_t cols);
// Elements of a factor copy rows x k stored as (up to) 2k x copy_ld(rows).
size_t factor_elems(int64_t rows, int k);
// Elements of the split-K partial buffer for an M x k product.
size_t parts_elems(int64_t M, int k);
// MMA N for rank k, and the number of K splits for an M x K product.
int bn_for(int k);
int splits_for(int64_t M, int64_t K, bool bf16);

// out (cols x rows, ld ldo) = in (rows x cols, ld ldi)^T rounded to nearest
// TF32 (stored as FP32) or BF16.
cudaError_t launch_transpose_to(const float *in, int64_t rows, int64_t cols, int64_t ldi, void *out,
                                int64_t ldo, bool bf16, cudaStream_t s);
// One pass over A: X = round(A) (m x n, ldx), Xt = round(A)^T (n x m, ldxt),
// norm2[0] = sum a_ij^2 and norm2[1] = 2 sum a_ij (round(a_ij) - a_ij) (FP64),
// via 2 x prepare_blocks() partials in part.
int prepare_blocks();
cudaError_t launch_prepare(const float *A, int64_t m, int64_t n, int64_t lda, void *X, int64_t ldx,
                           void *Xt, int64_t ldxt, bool bf16, double *part, double *norm2,
                           cudaStream_t s);
// out (m x n, ld ldo) = A (m x n, lda) rounded to nearest TF32 (stored as
// FP32) or BF16.  The transposed copies round the same way.
cudaError_t launch_round_copy(const float *A, int64_t m, int64_t n, int64_t lda, void *out,
                              int64_t ldo, bool bf16, cudaStream_t s);
// parts[s] (M x k) = X (M x K, ldx) * F (k x K)^T over the s-th K split, s < S;
// X, Y FP32 (TF32 MMA) or BF16.  split == false: Y = F (k x K, ldy);
// split == true: Y holds 2k rows, hi/lo of F's row i at rows 2i, 2i+1
// (launch_split_transpose), and the kernel adds each pair.  S == 1 writes the
// product itself.  scratch: scratch_elems() floats for the partial sums of
// wide products (k > ~160), or null (they are then added into parts).
size_t scratch_elems();
cudaError_t launch_gemm(const void *X, int64_t M, int64_t K, int64_t ldx, const void *Y, int k,
                        int64_t ldy, bool split, bool bf16, float *parts, int S, float *scratch,
                        int *err, cudaStream_t s);
// Y (2k x rows, ld ldo) = [hi; lo] rows of in (rows x k, ld ldi)^T, rounded to
// nearest TF32 (FP32 containers) or BF16: hi = round(x), lo = round(x - hi).
cudaError_t launch_split_transpose(const float *in, int64_t rows, int k, int64_t ldi, void *out,
                                   int64_t ldo, bool bf16, cudaStream_t s);
// Grouped products (one launch for many problems, e.g. a batch of NMF
// instances): each problem's descriptor is filled on the host into a
// problem_bytes()-sized slot (64-byte aligned) of a host array that the
// caller copies to device memory; unit0 numbers the problems' work units
// consecutively (no K splits: each problem writes C directly).
size_t problem_bytes();
bool fill_group_problem(void *host_dst, const void *X, int64_t M, int64_t K, int64_t ldx,
                        const void *Y, int k, int64_t ldy, bool split, bool bf16, float *C,
                        int64_t unit0, int64_t *units, int *BN);
// nstages: pipeline stages of the shared-memory ring (>= 2; 0 or above the
// most that fit: as many as fit, the default).  group_max_stages: that most
// (0 if the group cannot launch).
cudaError_t launch_gemm_group(const void *dev_problems, const void *host_first, int nprob,
                              int64_t units, int BNmax, bool bf16, int *err, cudaStream_t s,
                              int nstages = 0);
int group_max_stages(const void *host_first, int nprob, int64_t units, int BNmax);
// P = sum over s of parts[s] (len elements each), s ascending.
cudaError_t launch_sum_splits(const float *parts, int S, int64_t len, float *P, cudaStream_t s);

}  // namespace tc
}  // namespace aunmf
