// k_bpp.cu -- batched nonnegative least squares by block principal pivoting
// (Sec. 4.3: SolveBPP(C^T C, C^T B); Eqs. single NLS and KKT), to FP64
// accuracy.
//
// One warp solves one right-hand side r (a row of A H^T for W, a column of
// W^T A for H) against the shared Gram matrix G:
//     x = argmin_{x >= 0} ||C x - b||,   G = C^T C,  r = C^T b.
// Lane l owns the indices j = l and j = l + 32 (k <= 64): its passive flag,
// x_j and y_j = (G x - r)_j (FP32 pairs, ~48 bits) and the tolerance of the
// active-set test (FP32).
//
// Exchange rule (Kim-He-Park / Judice-Pires): V = {passive j: x_j < 0} U
// {active j: y_j < -tau_j}, tau_j = 1e-11 (|r_j| + sum_a |G_jF(a) x_F(a)|)
// (the scale tau_j summed in FP32);
// if |V| shrank, flip all of V and reset the backup counter to 3; else if
// the counter is positive, decrement it and flip all of V; else flip only
// the largest index in V.
//
// Each exchange solves the passive-set normal equations G_FF x_F = r_F with
// a Cholesky factorisation of at most k/2 rows:
//   |F| <= |B|: of G_FF itself;
//   |F| >  |B|: with Q = G^{-1} (computed once per update in FP64, kept as
//               an FP32 pair) and z = Q r (once per right-hand side): the
//               solution with x_B = 0 and y_F = 0 satisfies x = Q (r + y), so
//               Q_BB y_B = -z_B (Cholesky of Q_BB) and x_F = z_F + Q_FB y_B --
//               the block inverse G_FF^{-1} = Q_FF - Q_FB Q_BB^{-1} Q_BF in
//               other words.
// The factorisation is FP32, refined with residuals summed in FP32 pairs
// until a correction is below 2^-30 of x (bpp_core.cuh: solve_mixed); this
// part runs ~60 times more FP32 than FP64 operations per clock.
// The solution of each NLS is unique when G is positive definite (Sec. 4),
// so the starting passive set changes only the work: the run driver starts
// each right-hand side from the support of its previous iterate.  Rows whose
// fast solve cannot finish (an FP32 system too ill-conditioned to refine, or
// a passive set too large for the route) are redone by k_bpp_direct in FP64,
// with full-size Cholesky factorisations of G_FF, warm-started from the row's
// previous iterate (cold if that fails at once).
#include <math.h>

#include "internal.cuh"

#include "bpp_core.cuh"

namespace aunmf {
namespace {
using namespace bpp;

template <int KT>
__global__ void __launch_bounds__(32 * kBppWarps, 1)
    k_bpp(const double *__restrict__ Gd, const float *__restrict__ Qg, const int *__restrict__ q_ok,
          const float *__restrict__ R, int64_t rows, int k, float *__restrict__ X, int warm,
          int max_piv, DevCounters *ctr, uint8_t *__restrict__ redo) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  const BppWarp w = bpp_stage(Gd, Qg, q_ok, k, sm, wib);
  __syncthreads();
  // a run's first iteration (no relres written yet): the previous iterate is
  // the random start (or W = 0), so the solves start from the signs of the
  // unconstrained solution instead of its support
  if (warm == 1 && ctr->iter == 0) warm = 2;
  long long piv_total = 0, nonconv = 0;
  for (int64_t row = (int64_t)blockIdx.x * nwb + wib; row < rows;
       row += (int64_t)gridDim.x * nwb) {
    bool fnum, fcap;
    const int it = bpp_row_fast<KT>(w, R, row, k, X, warm, max_piv, &fnum, &fcap);
    if (lane == 0) redo[row] = fnum ? 1 : 0;
    if (!fnum) {
      piv_total += it;
      nonconv += fcap;
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (piv_total) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->bpp_pivots),
                             (unsigned long long)piv_total);
    if (nonconv) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->bpp_nonconv),
                           (unsigned long long)nonconv);
  }
}

__global__ void __launch_bounds__(256)
    k_chol(const double *__restrict__ Gd, int k, double *__restrict__ L, double *__restrict__ invd,
           int *__restrict__ ok) {
  extern __shared__ double sm[];
  chol_block(Gd, k, L, invd, ok, sm);
}

__global__ void k_inv_cols(const double *__restrict__ L, const double *__restrict__ invd, int k,
                           float *__restrict__ Q, double *__restrict__ colsum) {
  inv_col_warp(L, invd, k, blockIdx.x, Q, colsum);
}

__global__ void k_inv_check(const double *__restrict__ Gd, const double *__restrict__ colsum,
                            int k, const int *__restrict__ ok, int *__restrict__ q_ok) {
  inv_check(Gd, colsum, k, ok, q_ok);
}

template <int KT>
__global__ void __launch_bounds__(256)
    k_bpp_direct(const double *__restrict__ Gd, const float *__restrict__ R, int64_t rows, int k,
                 float *__restrict__ X, int warm, int max_piv, DevCounters *ctr,
                 const uint8_t *__restrict__ redo) {
  extern __shared__ double sm[];
  const int ldl = k | 1;
  double *G = sm;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) G[e] = Gd[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  double *L = sm + (size_t)k * k + (size_t)wib * ((size_t)k * ldl + 3 * (size_t)k);
  double *v = L + (size_t)k * ldl;
  double *rs = v + k;
  int *Fl = reinterpret_cast<int *>(rs + k);
  long long piv_total = 0, nonconv = 0, numeric = 0, redone = 0;
  for (int64_t row = (int64_t)blockIdx.x * nwb + wib; row < rows;
       row += (int64_t)gridDim.x * nwb) {
    if (!redo[row]) continue;
    bool fnum, fcap;
    const int it = bpp_row_direct<KT>(G, L, v, rs, Fl, R, row, k, X, warm, max_piv, &fnum, &fcap);
    piv_total += it;
    nonconv += fcap;
    numeric += fnum;
    redone += 1;
    __syncwarp();
  }
  if (lane == 0) {
    if (redone) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->bpp_redo),
                          (unsigned long long)redone);
    if (piv_total) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->bpp_pivots),
                             (unsigned long long)piv_total);
    if (nonconv) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->bpp_nonconv),
                           (unsigned long long)nonconv);
    if (numeric) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->bpp_numeric),
                           (unsigned long long)numeric);
  }
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

}  // namespace

// scratch: Q (k x k), L (k x k), 1 / diag(L) (k), column sums of |Q| (k) in
// FP64, two flags, then one byte per row (redo flags)
size_t bpp_scratch_bytes(int k, int64_t rows) {
  return sizeof(double) * (2 * (size_t)k * k + 2 * (size_t)k) + 256 + (size_t)rows;
}

cudaError_t launch_bpp(const double *G, const float *R, int64_t rows, int k, float *X,
                       int max_pivots, int warm, DevCounters *ctr, void *scratch, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  if (k < 1 || k > AUNMF_BPP_K_MAX) return cudaErrorInvalidValue;
  float *Q = reinterpret_cast<float *>(scratch);  // G^{-1} as an FP32 pair (2 k^2 floats)
  double *L = reinterpret_cast<double *>(scratch) + (size_t)k * k;
  double *invd = L + (size_t)k * k;
  double *colsum = invd + k;
  int *chol_ok = reinterpret_cast<int *>(colsum + k);
  int *q_ok = chol_ok + 1;
  uint8_t *redo = reinterpret_cast<uint8_t *>(scratch) +
                  sizeof(double) * (2 * (size_t)k * k + 2 * (size_t)k) + 256;
  const size_t chol_smem = sizeof(double) * (size_t)k * k;
  cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chol_smem);
  k_chol<<<1, 256, chol_smem, s>>>(G, k, L, invd, chol_ok);
  k_inv_cols<<<k, 32, 0, s>>>(L, invd, k, Q, colsum);
  k_inv_check<<<1, 32, 0, s>>>(G, colsum, k, chol_ok, q_ok);
  const BppLayout lay = bpp_layout(k);
  const size_t budget = 200 * 1024;
  int wpb = (int)((budget / sizeof(double) - lay.shared_dbl) / lay.warp_dbl);
  if (wpb > kBppWarps) wpb = kBppWarps;
  if (wpb < 1) wpb = 1;
  const size_t smem = sizeof(double) * (lay.shared_dbl + (size_t)wpb * lay.warp_dbl);
  int64_t nb = (rows + wpb - 1) / wpb;
  if (nb > (int64_t)sm_count() * 2) nb = (int64_t)sm_count() * 2;
  // fallback: a full-size factor per warp, as many warps (<= 8) as fit
  const size_t fb_warp = (size_t)k * (k | 1) + 3 * (size_t)k;
  int fbw = (int)((budget / sizeof(double) - (size_t)k * k) / fb_warp);
  if (fbw > 8) fbw = 8;
  if (fbw < 1) fbw = 1;
  const size_t fb_smem = sizeof(double) * ((size_t)k * k + (size_t)fbw * fb_warp);
  int64_t nbf = (rows + fbw - 1) / fbw;
  if (nbf > (int64_t)sm_count()) nbf = sm_count();
  if (k <= 32) {
    cudaFuncSetAttribute(k_bpp<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_bpp<1><<<(unsigned)nb, 32 * wpb, smem, s>>>(G, Q, q_ok, R, rows, k, X, warm, max_pivots,
                                                  ctr, redo);
    cudaFuncSetAttribute(k_bpp_direct<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fb_smem);
    k_bpp_direct<1><<<(unsigned)nbf, 32 * fbw, fb_smem, s>>>(G, R, rows, k, X, warm, max_pivots, ctr,
                                                             redo);
  } else {
    cudaFuncSetAttribute(k_bpp<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_bpp<2><<<(unsigned)nb, 32 * wpb, smem, s>>>(G, Q, q_ok, R, rows, k, X, warm, max_pivots,
                                                  ctr, redo);
    cudaFuncSetAttribute(k_bpp_direct<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fb_smem);
    k_bpp_direct<2><<<(unsigned)nbf, 32 * fbw, fb_smem, s>>>(G, R, rows, k, X, warm, max_pivots, ctr,
                                                             redo);
  }
  g_launches += 5;
  return cudaGetLastError();
}

}  // namespace aunmf
