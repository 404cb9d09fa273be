// k_bpp.cu -- batched nonnegative least squares by block principal pivoting
// (Sec. 4.3: SolveBPP(C^T C, C^T B); Eqs. single NLS and KKT), in FP64.
//
// One warp solves one right-hand side r (a row of A H^T for W, a column of
// W^T A for H) against the shared Gram matrix G:
//     x = argmin_{x >= 0} ||C x - b||,   G = C^T C,  r = C^T b.
// Lane l owns the indices j = l and j = l + 32 (k <= 64): its passive flag,
// x_j, y_j = (G x - r)_j and the tolerance of the active-set test.  Each
// exchange solves G_FF x_F = r_F through the normal equations by a Cholesky
// factorisation of the passive block in the warp's slice of shared memory.
//
// Exchange rule (Kim-He-Park / Judice-Pires): V = {passive j: x_j < 0} U
// {active j: y_j < -tau_j}, tau_j = 1e-11 (|r_j| + sum_a |G_jF(a) x_F(a)|);
// if |V| shrank, flip all of V and reset the backup counter to 3; else if
// the counter is positive, decrement it and flip all of V; else flip only
// the largest index in V.  Start: passive set empty (x = 0, y = -r).
#include <math.h>

#include "internal.cuh"

namespace aunmf {
namespace {

constexpr double kBppYTol = 1e-11;
constexpr int kBppMaxWarps = 8;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct BppLayout {
  int ldl;         // leading dimension of L (odd, to spread shared-memory banks)
  size_t g_dbl;    // doubles for G
  size_t warp_dbl; // doubles per warp: L, z, r, F (ints, packed two per double)
};

__host__ __device__ inline BppLayout bpp_layout(int k) {
  BppLayout l;
  l.ldl = k | 1;
  l.g_dbl = (size_t)k * k;
  l.warp_dbl = (size_t)k * l.ldl + 2 * (size_t)k + ((size_t)k + 1) / 2;
  return l;
}

template <int KT>
__global__ void k_bpp(const float *__restrict__ G32, const float *__restrict__ R, int64_t rows,
                      int k, float *__restrict__ X, int max_piv, DevCounters *ctr) {
  extern __shared__ double sm[];
  const BppLayout lay = bpp_layout(k);
  double *G = sm;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) G[e] = (double)G32[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  double *L = sm + lay.g_dbl + (size_t)wib * lay.warp_dbl;
  double *z = L + (size_t)k * lay.ldl;
  double *rs = z + k;
  int *F = reinterpret_cast<int *>(rs + k);
  const int ldl = lay.ldl;
  const unsigned lt_mask = (1u << lane) - 1u;

  long long piv_total = 0, nonconv = 0, numeric = 0;
  for (int64_t row = (int64_t)blockIdx.x * nwb + wib; row < rows;
       row += (int64_t)gridDim.x * nwb) {
    double rr[KT], x[KT], y[KT], tau[KT];
    bool pas[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      rr[t] = j < k ? (double)R[row * k + j] : 0.0;
      if (j < k) rs[j] = rr[t];
      x[t] = 0.0;
      y[t] = -rr[t];
      tau[t] = kBppYTol * fabs(rr[t]);
      pas[t] = false;
    }
    __syncwarp();
    int alpha = 3, beta = k + 1, it = 0;
    bool failed_numeric = false, failed_cap = false;
    for (;;) {
      bool inf[KT];
      unsigned bal[KT];
      int nv = 0;
#pragma unroll
      for (int t = 0; t < KT; ++t) {
        const int j = lane + 32 * t;
        inf[t] = j < k && (pas[t] ? (x[t] < 0.0) : (y[t] < -tau[t]));
        bal[t] = __ballot_sync(0xffffffffu, inf[t]);
        nv += __popc(bal[t]);
      }
      if (nv == 0) break;
      if (it >= max_piv) { failed_cap = true; break; }
      ++it;
      if (nv < beta || alpha >= 1) {
        if (nv < beta) { beta = nv; alpha = 3; } else { alpha -= 1; }
#pragma unroll
        for (int t = 0; t < KT; ++t)
          if (inf[t]) pas[t] = !pas[t];
      } else {
        int vmax = -1;
#pragma unroll
        for (int t = KT - 1; t >= 0; --t)
          if (vmax < 0 && bal[t]) vmax = 32 * t + 31 - __clz(bal[t]);
#pragma unroll
        for (int t = 0; t < KT; ++t)
          if (lane + 32 * t == vmax) pas[t] = !pas[t];
      }
      // passive list F, ascending, and each lane's position in it
      int nf = 0, pos[KT];
#pragma unroll
      for (int t = 0; t < KT; ++t) {
        const int j = lane + 32 * t;
        const unsigned pb = __ballot_sync(0xffffffffu, pas[t] && j < k);
        pos[t] = nf + __popc(pb & lt_mask);
        nf += __popc(pb);
      }
#pragma unroll
      for (int t = 0; t < KT; ++t)
        if (pas[t]) F[pos[t]] = lane + 32 * t;
      __syncwarp();
      // Cholesky of G_FF (left-looking, column c; lanes over rows below c)
      for (int c = 0; c < nf; ++c) {
        double part = 0.0;
        for (int t = lane; t < c; t += 32) part = fma(L[c * ldl + t], L[c * ldl + t], part);
        const double d = G[F[c] * k + F[c]] - warp_sum_d(part);
        if (!(d > 0.0)) { failed_numeric = true; break; }
        const double lcc = sqrt(d);
        for (int a = c + 1 + lane; a < nf; a += 32) {
          double s = G[F[a] * k + F[c]];
          for (int t = 0; t < c; ++t) s = fma(-L[a * ldl + t], L[c * ldl + t], s);
          L[a * ldl + c] = s / lcc;
        }
        if (lane == 0) L[c * ldl + c] = lcc;
        __syncwarp();
      }
      if (failed_numeric) break;
      // z = G_FF^{-1} r_F: forward (L) then backward (L^T), column-oriented
      for (int a = lane; a < nf; a += 32) z[a] = rs[F[a]];
      __syncwarp();
      for (int c = 0; c < nf; ++c) {
        const double zc = z[c] / L[c * ldl + c];
        __syncwarp();
        for (int a = c + 1 + lane; a < nf; a += 32) z[a] = fma(-L[a * ldl + c], zc, z[a]);
        if (lane == 0) z[c] = zc;
        __syncwarp();
      }
      for (int c = nf - 1; c >= 0; --c) {
        const double zc = z[c] / L[c * ldl + c];
        __syncwarp();
        for (int a = lane; a < c; a += 32) z[a] = fma(-L[c * ldl + a], zc, z[a]);
        if (lane == 0) z[c] = zc;
        __syncwarp();
      }
      // x on the passive set, y = G x - r on the active set
#pragma unroll
      for (int t = 0; t < KT; ++t) {
        const int j = lane + 32 * t;
        if (j >= k) continue;
        if (pas[t]) {
          x[t] = z[pos[t]];
          y[t] = 0.0;
          tau[t] = 0.0;
        } else {
          x[t] = 0.0;
          double s = -rr[t], mag = fabs(rr[t]);
          for (int a = 0; a < nf; ++a) {
            const double g = G[j * k + F[a]] * z[a];
            s += g;
            mag += fabs(g);
          }
          y[t] = s;
          tau[t] = kBppYTol * mag;
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      if (j < k) X[row * k + j] = (float)x[t];
    }
    piv_total += it;
    nonconv += failed_cap;
    numeric += failed_numeric;
    __syncwarp();
  }
  if (lane == 0) {
    if (piv_total) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->bpp_pivots),
                             (unsigned long long)piv_total);
    if (nonconv) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->bpp_nonconv),
                           (unsigned long long)nonconv);
    if (numeric) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->bpp_numeric),
                           (unsigned long long)numeric);
  }
}

}  // namespace

cudaError_t launch_bpp(const float *G, const float *R, int64_t rows, int k, float *X,
                       int max_pivots, DevCounters *ctr, double * /*unused*/, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  if (k < 1 || k > AUNMF_BPP_K_MAX) return cudaErrorInvalidValue;
  const BppLayout lay = bpp_layout(k);
  const size_t budget = 200 * 1024;
  int wpb = (int)((budget / sizeof(double) - lay.g_dbl) / lay.warp_dbl);
  if (wpb > kBppMaxWarps) wpb = kBppMaxWarps;
  if (wpb < 1) wpb = 1;
  const size_t smem = sizeof(double) * (lay.g_dbl + (size_t)wpb * lay.warp_dbl);
  int64_t nb = (rows + wpb - 1) / wpb;
  if (nb > 152 * 4) nb = 152 * 4;
  if (k <= 32) {
    cudaFuncSetAttribute(k_bpp<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_bpp<1><<<(unsigned)nb, 32 * wpb, smem, s>>>(G, R, rows, k, X, max_pivots, ctr);
  } else {
    cudaFuncSetAttribute(k_bpp<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_bpp<2><<<(unsigned)nb, 32 * wpb, smem, s>>>(G, R, rows, k, X, max_pivots, ctr);
  }
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace aunmf
