// k_bpp.cu -- batched nonnegative least squares by block principal pivoting
// (Sec. 4.3: SolveBPP(C^T C, C^T B); Eqs. single NLS and KKT), in FP64.
//
// One warp solves one right-hand side r (a row of A H^T for W, a column of
// W^T A for H) against the shared Gram matrix G:
//     x = argmin_{x >= 0} ||C x - b||,   G = C^T C,  r = C^T b.
// Lane l owns the indices j = l and j = l + 32 (k <= 64): its passive flag,
// x_j, y_j = (G x - r)_j and the tolerance of the active-set test.
//
// Exchange rule (Kim-He-Park / Judice-Pires): V = {passive j: x_j < 0} U
// {active j: y_j < -tau_j}, tau_j = 1e-11 (|r_j| + sum_a |G_jF(a) x_F(a)|)
// (y_j in FP64, the scale tau_j in FP32 in the fast kernel);
// if |V| shrank, flip all of V and reset the backup counter to 3; else if
// the counter is positive, decrement it and flip all of V; else flip only
// the largest index in V.
//
// Each exchange solves the passive-set normal equations G_FF x_F = r_F in
// FP64 with a Cholesky factorisation of at most k/2 rows:
//   |F| <= |B|: Cholesky of G_FF itself;
//   |F| >  |B|: with Q = G^{-1} (FP64, computed once per update) and
//               z = Q r (once per right-hand side): the solution with x_B = 0
//               and y_F = 0 satisfies x = Q (r + y), so Q_BB y_B = -z_B
//               (Cholesky of Q_BB) and x_F = z_F + Q_FB y_B -- the block
//               inverse G_FF^{-1} = Q_FF - Q_FB Q_BB^{-1} Q_BF in other words.
// The solution of each NLS is unique when G is positive definite (Sec. 4),
// so the starting passive set changes only the work: the run driver starts
// each right-hand side from the support of its previous iterate.  Rows whose
// fast solve is not trustworthy (see k_bpp_direct) are redone from a cold
// start with full-size Cholesky factorisations of G_FF.
#include <math.h>

#include "internal.cuh"

namespace aunmf {
namespace {

constexpr double kBppYTol = 1e-11;
// G^{-1} is used for the passive-set solves only when cond_1(G) is below
// this (FP64 solves through it then keep at least ~8 digits)
constexpr double kQMaxCond = 1e8;
constexpr int kBppWarps = 16;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct BppLayout {
  int kh;          // largest factorisation: floor(k / 2)
  int ldl;         // leading dimension of L (odd)
  size_t g_dbl;    // doubles for G and for Q (each)
  size_t gf_dbl;   // doubles holding |G| in FP32 (tolerance scales)
  size_t warp_dbl; // doubles per warp: L, v (k), r (k), index lists (2k ints), |x_F| FP32 (k)
};

__host__ __device__ inline BppLayout bpp_layout(int k) {
  BppLayout l;
  l.kh = k / 2 > 0 ? k / 2 : 1;
  l.ldl = l.kh | 1;
  l.g_dbl = (size_t)k * k;
  l.gf_dbl = ((size_t)k * k + 1) / 2;
  l.warp_dbl = (size_t)l.kh * l.ldl + 2 * (size_t)k + (size_t)k + ((size_t)k + 1) / 2;
  return l;
}

// In-warp Cholesky of the n x n SPD matrix M(a, b) = Mg[I[a] * k + I[b]]
// into L (lower, ld ldl); the diagonal slot holds 1 / L_cc instead of L_cc
// (one reciprocal square root per column, then only multiplications: the
// FP64 pipe is the bottleneck, and each FP64 division or square root costs
// it several instructions).  Returns false (warp-uniform) on a non-positive
// pivot.
__device__ __forceinline__ bool warp_cholesky(const double *Mg, int k, const int *I, int n,
                                              double *L, int ldl, int lane) {
  for (int c = 0; c < n; ++c) {
    double part = 0.0;
    for (int t = lane; t < c; t += 32) part = fma(L[c * ldl + t], L[c * ldl + t], part);
    const double d = Mg[I[c] * k + I[c]] - warp_sum_d(part);
    if (!(d > 0.0)) return false;
    const double inv = rsqrt(d);
    for (int a = c + 1 + lane; a < n; a += 32) {
      double s = Mg[I[a] * k + I[c]];
      for (int t = 0; t < c; ++t) s = fma(-L[a * ldl + t], L[c * ldl + t], s);
      L[a * ldl + c] = s * inv;
    }
    if (lane == 0) L[c * ldl + c] = inv;
    __syncwarp();
  }
  return true;
}

// v <- (L L^T)^{-1} v for v[0..n) in shared memory (L from warp_cholesky,
// reciprocal diagonal).
__device__ __forceinline__ void warp_chol_solve(const double *L, int ldl, int n, double *v,
                                                int lane) {
  for (int c = 0; c < n; ++c) {
    const double vc = v[c] * L[c * ldl + c];
    __syncwarp();
    for (int a = c + 1 + lane; a < n; a += 32) v[a] = fma(-L[a * ldl + c], vc, v[a]);
    if (lane == 0) v[c] = vc;
    __syncwarp();
  }
  for (int c = n - 1; c >= 0; --c) {
    const double vc = v[c] * L[c * ldl + c];
    __syncwarp();
    for (int a = lane; a < c; a += 32) v[a] = fma(-L[c * ldl + a], vc, v[a]);
    if (lane == 0) v[c] = vc;
    __syncwarp();
  }
}

// Q = G^{-1} in FP64 (one block): Cholesky of G in shared memory, then each
// thread solves G q_j = e_j for its column j.  *ok = 0 if G is not positive
// definite or cond_1(G) >= kQMaxCond (the Q-based solves are then not used).
__global__ void k_gram_inverse(const float *__restrict__ G32, int k, double *__restrict__ Q,
                               int *__restrict__ ok) {
  extern __shared__ double sm[];
  double *L = sm;            // k x k
  double *tmp = sm + k * k;  // one column of k per thread
  __shared__ int good;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) L[e] = (double)G32[e];
  if (threadIdx.x == 0) good = 1;
  __syncthreads();
  for (int c = 0; c < k; ++c) {  // right-looking, lower triangle
    if (threadIdx.x == 0) {
      const double d = L[c * k + c];
      if (!(d > 0.0)) good = 0;
      L[c * k + c] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double lcc = L[c * k + c];
    for (int a = c + 1 + threadIdx.x; a < k; a += blockDim.x) L[a * k + c] /= lcc;
    __syncthreads();
    const int w = k - c - 1;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int a = c + 1 + e / w, b = c + 1 + e % w;
      if (b <= a) L[a * k + b] -= L[a * k + c] * L[b * k + c];
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double *v = tmp + (size_t)threadIdx.x * k;
    for (int i = 0; i < k; ++i) v[i] = (i == j) ? 1.0 : 0.0;
    for (int i = 0; i < k; ++i) {  // L v' = e_j
      double s = v[i];
      for (int t = 0; t < i; ++t) s -= L[i * k + t] * v[t];
      v[i] = s / L[i * k + i];
    }
    for (int i = k - 1; i >= 0; --i) {  // L^T q = v'
      double s = v[i];
      for (int t = i + 1; t < k; ++t) s -= L[t * k + i] * v[t];
      v[i] = s / L[i * k + i];
    }
    for (int i = 0; i < k; ++i) Q[i * k + j] = v[i];
  }
  __syncthreads();
  // cond_1(G) = ||G||_1 ||Q||_1 (max column sums): solves through Q lose
  // about log10(cond) digits, so Q is used only for well-conditioned G
  if (threadIdx.x == 0) {
    double ng = 0.0, nq = 0.0;
    for (int j = 0; j < k; ++j) {
      double cg = 0.0, cq = 0.0;
      for (int i = 0; i < k; ++i) {
        cg += fabs((double)G32[i * k + j]);
        cq += fabs(Q[i * k + j]);
      }
      ng = cg > ng ? cg : ng;
      nq = cq > nq ? cq : nq;
    }
    *ok = (good && ng * nq < kQMaxCond) ? 1 : 0;
  }
}

template <int KT>
__global__ void __launch_bounds__(32 * kBppWarps, 1)
    k_bpp(const float *__restrict__ G32, const double *__restrict__ Qg, const int *__restrict__ q_ok,
          const float *__restrict__ R, int64_t rows, int k, float *__restrict__ X, int warm,
          int max_piv, DevCounters *ctr, uint8_t *__restrict__ redo) {
  extern __shared__ double sm[];
  const BppLayout lay = bpp_layout(k);
  double *G = sm;
  double *Q = sm + lay.g_dbl;
  float *Gabs = reinterpret_cast<float *>(sm + 2 * lay.g_dbl);  // |G| in FP32
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    G[e] = (double)G32[e];
    Q[e] = Qg[e];
    Gabs[e] = fabsf(G32[e]);
  }
  const bool have_q = *q_ok != 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  double *L = sm + 2 * lay.g_dbl + lay.gf_dbl + (size_t)wib * lay.warp_dbl;
  double *v = L + (size_t)lay.kh * lay.ldl;   // small system's right-hand side, then x_F
  double *rs = v + k;                         // r, by index
  int *Fl = reinterpret_cast<int *>(rs + k);  // passive indices, ascending
  int *Bl = Fl + k;                           // active indices, ascending
  float *xa = reinterpret_cast<float *>(Bl + k);  // |x_F| in FP32, F order
  const int ldl = lay.ldl;
  const unsigned lt_mask = (1u << lane) - 1u;

  long long piv_total = 0, nonconv = 0;
  for (int64_t row = (int64_t)blockIdx.x * nwb + wib; row < rows;
       row += (int64_t)gridDim.x * nwb) {
    double rr[KT], x[KT], y[KT], tau[KT];
    bool pas[KT];
    bool any = false;
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      rr[t] = j < k ? (double)R[row * k + j] : 0.0;
      if (j < k) rs[j] = rr[t];
      pas[t] = warm && j < k && X[row * k + j] > 0.f;
      any |= pas[t];
      x[t] = 0.0;
      y[t] = -rr[t];
      tau[t] = kBppYTol * fabs(rr[t]);
    }
    __syncwarp();
    // z = G^{-1} r, shared by every exchange of this right-hand side
    double z[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      double acc = 0.0;
      if (have_q && j < k)
        for (int l = 0; l < k; ++l) acc = fma(Q[j * k + l], rs[l], acc);
      z[t] = acc;
    }
    int alpha = 3, beta = k + 1, it = 0;
    bool failed_numeric = false, failed_cap = false;
    bool need_solve = __any_sync(0xffffffffu, any);
    for (;;) {
      if (need_solve) {
        // ---- passive / active lists and each lane's positions in them
        int nf = 0, nb = 0, posf[KT], posb[KT];
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          const int j = lane + 32 * t;
          const unsigned pf = __ballot_sync(0xffffffffu, pas[t] && j < k);
          const unsigned pb = __ballot_sync(0xffffffffu, !pas[t] && j < k);
          posf[t] = nf + __popc(pf & lt_mask);
          posb[t] = nb + __popc(pb & lt_mask);
          nf += __popc(pf);
          nb += __popc(pb);
        }
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          const int j = lane + 32 * t;
          if (j < k) {
            if (pas[t]) Fl[posf[t]] = j; else Bl[posb[t]] = j;
          }
        }
        __syncwarp();
        if (nf <= nb || !have_q) {
          // ---- direct: G_FF x_F = r_F; v[0..nf) ends as x_F in F order
          if (nf > lay.kh) { failed_numeric = true; break; }
          if (!warp_cholesky(G, k, Fl, nf, L, ldl, lane)) { failed_numeric = true; break; }
          for (int a = lane; a < nf; a += 32) v[a] = rs[Fl[a]];
          __syncwarp();
          warp_chol_solve(L, ldl, nf, v, lane);
#pragma unroll
          for (int t = 0; t < KT; ++t) x[t] = pas[t] ? v[posf[t]] : 0.0;
        } else {
          // ---- through Q = G^{-1} and z = Q r: the constrained solution has
          // Q_BB y_B = -z_B and x_F = z_F + Q_FB y_B (y_F = 0, x_B = 0)
#pragma unroll
          for (int t = 0; t < KT; ++t) {
            const int j = lane + 32 * t;
            if (j < k && !pas[t]) v[posb[t]] = z[t];
          }
          __syncwarp();
          if (!warp_cholesky(Q, k, Bl, nb, L, ldl, lane)) { failed_numeric = true; break; }
          warp_chol_solve(L, ldl, nb, v, lane);  // v = Q_BB^{-1} z_B = -y_B
#pragma unroll
          for (int t = 0; t < KT; ++t) {
            const int j = lane + 32 * t;
            double s = z[t];
            if (j < k && pas[t])
              for (int b = 0; b < nb; ++b) s = fma(-Q[j * k + Bl[b]], v[b], s);
            x[t] = (j < k && pas[t]) ? s : 0.0;
            if (j < k && !pas[t]) y[t] = -v[posb[t]];
          }
          __syncwarp();
#pragma unroll
          for (int t = 0; t < KT; ++t)
            if (pas[t]) v[posf[t]] = x[t];  // x_F in F order for the tolerance scales
        }
        __syncwarp();
        for (int a = lane; a < nf; a += 32) xa[a] = fabsf((float)v[a]);
        __syncwarp();
        // ---- active set: y = G_BF x_F - r_B (direct route; the Q route has
        // it already) and the tolerance scale |r_j| + sum |G_jF x_F|, summed
        // in FP32 from |G| and |x_F|
        const bool direct = nf <= nb || !have_q;
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          const int j = lane + 32 * t;
          if (j >= k) continue;
          if (pas[t]) {
            y[t] = 0.0;
            tau[t] = 0.0;
          } else {
            float mag = fabsf((float)rr[t]);
            for (int a = 0; a < nf; ++a) mag = fmaf(Gabs[j * k + Fl[a]], xa[a], mag);
            tau[t] = kBppYTol * (double)mag;
            if (direct) {
              double s = -rr[t];
              for (int a = 0; a < nf; ++a) s = fma(G[j * k + Fl[a]], v[a], s);
              y[t] = s;
            }
          }
        }
        __syncwarp();
      }
      // ---- infeasible set and exchange
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
      need_solve = true;
    }
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      if (j < k) X[row * k + j] = (float)x[t];
    }
    if (lane == 0) redo[row] = failed_numeric ? 1 : 0;
    if (!failed_numeric) {
      piv_total += it;
      nonconv += failed_cap;
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

// Fallback for the rows the fast kernel flagged (a non-positive pivot in a
// k/2-sized factorisation, or a passive set too large for it while Q is not
// in use because G is not numerically positive definite or is badly
// conditioned): the same exchange rule from a cold start, every passive
// system solved by a Cholesky factorisation of G_FF of any size.
template <int KT>
__global__ void __launch_bounds__(256)
    k_bpp_direct(const float *__restrict__ G32, const float *__restrict__ R, int64_t rows, int k,
                 float *__restrict__ X, int max_piv, DevCounters *ctr,
                 const uint8_t *__restrict__ redo) {
  extern __shared__ double sm[];
  const int ldl = k | 1;
  double *G = sm;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) G[e] = (double)G32[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  double *L = sm + (size_t)k * k + (size_t)wib * ((size_t)k * ldl + 3 * (size_t)k);
  double *v = L + (size_t)k * ldl;
  double *rs = v + k;
  int *Fl = reinterpret_cast<int *>(rs + k);
  const unsigned lt_mask = (1u << lane) - 1u;
  long long piv_total = 0, nonconv = 0, numeric = 0;
  for (int64_t row = (int64_t)blockIdx.x * nwb + wib; row < rows;
       row += (int64_t)gridDim.x * nwb) {
    if (!redo[row]) continue;
    double rr[KT], x[KT], y[KT], tau[KT];
    bool pas[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      rr[t] = j < k ? (double)R[row * k + j] : 0.0;
      if (j < k) rs[j] = rr[t];
      pas[t] = false;
      x[t] = 0.0;
      y[t] = -rr[t];
      tau[t] = kBppYTol * fabs(rr[t]);
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
        if (pas[t]) Fl[pos[t]] = lane + 32 * t;
      __syncwarp();
      if (!warp_cholesky(G, k, Fl, nf, L, ldl, lane)) { failed_numeric = true; break; }
      for (int a = lane; a < nf; a += 32) v[a] = rs[Fl[a]];
      __syncwarp();
      warp_chol_solve(L, ldl, nf, v, lane);
#pragma unroll
      for (int t = 0; t < KT; ++t) {
        const int j = lane + 32 * t;
        if (j >= k) continue;
        if (pas[t]) {
          x[t] = v[pos[t]];
          y[t] = 0.0;
          tau[t] = 0.0;
        } else {
          x[t] = 0.0;
          double s = -rr[t], mag = fabs(rr[t]);
          for (int a = 0; a < nf; ++a) {
            const double g = G[j * k + Fl[a]] * v[a];
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

size_t bpp_scratch_bytes(int k, int64_t rows) {
  return sizeof(double) * (size_t)k * k + 256 + (size_t)rows;
}

cudaError_t launch_bpp(const float *G, const float *R, int64_t rows, int k, float *X,
                       int max_pivots, int warm, DevCounters *ctr, void *scratch, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  if (k < 1 || k > AUNMF_BPP_K_MAX) return cudaErrorInvalidValue;
  double *Q = reinterpret_cast<double *>(scratch);
  int *q_ok = reinterpret_cast<int *>(Q + (size_t)k * k);
  uint8_t *redo = reinterpret_cast<uint8_t *>(scratch) + sizeof(double) * (size_t)k * k + 256;
  const size_t inv_smem = sizeof(double) * ((size_t)k * k + (size_t)k * 64);
  cudaFuncSetAttribute(k_gram_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_smem);
  k_gram_inverse<<<1, 64, inv_smem, s>>>(G, k, Q, q_ok);
  const BppLayout lay = bpp_layout(k);
  const size_t budget = 200 * 1024;
  int wpb = (int)((budget / sizeof(double) - 2 * lay.g_dbl - lay.gf_dbl) / lay.warp_dbl);
  if (wpb > kBppWarps) wpb = kBppWarps;
  if (wpb < 1) wpb = 1;
  const size_t smem = sizeof(double) * (2 * lay.g_dbl + lay.gf_dbl + (size_t)wpb * lay.warp_dbl);
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
    k_bpp_direct<1><<<(unsigned)nbf, 32 * fbw, fb_smem, s>>>(G, R, rows, k, X, max_pivots, ctr,
                                                             redo);
  } else {
    cudaFuncSetAttribute(k_bpp<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_bpp<2><<<(unsigned)nb, 32 * wpb, smem, s>>>(G, Q, q_ok, R, rows, k, X, warm, max_pivots,
                                                  ctr, redo);
    cudaFuncSetAttribute(k_bpp_direct<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fb_smem);
    k_bpp_direct<2><<<(unsigned)nbf, 32 * fbw, fb_smem, s>>>(G, R, rows, k, X, max_pivots, ctr,
                                                             redo);
  }
  g_launches += 3;
  return cudaGetLastError();
}

}  // namespace aunmf
