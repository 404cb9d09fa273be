// bpp_core.cuh -- device routines of block principal pivoting (Sec. 4.3,
// SolveBPP; Eqs. single NLS and KKT) shared by the single-problem kernels
// (k_bpp.cu) and the batched kernels (k_batched.cu).  See k_bpp.cu for the
// method and the exchange rule.
#pragma once

#include <math.h>

#include "internal.cuh"

namespace aunmf {
namespace bpp {

constexpr double kBppYTol = 1e-11;
// An index whose Gram diagonal is <= kDead of the largest (a zero column of
// the fixed factor, which ABPP can produce) never becomes passive: the normal
// equations leave its value undetermined and it stays 0.
constexpr double kDead = 1e-12;
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
__device__ __forceinline__ void gram_inverse_block(const double *__restrict__ Gd, int k,
                                                   double *__restrict__ Q, int *__restrict__ ok,
                                                   double *sm, int &good) {
  double *L = sm;            // k x k
  double *tmp = sm + k * k;  // one column of k per thread
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) L[e] = Gd[e];
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
        cg += fabs(Gd[i * k + j]);
        cq += fabs(Q[i * k + j]);
      }
      ng = cg > ng ? cg : ng;
      nq = cq > nq ? cq : nq;
    }
    *ok = (good && ng * nq < kQMaxCond) ? 1 : 0;
  }
}


// Shared-memory view of one warp's BPP state (fast kernel).
struct BppWarp {
  const double *G, *Q;
  const float *Gabs;
  double dead_below;  // kDead * max diagonal of G
  bool have_q;
  double *L, *v, *rs;
  int *Fl, *Bl;
  float *xa;
  int ldl, kh;
};

// Stage G (FP64), Q and |G| (FP32) of one problem into shared memory (block-
// wide; the caller synchronises) and return warp wib's view.
__device__ __forceinline__ BppWarp bpp_stage(const double *__restrict__ Gd,
                                             const double *__restrict__ Qg, const int *q_ok, int k,
                                             double *sm, int wib) {
  const BppLayout lay = bpp_layout(k);
  double *G = sm;
  double *Q = sm + lay.g_dbl;
  float *Gabs = reinterpret_cast<float *>(sm + 2 * lay.g_dbl);
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    G[e] = Gd[e];
    Q[e] = Qg[e];
    Gabs[e] = (float)fabs(Gd[e]);
  }
  BppWarp w;
  w.G = G;
  w.Q = Q;
  w.Gabs = Gabs;
  double gmax = 0.0;
  for (int i = 0; i < k; ++i) gmax = fmax(gmax, Gd[i * k + i]);
  w.dead_below = kDead * gmax;
  w.have_q = *q_ok != 0;
  w.L = sm + 2 * lay.g_dbl + lay.gf_dbl + (size_t)wib * lay.warp_dbl;
  w.v = w.L + (size_t)lay.kh * lay.ldl;  // small system's right-hand side, then x_F
  w.rs = w.v + k;                        // r, by index
  w.Fl = reinterpret_cast<int *>(w.rs + k);  // passive indices, ascending
  w.Bl = w.Fl + k;                           // active indices, ascending
  w.xa = reinterpret_cast<float *>(w.Bl + k);  // |x_F| in FP32, F order
  w.ldl = lay.ldl;
  w.kh = lay.kh;
  return w;
}

// Solves row `row` of R (rows x k) into X (warm: start from the support of
// X's row); returns the exchanges, *failed_numeric / *failed_cap.
template <int KT>
__device__ __forceinline__ int bpp_row_fast(const BppWarp &w, const float *__restrict__ R,
                                            int64_t row, int k, float *__restrict__ X, int warm,
                                            int max_piv, bool *failed_numeric_out,
                                            bool *failed_cap_out) {
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const double *G = w.G, *Q = w.Q;
  const float *Gabs = w.Gabs;
  const bool have_q = w.have_q;
  double *L = w.L, *v = w.v, *rs = w.rs;
  int *Fl = w.Fl, *Bl = w.Bl;
  float *xa = w.xa;
  const int ldl = w.ldl;
  struct {
    int kh;
  } lay{w.kh};
    double rr[KT], x[KT], y[KT], tau[KT];
    bool pas[KT], dead[KT];
    bool any = false;
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      rr[t] = j < k ? (double)R[row * k + j] : 0.0;
      if (j < k) rs[j] = rr[t];
      dead[t] = !(j < k && G[j * k + j] > w.dead_below);
      pas[t] = warm && !dead[t] && X[row * k + j] > 0.f;
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
        inf[t] = j < k && (pas[t] ? (x[t] < 0.0) : (!dead[t] && y[t] < -tau[t]));
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
    *failed_numeric_out = failed_numeric;
    *failed_cap_out = failed_cap;
    return it;
}

// Fallback for the rows the fast kernel flagged (a non-positive pivot in a
// k/2-sized factorisation, or a passive set too large for it while Q is not
// in use because G is not numerically positive definite or is badly
// conditioned): the same exchange rule from a cold start, every passive
// system solved by a Cholesky factorisation of G_FF of any size.
template <int KT>
__device__ __forceinline__ int bpp_row_direct(const double *__restrict__ G, double *L, double *v,
                                              double *rs, int *Fl, const float *__restrict__ R,
                                              int64_t row, int k, float *__restrict__ X,
                                              int max_piv, bool *failed_numeric_out,
                                              bool *failed_cap_out) {
  const int lane = threadIdx.x & 31;
  const int ldl = k | 1;
  const unsigned lt_mask = (1u << lane) - 1u;
  double gmax = 0.0;
  for (int i = 0; i < k; ++i) gmax = fmax(gmax, G[i * k + i]);
    double rr[KT], x[KT], y[KT], tau[KT];
    bool pas[KT], dead[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      rr[t] = j < k ? (double)R[row * k + j] : 0.0;
      if (j < k) rs[j] = rr[t];
      dead[t] = !(j < k && G[j * k + j] > kDead * gmax);
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
        inf[t] = j < k && (pas[t] ? (x[t] < 0.0) : (!dead[t] && y[t] < -tau[t]));
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
    *failed_numeric_out = failed_numeric;
    *failed_cap_out = failed_cap;
    return it;
}

}  // namespace bpp
}  // namespace aunmf
