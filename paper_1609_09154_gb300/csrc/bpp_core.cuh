// bpp_core.cuh -- device routines of block principal pivoting (Sec. 4.3,
// SolveBPP; Eqs. single NLS and KKT) shared by the single-problem kernels
// (k_bpp.cu) and the batched kernels (k_batched.cu).  See k_bpp.cu for the
// method and the exchange rule.
#pragma once

#include <math.h>

#include "internal.cuh"

namespace aunmf {
namespace bpp {

// G and Q = G^{-1} are symmetric; the loops below read them as G[l][j] with
// the lane on j (consecutive addresses) rather than G[j][l], whose stride of
// k elements puts a warp's reads in a few shared-memory banks (32-way
// conflicts at k = 64).

constexpr double kBppYTol = 1e-11;
constexpr float kBppYTolF = 1e-11f;
// An index whose Gram diagonal is <= kDead of the largest (a zero column of
// the fixed factor, which ABPP can produce) never becomes passive: the normal
// equations leave its value undetermined and it stays 0.
constexpr double kDead = 1e-12;
// G^{-1} is used for the passive-set solves only when cond_1(G) is below
// this (FP64 solves through it then keep at least ~8 digits)
// G^{-1} is used while cond_1(G) < kQMaxCond; from kQRefineCond on, each
// solve through it takes one step of iterative refinement.  (ABPP's factors
// on uniform low-rank data reach cond ~1e9: without the refinement those
// rows would need full-size factorisations of G_FF.)
constexpr double kQRefineCond = 1e8;
constexpr double kQMaxCond = 1e12;
constexpr int kBppWarps = 16;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared memory of the fast kernel: Q = G^{-1} and G as FP32 pairs (k^2
// doubles each), then per warp: the FP32 Cholesky factor L (kh x ldl floats),
// a right-hand-side pair (2k floats), corrections (k floats), the index lists
// (2k ints), |x_F|, r, and a solution pair (k floats each).  Nothing is FP64:
// a row whose FP32 solve cannot finish goes to the FP64 fallback kernel.
struct BppLayout {
  int kh;            // largest factorisation: floor(k / 2)
  int ldl;           // leading dimension of L (odd)
  size_t shared_dbl; // doubles shared by the block (the two pairs)
  size_t warp_dbl;   // doubles per warp
};

__host__ __device__ inline BppLayout bpp_layout(int k) {
  BppLayout l;
  l.kh = k / 2 > 0 ? k / 2 : 1;
  l.ldl = l.kh | 1;
  l.shared_dbl = 2 * (size_t)k * k;
  const size_t kf = 2 * (((size_t)k + 1) / 2);  // k floats, rounded up to whole doubles
  l.warp_dbl = ((size_t)l.kh * l.ldl + 1) / 2 + kf + kf / 2 + (size_t)k + 4 * (kf / 2);
  return l;
}

// In-warp Cholesky of the n x n SPD matrix M(a, b) = Mg[I[a] * k + I[b]]
// into L (lower, ld ldl); the diagonal slot holds 1 / L_cc instead of L_cc
// (one reciprocal square root per column, then only multiplications: the
// FP64 pipe is the bottleneck, and each FP64 division or square root costs
// it several instructions).  Right-looking: after column c is scaled, the
// warp's lanes share the entries of the trailing lower triangle (w (w + 1) / 2
// of them, w = n - c - 1), so a factorisation costs ~n^3 / 192 FP64 warp
// instructions plus ~10 per column, where one lane per row would cost
// ~n^2 / 2 (each lane running the longest dot product of its column).
// Returns false (warp-uniform) on a non-positive pivot.
__device__ __forceinline__ double rsq(double d) { return rsqrt(d); }
__device__ __forceinline__ float rsq(float d) { return rsqrtf(d); }

template <class T, class Acc>
__device__ __forceinline__ bool warp_cholesky(Acc M, const int *I, int n, T *L, int ldl,
                                              int lane) {
  // lower triangle of M_FF into L; entry e of the triangle is (a, b) with
  // a (a + 1) / 2 <= e < (a + 1) (a + 2) / 2
  const int tri = n * (n + 1) / 2;
  for (int e = lane; e < tri; e += 32) {
    int a = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    if ((a + 1) * (a + 2) / 2 <= e) ++a;
    if (a * (a + 1) / 2 > e) --a;
    const int b = e - a * (a + 1) / 2;
    L[a * ldl + b] = M(I[b], I[a]);
  }
  __syncwarp();
  for (int c = 0; c < n; ++c) {
    const T d = L[c * ldl + c];
    if (!(d > T(0))) return false;
    const T r = rsq(d);
    for (int a = c + 1 + lane; a < n; a += 32) L[a * ldl + c] *= r;
    __syncwarp();
    if (lane == 0) L[c * ldl + c] = r;
    const int w = n - c - 1, tw = w * (w + 1) / 2;
    for (int e = lane; e < tw; e += 32) {
      int a = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      if ((a + 1) * (a + 2) / 2 <= e) ++a;
      if (a * (a + 1) / 2 > e) --a;
      const int b = e - a * (a + 1) / 2;
      const int ra = c + 1 + a, rb = c + 1 + b;
      L[ra * ldl + rb] = fma(-L[ra * ldl + c], L[rb * ldl + c], L[ra * ldl + rb]);
    }
    __syncwarp();
  }
  return true;
}

// v <- (L L^T)^{-1} v for v[0..n) in shared memory (L from warp_cholesky,
// reciprocal diagonal).
template <class T>
__device__ __forceinline__ void warp_chol_solve(const T *L, int ldl, int n, T *v, int lane) {
  for (int c = 0; c < n; ++c) {
    const T vc = v[c] * L[c * ldl + c];
    __syncwarp();
    for (int a = c + 1 + lane; a < n; a += 32) v[a] = fma(-L[a * ldl + c], vc, v[a]);
    if (lane == 0) v[c] = vc;
    __syncwarp();
  }
  for (int c = n - 1; c >= 0; --c) {
    const T vc = v[c] * L[c * ldl + c];
    __syncwarp();
    for (int a = lane; a < c; a += 32) v[a] = fma(-L[c * ldl + a], vc, v[a]);
    if (lane == 0) v[c] = vc;
    __syncwarp();
  }
}

// Q = G^{-1} in three steps, spread over the GPU (a single block doing it
// serially spent ~0.5 ms per update in FP64 latency):
//   chol_block:   L = chol(G) (lower, row-major k x k) and invd = 1 / diag(L),
//                 one block; ok = 0 on a non-positive pivot;
//   inv_col_warp: column j of Q by forward and back substitution against
//                 e_j, one warp per column (lane i owns rows i, i + 32),
//                 stored as an FP32 pair Qs[e] = hi, Qs[k^2 + e] = lo with
//                 hi + lo = Q_e to ~2^-48, and the column's sum of |Q_ij|;
//   inv_check:    q_ok = 0 unless ok and cond_1(G) = ||G||_1 ||Q||_1 <
//                 kQMaxCond; 2 when cond_1(G) >= kQRefineCond, else 1.
__device__ __forceinline__ void chol_block(const double *__restrict__ G, int k,
                                           double *__restrict__ Lg, double *__restrict__ invd,
                                           int *__restrict__ ok, double *A) {
  __shared__ int good;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) A[e] = G[e];
  if (threadIdx.x == 0) good = 1;
  __syncthreads();
  for (int c = 0; c < k; ++c) {
    if (threadIdx.x == 0) {
      const double d = A[c * k + c];
      if (!(d > 0.0)) good = 0;
      const double r = d > 0.0 ? rsqrt(d) : 1.0;
      A[c * k + c] = r;  // reciprocal of L_cc
    }
    __syncthreads();
    const double r = A[c * k + c];
    for (int a = c + 1 + threadIdx.x; a < k; a += blockDim.x) A[a * k + c] *= r;
    __syncthreads();
    const int w = k - c - 1;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int a = c + 1 + e / w, b = c + 1 + e % w;
      if (b <= a) A[a * k + b] = fma(-A[a * k + c], A[b * k + c], A[a * k + b]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, b = e % k;
    Lg[e] = b < a ? A[e] : 0.0;
    if (a == b) invd[a] = A[e];
  }
  if (threadIdx.x == 0) *ok = good;
}

__device__ __forceinline__ void inv_col_warp(const double *__restrict__ Lg,
                                             const double *__restrict__ invd, int k, int j,
                                             float *__restrict__ Qs, double *__restrict__ colsum) {
  const int lane = threadIdx.x & 31;
  double w[2], acc[2] = {0.0, 0.0};
  // forward: w_i = (e_ij - sum_{t < i} L_it w_t) / L_ii
  for (int t = 0; t < k; ++t) {
    const int o = t >> 5, ol = t & 31;
    double wt = 0.0;
    if (lane == ol) {
      const double e = t == j ? 1.0 : 0.0;
      wt = (e - acc[o]) * invd[t];
      w[o] = wt;
    }
    wt = __shfl_sync(0xffffffffu, wt, ol);
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const int i = lane + 32 * s2;
      if (i > t && i < k) acc[s2] = fma(Lg[i * k + t], wt, acc[s2]);
    }
  }
  // back: q_i = (w_i - sum_{t > i} L_ti q_t) / L_ii
  double q[2];
  acc[0] = acc[1] = 0.0;
  for (int t = k - 1; t >= 0; --t) {
    const int o = t >> 5, ol = t & 31;
    double qt = 0.0;
    if (lane == ol) {
      qt = (w[o] - acc[o]) * invd[t];
      q[o] = qt;
    }
    qt = __shfl_sync(0xffffffffu, qt, ol);
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const int i = lane + 32 * s2;
      if (i < t) acc[s2] = fma(Lg[t * k + i], qt, acc[s2]);
    }
  }
  double cs = 0.0;
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
    const int i = lane + 32 * s2;
    if (i < k) {
      const float hi = (float)q[s2];
      Qs[i * k + j] = hi;
      Qs[k * k + i * k + j] = (float)(q[s2] - (double)hi);
      cs += fabs(q[s2]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
  if (lane == 0) colsum[j] = cs;
}

__device__ __forceinline__ void inv_check(const double *__restrict__ G,
                                          const double *__restrict__ colsum, int k, const int *ok,
                                          int *__restrict__ q_ok) {
  // one warp: lane l takes columns l, l + 32 (k <= 64), then max-reduce
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  double ng = 0.0, nq = 0.0;
  for (int c = lane; c < k; c += 32) {
    double cg = 0.0;
    for (int i = 0; i < k; ++i) cg += fabs(G[i * k + c]);
    ng = fmax(ng, cg);
    nq = fmax(nq, colsum[c]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ng = fmax(ng, __shfl_xor_sync(0xffffffffu, ng, o));
    nq = fmax(nq, __shfl_xor_sync(0xffffffffu, nq, o));
  }
  if (lane == 0) {
    const double cond = ng * nq;
    *q_ok = (*ok && cond < kQMaxCond) ? (cond < kQRefineCond ? 1 : 2) : 0;
  }
}

// Shared-memory view of one warp's BPP state (fast kernel).
struct BppWarp {
  const float *Qh, *Ql;  // G^{-1} = Qh + Ql (FP32 pair)
  const float *Gh, *Gl;  // G = Gh + Gl (to ~2^-48); |Gh| scales the tolerances
  double dead_below;  // kDead * max diagonal of G
  unsigned live[2];    // bit j % 32 of live[j / 32]: G_jj > dead_below (k <= 64)
  bool have_q;
  bool refine;  // solves through G^{-1} take a refinement step
  float *Lf;       // FP32 Cholesky factor (kh x ldl)
  float *bh, *bl;  // right-hand side pair (k each)
  float *dv;       // corrections (k)
  int *Fl, *Bl;
  float *xa;
  float *rsf;  // r in FP32, by index
  float *vh, *vl;  // solution pairs: x_F in F order or Q_BB^{-1} z_B in B order
  int ldl, kh;
};

// Stage Q and G (FP32 pairs) of one problem into shared memory (block-wide;
// the caller synchronises) and return warp wib's view.
__device__ __forceinline__ BppWarp bpp_stage(const double *__restrict__ Gd,
                                             const float *__restrict__ Qsg, const int *q_ok, int k,
                                             double *sm, int wib) {
  const BppLayout lay = bpp_layout(k);
  float *Qs = reinterpret_cast<float *>(sm);                        // hi (k^2), lo (k^2)
  float *Gp = reinterpret_cast<float *>(sm + (size_t)k * k);        // hi (k^2), lo (k^2)
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const double g = Gd[e];
    Qs[e] = Qsg[e];
    Qs[k * k + e] = Qsg[k * k + e];
    const float gh = (float)g;
    Gp[e] = gh;
    Gp[k * k + e] = (float)(g - (double)gh);
  }
  BppWarp w;
  w.Qh = Qs;
  w.Ql = Qs + k * k;
  w.Gh = Gp;
  w.Gl = Gp + k * k;
  double gmax = 0.0;
  for (int i = 0; i < k; ++i) gmax = fmax(gmax, Gd[i * k + i]);
  w.dead_below = kDead * gmax;
  {
    // the warp's own copy of the live-index mask (its lanes are converged here)
    const int lane = threadIdx.x & 31;
    const int j0 = lane, j1 = lane + 32;
    w.live[0] = __ballot_sync(0xffffffffu, j0 < k && Gd[j0 * k + j0] > w.dead_below);
    w.live[1] = __ballot_sync(0xffffffffu, j1 < k && Gd[j1 * k + j1] > w.dead_below);
  }
  w.have_q = *q_ok != 0;
  w.refine = *q_ok == 2;
  const size_t kf = 2 * (((size_t)k + 1) / 2);
  float *base = reinterpret_cast<float *>(sm + lay.shared_dbl + (size_t)wib * lay.warp_dbl);
  w.Lf = base;
  w.bh = base + 2 * (((size_t)lay.kh * lay.ldl + 1) / 2);
  w.bl = w.bh + kf;
  w.dv = w.bl + kf;
  w.Fl = reinterpret_cast<int *>(w.dv + kf);  // passive indices, ascending (k)
  w.Bl = w.Fl + k;                            // active indices, ascending (k)
  w.xa = reinterpret_cast<float *>(w.Bl + k);  // |x_F| in FP32, F order
  w.rsf = w.xa + kf;
  w.vh = w.rsf + kf;
  w.vl = w.vh + kf;
  w.ldl = lay.ldl;
  w.kh = lay.kh;
  return w;
}

// ---- FP32-pair arithmetic (no FP64 instruction): a value is hi + lo with
// |lo| <= ulp(hi) / 2, ~48 bits.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// (h, l) += (bh, bl)
__device__ __forceinline__ void pair_add(float &h, float &l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(l, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}
// (h, l) = sum_b M(I[b], j) x_b, M = Mh + Ml and x = xh + xl (pairs): each
// Mh xh product exact, the cross terms at FP32 precision, summed in a pair.
__device__ __forceinline__ void pair_dot(const float *Mh, const float *Ml, int k, const int *I,
                                         int n, int j, const float *xh, const float *xl,
                                         float &h, float &l) {
  float hi = 0.f, lo = 0.f;
  for (int b = 0; b < n; ++b) {
    const int e = I[b] * k + j;
    const float mh = Mh[e], ph = xh[b];
    two_fma_acc(mh, ph, hi, lo);
    lo = fmaf(mh, xl[b], lo);
    lo = fmaf(Ml[e], ph, lo);
  }
  h = __fadd_rn(hi, lo);
  l = __fsub_rn(lo, __fsub_rn(h, hi));
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

constexpr int kRefineSteps = 6;
constexpr float kRefineTol = 9.31322575e-10f;  // 2^-30

// M x = b for the n x n SPD matrix M = Mh + Ml (an FP32 pair; rows and
// columns I of a k x k matrix) and b = bh + bl (a pair, in I order): an FP32
// Cholesky of Mh, then iterative refinement with the residual b - M x summed
// in pairs, until a correction is below 2^-30 of x (x goes out in FP32).  No
// FP64 instruction: this part runs ~60x more FP32 than FP64 operations per
// clock, and its FP64 solves cost ~16 SM clocks per warp instruction, most of
// them serial (one per column).  x = xh + xl, in I order.  Returns false
// (warp-uniform) on a pivot <= 0 of Mh or when the corrections stall (an
// ill-conditioned M); the caller then takes the FP64 solve.
__device__ __forceinline__ bool solve_mixed(const float *Mh, const float *Ml, int k, const int *I,
                                            int n, const float *bh, const float *bl, float *Lf,
                                            int ldl, float *d, float *xh, float *xl, int lane) {
  auto Mf = [Mh, k](int a, int b) { return Mh[a * k + b]; };
  if (!warp_cholesky(Mf, I, n, Lf, ldl, lane)) return false;
  for (int a = lane; a < n; a += 32) {
    xh[a] = 0.f;
    xl[a] = 0.f;
    d[a] = bh[a];
  }
  __syncwarp();
  for (int step = 0; step < kRefineSteps; ++step) {
    warp_chol_solve(Lf, ldl, n, d, lane);
    float dm = 0.f, xm = 0.f;
    for (int a = lane; a < n; a += 32) {
      pair_add(xh[a], xl[a], d[a], 0.f);
      dm = fmaxf(dm, fabsf(d[a]));
      xm = fmaxf(xm, fabsf(xh[a]));
    }
    dm = warp_max(dm);
    xm = warp_max(xm);
    if (dm <= kRefineTol * xm) return true;
    if (!(dm < 3.0e38f)) return false;
    __syncwarp();
    for (int a = lane; a < n; a += 32) {
      float h, l;
      pair_dot(Mh, Ml, k, I, n, I[a], xh, xl, h, l);  // (M x)_a
      float rh = bh[a], rl = bl[a];
      pair_add(rh, rl, -h, -l);
      d[a] = __fadd_rn(rh, rl);
    }
    __syncwarp();
  }
  return false;
}

// Solves row `row` of R (rows x k) into X (warm 1: start from the support of
// X's row; warm 2: from the positive entries of the unconstrained solution
// z = G^{-1} r when G^{-1} is usable (else as warm 1) -- for a first update,
// whose X (zero, or a random start) says nothing about the solution; warm 0:
// from the empty passive set); returns the exchanges, *failed_numeric /
// *failed_cap.  Each
// lane keeps its entries of r (FP32), x and y (FP32 pairs) and the
// tolerances (FP32): the exchange rule needs only their signs and
// magnitudes, and FP64 instructions -- conversions and compares included --
// run at ~1/60 of the FP32 rate.  The passive-set systems are solved by
// solve_mixed; a system it cannot finish sends the row to the FP64 fallback
// kernel (k_bpp_direct), so this kernel keeps no FP64 state.
template <int KT>
__device__ __forceinline__ int bpp_row_fast(const BppWarp &w, const float *__restrict__ R,
                                            int64_t row, int k, float *__restrict__ X, int warm,
                                            int max_piv, bool *failed_numeric_out,
                                            bool *failed_cap_out) {
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const float *Qh = w.Qh, *Ql = w.Ql;
  const float *Gh = w.Gh, *Gl = w.Gl;
  const bool have_q = w.have_q;
  float *Lf = w.Lf;
  float *bh = w.bh, *bl = w.bl;  // right-hand side pair
  float *dv = w.dv;              // corrections
  float *vh = w.vh, *vl = w.vl;  // solution pairs: F order (x_F) or B order (Q_BB^-1 z_B)
  int *Fl = w.Fl, *Bl = w.Bl;
  float *xa = w.xa, *rsf = w.rsf;
  const int ldl = w.ldl, kh = w.kh;
  float rf[KT], xh[KT], xl[KT], yh[KT], yl[KT], tauf[KT];
  bool pas[KT], dead[KT];
  bool any = false;
#pragma unroll
  for (int t = 0; t < KT; ++t) {
    const int j = lane + 32 * t;
    rf[t] = j < k ? R[row * k + j] : 0.f;
    if (j < k) rsf[j] = rf[t];
    dead[t] = !(j < k && ((w.live[j >> 5] >> (j & 31)) & 1u));
    pas[t] = warm && !dead[t] && X[row * k + j] > 0.f;
    any |= pas[t];
    xh[t] = xl[t] = 0.f;
    yh[t] = -rf[t];
    yl[t] = 0.f;
    tauf[t] = kBppYTolF * fabsf(rf[t]);
  }
  __syncwarp();
  // z = G^{-1} r (a pair), shared by every exchange of this right-hand side
  // that takes the Q route; formed on the first such exchange (or first of
  // all, for warm 2)
  float zh[KT], zl[KT];
  bool have_z = false;
  auto form_z = [&]() {
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      // z_j = sum_l (Qh + Ql)_lj r_l, r_l an FP32 value
      const int j = lane + 32 * t;
      float hi = 0.f, lo = 0.f;
      if (j < k)
        for (int l = 0; l < k; ++l) {
          const float rl = rsf[l];
          two_fma_acc(Qh[l * k + j], rl, hi, lo);
          lo = fmaf(Ql[l * k + j], rl, lo);
        }
      zh[t] = __fadd_rn(hi, lo);
      zl[t] = __fsub_rn(lo, __fsub_rn(zh[t], hi));
    }
    have_z = true;
  };
  if (warm == 2 && have_q) {
    // the solution is unique (G positive definite), so the starting set
    // changes only the number of exchanges
    form_z();
    any = false;
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      pas[t] = !dead[t] && lane + 32 * t < k && zh[t] > 0.f;
      any |= pas[t];
    }
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
        if (j < k && AUNMF_BOUND(posf[t] < k && posb[t] < k, AUNMF_CHECK_BPP_LIST)) {
          if (pas[t]) Fl[posf[t]] = j; else Bl[posb[t]] = j;
        }
      }
      __syncwarp();
      const bool direct = nf <= nb || !have_q;
      if (direct) {
        // ---- direct: G_FF x_F = r_F; (vh, vl)[0..nf) end as x_F in F order
        if (nf > kh) { failed_numeric = true; break; }
#pragma unroll
        for (int t = 0; t < KT; ++t)
          if (pas[t]) {
            bh[posf[t]] = rf[t];
            bl[posf[t]] = 0.f;
          }
        __syncwarp();
        // a system the FP32 solve cannot finish (an ill-conditioned G_FF)
        // sends the row to the FP64 fallback kernel
        if (!solve_mixed(Gh, Gl, k, Fl, nf, bh, bl, Lf, ldl, dv, vh, vl, lane)) {
          failed_numeric = true;
          break;
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          xh[t] = pas[t] ? vh[posf[t]] : 0.f;
          xl[t] = pas[t] ? vl[posf[t]] : 0.f;
        }
      } else {
        // ---- through Q = G^{-1} and z = Q r: the constrained solution has
        // Q_BB y_B = -z_B and x_F = z_F + Q_FB y_B (y_F = 0, x_B = 0)
        if (!have_z) form_z();
#pragma unroll
        for (int t = 0; t < KT; ++t)
          if (!pas[t] && lane + 32 * t < k) {
            bh[posb[t]] = zh[t];
            bl[posb[t]] = zl[t];
          }
        __syncwarp();
        // (vh, vl)[0..nb) = Q_BB^{-1} z_B = -y_B
        if (!solve_mixed(Qh, Ql, k, Bl, nb, bh, bl, Lf, ldl, dv, vh, vl, lane)) {
          failed_numeric = true;
          break;
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          const int j = lane + 32 * t;
          xh[t] = xl[t] = 0.f;
          if (j < k && pas[t]) {
            float h, l;
            pair_dot(Qh, Ql, k, Bl, nb, j, vh, vl, h, l);
            xh[t] = zh[t];
            xl[t] = zl[t];
            pair_add(xh[t], xl[t], -h, -l);
          }
          if (j < k && !pas[t]) {
            yh[t] = -vh[posb[t]];
            yl[t] = -vl[posb[t]];
          }
        }
        __syncwarp();
        // x_F in F order for the tolerance scales (and the refinement)
#pragma unroll
        for (int t = 0; t < KT; ++t)
          if (pas[t]) {
            vh[posf[t]] = xh[t];
            vl[posf[t]] = xl[t];
          }
        __syncwarp();
        if (w.refine) {
          // one step of iterative refinement of the route through Q: the
          // passive system's residual rho_F = r_F - G_FF x_F, its correction
          // through the same route (z' = Q [rho_F; 0], rho rounded to FP32:
          // a correction needs no more), and y_B = G_BF x_F - r_B formed
          // directly; the error of the route drops from ~cond u to ~(cond
          // u)^2.  The sums with G take its FP32 pair: ~2^-44 of the terms,
          // on a par with the ~1e-14 to which G itself is formed.  r in FP32
          // (rsf) is no longer needed: z is formed, and a direct solve takes
          // r from the lanes' registers.
#pragma unroll
          for (int t = 0; t < KT; ++t) {
            const int j = lane + 32 * t;
            float rho = 0.f;
            if (j < k && pas[t]) {
              float h, l, rh = rf[t], rl = 0.f;
              pair_dot(Gh, Gl, k, Fl, nf, j, vh, vl, h, l);
              pair_add(rh, rl, -h, -l);
              rho = __fadd_rn(rh, rl);
            }
            if (j < k) rsf[j] = rho;
          }
          __syncwarp();
          // z' = Q rho in plain FP32 with Q's high half: z' only corrects an
          // error of ~cond u_pair in x, so its own relative error (~2^-24 per
          // term) leaves the refined x far below FP32 resolution, at a quarter
          // of the pair form's instructions (the residual rho above is the
          // part that needs the pairs)
          float zrh[KT], zrl[KT];
#pragma unroll
          for (int t = 0; t < KT; ++t) {
            const int j = lane + 32 * t;
            float hi = 0.f;
            if (j < k)
              for (int l = 0; l < k; ++l) hi = fmaf(Qh[l * k + j], rsf[l], hi);
            zrh[t] = hi;
            zrl[t] = 0.f;
          }
#pragma unroll
          for (int t = 0; t < KT; ++t)
            if (!pas[t] && lane + 32 * t < k) {
              bh[posb[t]] = zrh[t];
              bl[posb[t]] = zrl[t];
            }
          __syncwarp();
          if (!solve_mixed(Qh, Ql, k, Bl, nb, bh, bl, Lf, ldl, dv, vh, vl, lane)) {
            failed_numeric = true;
            break;
          }
          __syncwarp();
#pragma unroll
          for (int t = 0; t < KT; ++t) {
            const int j = lane + 32 * t;
            if (j < k && pas[t]) {
              float h, l, ch = zrh[t], cl = zrl[t];
              pair_dot(Qh, Ql, k, Bl, nb, j, vh, vl, h, l);
              pair_add(ch, cl, -h, -l);
              pair_add(xh[t], xl[t], ch, cl);
            }
          }
          __syncwarp();
#pragma unroll
          for (int t = 0; t < KT; ++t)
            if (pas[t]) {
              vh[posf[t]] = xh[t];
              vl[posf[t]] = xl[t];
            }
          __syncwarp();
#pragma unroll
          for (int t = 0; t < KT; ++t) {
            const int j = lane + 32 * t;
            if (j < k && !pas[t]) {
              float h, l;
              pair_dot(Gh, Gl, k, Fl, nf, j, vh, vl, h, l);
              yh[t] = h;
              yl[t] = l;
              pair_add(yh[t], yl[t], -rf[t], 0.f);
            }
          }
        }
      }
      // ---- active set: y = G_BF x_F - r_B (direct route; the Q route has
      // it already) and the tolerance scale |r_j| + sum |G_jF x_F|, in FP32
#pragma unroll
      for (int t = 0; t < KT; ++t)
        if (pas[t]) xa[posf[t]] = fabsf(__fadd_rn(xh[t], xl[t]));
      __syncwarp();
#pragma unroll
      for (int t = 0; t < KT; ++t) {
        const int j = lane + 32 * t;
        if (j >= k) continue;
        if (pas[t]) {
          yh[t] = yl[t] = 0.f;
          tauf[t] = 0.f;
        } else {
          float mag = fabsf(rf[t]);
          for (int a = 0; a < nf; ++a) mag = fmaf(fabsf(Gh[Fl[a] * k + j]), xa[a], mag);
          tauf[t] = kBppYTolF * mag;
          if (direct) {
            float h, l;
            pair_dot(Gh, Gl, k, Fl, nf, j, vh, vl, h, l);
            yh[t] = h;
            yl[t] = l;
            pair_add(yh[t], yl[t], -rf[t], 0.f);
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
      const bool xneg = xh[t] < 0.f || (xh[t] == 0.f && xl[t] < 0.f);
      inf[t] = j < k && (pas[t] ? xneg : (!dead[t] && __fadd_rn(yh[t], yl[t]) < -tauf[t]));
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
  // a row handed to the fallback gets the passive set it had reached (1 on
  // it, 0 elsewhere), which the fallback starts from: in the first
  // iteration, whose previous iterate is the random start, that saves the
  // fallback most of its exchanges (the fallback always overwrites the row)
#pragma unroll
  for (int t = 0; t < KT; ++t) {
    const int j = lane + 32 * t;
    if (j < k) X[row * k + j] = failed_numeric ? (pas[t] ? 1.f : 0.f) : __fadd_rn(xh[t], xl[t]);
  }
  *failed_numeric_out = failed_numeric;
  *failed_cap_out = failed_cap;
  return it;
}

// Fallback for the rows the fast kernel flagged (a non-positive pivot in a
// k/2-sized factorisation, or a passive set too large for it while Q is not
// in use because G is not numerically positive definite or is badly
// conditioned): the same exchange rule, from the support of the row's
// previous iterate when warm (else from the empty passive set), every
// passive system solved by a Cholesky factorisation of G_FF of any size.
template <int KT>
__device__ __forceinline__ int bpp_row_direct(const double *__restrict__ G, double *L, double *v,
                                              double *rs, int *Fl, const float *__restrict__ R,
                                              int64_t row, int k, float *__restrict__ X, int warm,
                                              int max_piv, bool *failed_numeric_out,
                                              bool *failed_cap_out) {
  const int lane = threadIdx.x & 31;
  const int ldl = k | 1;
  const unsigned lt_mask = (1u << lane) - 1u;
  double gmax = 0.0;
  for (int i = 0; i < k; ++i) gmax = fmax(gmax, G[i * k + i]);
  double rr[KT], x[KT], y[KT], tau[KT];
  bool pas[KT], dead[KT];
  int it = 0;
  bool failed_numeric = false, failed_cap = false;
  // a warm start whose first factorisation fails is retried from the empty
  // passive set
  for (int attempt = warm ? 0 : 1; attempt < 2; ++attempt) {
  bool any = false;
#pragma unroll
  for (int t = 0; t < KT; ++t) {
    const int j = lane + 32 * t;
    rr[t] = j < k ? (double)R[row * k + j] : 0.0;
    if (j < k) rs[j] = rr[t];
    dead[t] = !(j < k && G[j * k + j] > kDead * gmax);
    pas[t] = attempt == 0 && !dead[t] && X[row * k + j] > 0.f;
    any |= pas[t];
    x[t] = 0.0;
    y[t] = -rr[t];
    tau[t] = kBppYTol * fabs(rr[t]);
  }
  __syncwarp();
  int alpha = 3, beta = k + 1;
  it = 0;
  failed_numeric = false;
  failed_cap = false;
  bool need_solve = __any_sync(0xffffffffu, any);
  for (;;) {
    if (need_solve) {
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
        if (pas[t] && AUNMF_BOUND(pos[t] < k && lane + 32 * t < k, AUNMF_CHECK_BPP_LIST))
          Fl[pos[t]] = lane + 32 * t;
      __syncwarp();
      if (!warp_cholesky([G, k](int a, int b) { return G[a * k + b]; }, Fl, nf, L, ldl, lane)) {
        failed_numeric = true;
        break;
      }
      for (int a = lane; a < nf; a += 32)
        v[a] = AUNMF_BOUND(Fl[a] >= 0 && Fl[a] < k, AUNMF_CHECK_BPP_LIST) ? rs[Fl[a]] : 0.0;
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
            const double g = G[Fl[a] * k + j] * v[a];
            s += g;
            mag += fabs(g);
          }
          y[t] = s;
          tau[t] = kBppYTol * mag;
        }
      }
      __syncwarp();
    }
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
  if (!(failed_numeric && it == 0)) break;
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
