/*
 * aunmf_oracle.c -- plain, slow, FP64 CPU oracle for alternating-updating NMF
 * (Kannan, Ballard, Park: "MPI-FAUN", arXiv:1609.09154).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only the tests, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py do.  It shares no code, header, table or helper
 * with the CUDA library.
 *
 * Every routine is written for a reader checking it against the paper by eye:
 * plain loops in double precision, no blocking, no reordering beyond what the
 * cited passage states.  OpenMP is used only on loops whose iterations are
 * independent (rows of W, columns of H), which the paper itself notes can be
 * solved independently (Sec. 5.1).
 *
 * Layouts (all row-major, double):
 *   A  m x n dense, or CSR (rowptr[m+1], colidx[nnz], val[nnz])
 *   W  m x k          H  k x n
 *   G  k x k          P_W = A H^T  m x k        P_H = W^T A  k x n
 *
 * Readings of the paper that the code takes where the text is silent or
 * ambiguous (each is also listed in the design notes):
 *   R1 (Eq. muupdate) the denominator gets + eps (eps = 1e-16 by default) so
 *      that a zero denominator cannot divide by zero.
 *   R2 (Eq. halsupdate) each column step is the exact coordinate minimiser,
 *      i.e. the correction is divided by the diagonal entry of the Gram matrix
 *      (the printed rule omits it; for H it is 1 after W is normalised).  A
 *      zero diagonal leaves that column/row unchanged.
 *   R3 (Eq. halsupdate) normalising w^i is compensated by scaling h_i by the
 *      same norm, so WH is unchanged; this is done once after the sweep, which
 *      is algebraically identical to doing it inside the sweep (the terms
 *      w^i (HH^T)_{ij} of later columns are invariant).  Zero columns are left
 *      unnormalised.
 *   R4 (Sec. 4.3) SolveBPP is block principal pivoting (Kim-He-Park /
 *      Judice-Pires): a passive index is infeasible when x_i < 0, an active
 *      one when y_i < -tau_i with tau_i = 1e-11 (|r_i| + sum_j |G_ij x_j|),
 *      the rounding scale of y_i (without it, an index with x_i = y_i = 0 at
 *      the solution can flip forever on rounding noise); full exchange with
 *      a backup counter of 3, single-index exchange (largest index) after
 *      that; the passive-set systems are solved through the normal equations
 *      by Cholesky, as the paper states.  Cold start (empty passive set).
 *      An index whose Gram diagonal is <= 1e-12 of the largest one (a zero
 *      column of the fixed factor, which ABPP can produce) is never made
 *      passive: its x is 0, as the normal equations leave it undetermined.
 *   R5 (Sec. 6.2) the relative error is measured after both updates of an
 *      iteration, directly as ||A - WH||_F / ||A||_F.
 *   R9 (Eq. halsupdate, taken as printed: hals_variant 1) the correction is
 *      not divided by the Gram diagonal, and w^i is normalised inside the
 *      sweep, before column i+1 is updated, without any rescaling of h_i.
 *   R10 (Sec. 6.2, the projected gradient as a stopping measure; the paper
 *      gives no formula) for f = 0.5 ||A - WH||_F^2 the gradient is
 *      (W H H^T - A H^T, W^T W H - W^T A); its projection keeps an entry
 *      where the factor's entry is > 0 and min(0, g) where it is 0.  The
 *      norm of the state an iteration starts from is taken with that
 *      iteration's H H^T, A H^T and the previous iteration's W^T W, W^T A;
 *      when it is <= stop_tol times the norm at the start (W0, H0), the run
 *      stops after that iteration.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MU 0
#define OR_HALS 1
#define OR_ABPP 2

#define OR_OK 0
#define OR_E_INVAL -1
#define OR_E_NOMEM -2
#define OR_E_NUMERIC -4
#define OR_E_NOCONVERGE -5

/* relative tolerance of the active-set test y_i < -tau_i (reading R4) */
#define BPP_YTOL 1e-11
/* Gram diagonal (relative to the largest) below which an index is a zero
   column and stays active (reading R4) */
#define BPP_DEAD 1e-12

/* ------------------------------------------------------------------------ */
/* Input matrix: dense row-major or CSR.                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t m, n;
  const double *dense;     /* m x n row-major, or NULL */
  const int64_t *rowptr;   /* CSR, used when dense == NULL */
  const int32_t *colidx;
  const double *val;
} or_matrix;

int or_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Gram matrices (Alg. 1 lines 3-4; Alg. 3: U = H H^T, X = W^T W)            */
/* ------------------------------------------------------------------------ */

/* G = W^T W for W m x k:  G_ij = sum_r W_ri W_rj  (r ascending) */
void or_gram_w(const double *W, int64_t m, int k, double *G) {
  for (int t = 0; t < k * k; ++t) G[t] = 0.0;
  for (int64_t r = 0; r < m; ++r)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) G[i * k + j] += W[r * k + i] * W[r * k + j];
}

/* G = H H^T for H k x n:  G_ij = sum_c H_ic H_jc */
void or_gram_h(const double *H, int k, int64_t n, double *G) {
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int64_t c = 0; c < n; ++c) s += H[i * n + c] * H[j * n + c];
      G[i * k + j] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Products with the data matrix (Alg. 1 lines 3-4; Alg. 3: V = A H^T,      */
/* Y = W^T A; dense and sparse cost in Sec. 5.2.1)                            */
/* ------------------------------------------------------------------------ */

/* P = A H^T, m x k:  P_ri = sum_c A_rc H_ic */
void or_aht(const or_matrix *A, const double *H, int k, double *P) {
  const int64_t m = A->m, n = A->n;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < m; ++r) {
    for (int i = 0; i < k; ++i) {
      double s = 0.0;
      if (A->dense) {
        for (int64_t c = 0; c < n; ++c) s += A->dense[r * n + c] * H[i * n + c];
      } else {
        for (int64_t e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e)
          s += A->val[e] * H[i * n + A->colidx[e]];
      }
      P[r * k + i] = s;
    }
  }
}

/* P = W^T A, k x n:  P_ic = sum_r W_ri A_rc  (r ascending).  The columns c
   are independent; they are split across threads in contiguous runs of 256
   so that each thread walks the rows of A in memory order. */
void or_wta(const or_matrix *A, const double *W, int k, double *P) {
  const int64_t m = A->m, n = A->n;
  if (A->dense) {
#pragma omp parallel for schedule(static)
    for (int64_t c0 = 0; c0 < n; c0 += 256) {
      const int64_t c1 = c0 + 256 < n ? c0 + 256 : n;
      for (int i = 0; i < k; ++i)
        for (int64_t c = c0; c < c1; ++c) P[i * n + c] = 0.0;
      for (int64_t r = 0; r < m; ++r)
        for (int i = 0; i < k; ++i) {
          const double w = W[r * k + i];
          for (int64_t c = c0; c < c1; ++c) P[i * n + c] += w * A->dense[r * n + c];
        }
    }
  } else {
    /* sparse: scatter each nonzero A_rc into column c of P, rows ascending
       (serial: the scatter targets of different rows overlap) */
    memset(P, 0, sizeof(double) * (size_t)k * (size_t)n);
    for (int64_t r = 0; r < m; ++r)
      for (int64_t e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e) {
        const int64_t c = A->colidx[e];
        for (int i = 0; i < k; ++i) P[i * n + c] += W[r * k + i] * A->val[e];
      }
  }
}

/* ------------------------------------------------------------------------ */
/* Multiplicative update (Sec. 4.1, Eq. muupdate)                             */
/* ------------------------------------------------------------------------ */

/* w_ij <- w_ij (A H^T)_ij / ((W H H^T)_ij + eps), all entries at once. */
void or_mu_update_w(double *W, const double *PW, const double *GH, int64_t m, int k, double eps) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < m; ++r) {
    double wold[1024];
    for (int j = 0; j < k; ++j) wold[j] = W[r * k + j];
    for (int j = 0; j < k; ++j) {
      double den = 0.0;
      for (int l = 0; l < k; ++l) den += wold[l] * GH[l * k + j];
      W[r * k + j] = wold[j] * PW[r * k + j] / (den + eps);
    }
  }
}

/* h_ij <- h_ij (W^T A)_ij / ((W^T W H)_ij + eps), all entries at once. */
void or_mu_update_h(double *H, const double *PH, const double *GW, int k, int64_t n, double eps) {
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n; ++c) {
    double hold[1024];
    for (int i = 0; i < k; ++i) hold[i] = H[i * n + c];
    for (int i = 0; i < k; ++i) {
      double den = 0.0;
      for (int l = 0; l < k; ++l) den += GW[i * k + l] * hold[l];
      H[i * n + c] = hold[i] * PH[i * n + c] / (den + eps);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* HALS (Sec. 4.2, Eq. halsupdate; readings R2, R3)                           */
/* ------------------------------------------------------------------------ */

/* Columns i = 0..k-1 of W in order, each with the current (already updated)
   values of the other columns:
     w^i <- [ w^i + ((A H^T)^i - W (H H^T)^i) / (H H^T)_ii ]_+
   then w^i <- w^i / ||w^i|| with h_i <- ||w^i|| h_i (R3).  H may be NULL, in
   which case only W is normalised (used by tests that look at W alone). */
void or_hals_update_w(double *W, const double *PW, const double *GH, int64_t m, int k,
                      double *H, int64_t n) {
  for (int i = 0; i < k; ++i) {
    const double gii = GH[i * k + i];
    if (!(gii > 0.0)) continue;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r) {
      double wg = 0.0; /* (W (HH^T)^i)_r with the current W */
      for (int l = 0; l < k; ++l) wg += W[r * k + l] * GH[l * k + i];
      const double v = W[r * k + i] + (PW[r * k + i] - wg) / gii;
      W[r * k + i] = v > 0.0 ? v : 0.0;
    }
  }
  for (int i = 0; i < k; ++i) {
    double ss = 0.0;
    for (int64_t r = 0; r < m; ++r) ss += W[r * k + i] * W[r * k + i];
    const double s = sqrt(ss);
    if (!(s > 0.0)) continue;
    for (int64_t r = 0; r < m; ++r) W[r * k + i] /= s;
    if (H)
      for (int64_t c = 0; c < n; ++c) H[i * n + c] *= s;
  }
}

/* Rows i = 0..k-1 of H in order, each with the current values:
     h_i <- [ h_i + ((W^T A)_i - (W^T W)_i H) / (W^T W)_ii ]_+
   (the division is by 1 when W has unit columns, which is the printed rule). */
void or_hals_update_h(double *H, const double *PH, const double *GW, int k, int64_t n) {
  for (int i = 0; i < k; ++i) {
    const double gii = GW[i * k + i];
    if (!(gii > 0.0)) continue;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
      double gh = 0.0; /* ((W^T W)_i H)_c with the current H */
      for (int l = 0; l < k; ++l) gh += GW[i * k + l] * H[l * n + c];
      const double v = H[i * n + c] + (PH[i * n + c] - gh) / gii;
      H[i * n + c] = v > 0.0 ? v : 0.0;
    }
  }
}

/* HALS as printed (Eq. halsupdate; reading R9).  W: columns i = 0..k-1 in
   order,
     w^i <- [ w^i + (A H^T)^i - W (H H^T)^i ]_+,   w^i <- w^i / ||w^i||,
   the normalisation taking effect before column i+1 is updated (a zero column
   stays zero); H is not touched. */
void or_hals_update_w_printed(double *W, const double *PW, const double *GH, int64_t m,
                              int k) {
  for (int i = 0; i < k; ++i) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r) {
      double wg = 0.0; /* (W (HH^T)^i)_r with the current W */
      for (int l = 0; l < k; ++l) wg += W[r * k + l] * GH[l * k + i];
      const double v = W[r * k + i] + PW[r * k + i] - wg;
      W[r * k + i] = v > 0.0 ? v : 0.0;
    }
    double ss = 0.0;
    for (int64_t r = 0; r < m; ++r) ss += W[r * k + i] * W[r * k + i];
    const double s = sqrt(ss);
    if (s > 0.0)
      for (int64_t r = 0; r < m; ++r) W[r * k + i] /= s;
  }
}

/* Rows i = 0..k-1 of H in order:  h_i <- [ h_i + (W^T A)_i - (W^T W)_i H ]_+ */
void or_hals_update_h_printed(double *H, const double *PH, const double *GW, int k, int64_t n) {
  for (int i = 0; i < k; ++i) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
      double gh = 0.0;
      for (int l = 0; l < k; ++l) gh += GW[i * k + l] * H[l * n + c];
      const double v = H[i * n + c] + PH[i * n + c] - gh;
      H[i * n + c] = v > 0.0 ? v : 0.0;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Projected gradient (Sec. 6.2; reading R10)                                  */
/* ------------------------------------------------------------------------ */

/* Squared Frobenius norm of the projected gradient of 0.5 ||A - WH||^2 at
   (W, H), from GH = H H^T, PW = A H^T, GW = W^T W, PH = W^T A:
     g = W GH - PW  (m x k),   g' = GW H - PH  (k x n),
   each entry kept where the factor's entry is > 0, else min(0, entry). */
double or_pgrad2(const double *W, const double *H, const double *GH, const double *PW,
                 const double *GW, const double *PH, int64_t m, int64_t n, int k) {
  double sw = 0.0, sh = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sw)
  for (int64_t r = 0; r < m; ++r)
    for (int j = 0; j < k; ++j) {
      double g = -PW[r * k + j];
      for (int l = 0; l < k; ++l) g += W[r * k + l] * GH[l * k + j];
      const double p = W[r * k + j] > 0.0 ? g : (g < 0.0 ? g : 0.0);
      sw += p * p;
    }
#pragma omp parallel for schedule(static) reduction(+ : sh)
  for (int64_t c = 0; c < n; ++c)
    for (int i = 0; i < k; ++i) {
      double g = -PH[i * n + c];
      for (int l = 0; l < k; ++l) g += GW[i * k + l] * H[l * n + c];
      const double p = H[i * n + c] > 0.0 ? g : (g < 0.0 ? g : 0.0);
      sh += p * p;
    }
  return sw + sh;
}

/* ------------------------------------------------------------------------ */
/* Block principal pivoting (Sec. 4.3, Eqs. single NLS and KKT; reading R4)  */
/* ------------------------------------------------------------------------ */

/* Solve G_FF z = b_F by Cholesky of the principal submatrix indexed by the
   passive set F (normal equations, as the paper does).  Returns 0, or -1 if
   a pivot is not positive. */
static int chol_solve_subset(const double *G, int k, const int *F, int nf, const double *b,
                             double *z, double *L /* k*k scratch */) {
  for (int a = 0; a < nf; ++a) {
    for (int c = 0; c <= a; ++c) {
      double s = G[F[a] * k + F[c]];
      for (int t = 0; t < c; ++t) s -= L[a * k + t] * L[c * k + t];
      if (a == c) {
        if (!(s > 0.0)) return -1;
        L[a * k + a] = sqrt(s);
      } else {
        L[a * k + c] = s / L[c * k + c];
      }
    }
  }
  double y[1024];
  for (int a = 0; a < nf; ++a) { /* L y = b_F */
    double s = b[F[a]];
    for (int t = 0; t < a; ++t) s -= L[a * k + t] * y[t];
    y[a] = s / L[a * k + a];
  }
  for (int a = nf - 1; a >= 0; --a) { /* L^T z = y */
    double s = y[a];
    for (int t = a + 1; t < nf; ++t) s -= L[t * k + a] * z[t];
    z[a] = s / L[a * k + a];
  }
  return 0;
}

/* One right-hand side: x = argmin_{x >= 0} ||C x - b|| given G = C^T C and
   r = C^T b (k <= 1024).  Returns the number of exchanges (>= 0),
   OR_E_NUMERIC for a non-positive Cholesky pivot, or OR_E_NOCONVERGE when
   max_iter exchanges did not reach the KKT point (x then holds the last
   iterate). */
int or_bpp_solve(const double *G, const double *r, int k, double *x, int max_iter) {
  if (k < 1 || k > 1024) return OR_E_INVAL;
  char passive[1024];
  double y[1024], z[1024], tau[1024];
  int F[1024];
  double *L = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k);
  if (!L) return OR_E_NOMEM;
  /* start: passive set empty, x = 0, y = G x - r = -r */
  double gmax = 0.0;
  for (int i = 0; i < k; ++i) gmax = G[i * k + i] > gmax ? G[i * k + i] : gmax;
  char dead[1024]; /* zero columns of the fixed factor: kept active */
  for (int i = 0; i < k; ++i) {
    passive[i] = 0;
    dead[i] = !(G[i * k + i] > BPP_DEAD * gmax);
    x[i] = 0.0;
    y[i] = -r[i];
    tau[i] = BPP_YTOL * fabs(r[i]);
  }
  int alpha = 3, beta = k + 1, it = 0, rc = OR_E_NOCONVERGE;
  for (;;) {
    /* infeasible set V: passive with x < 0, active with y < 0 (Eq. KKT) */
    int nv = 0, vmax = -1;
    for (int i = 0; i < k; ++i) {
      const int bad = passive[i] ? (x[i] < 0.0) : (!dead[i] && y[i] < -tau[i]);
      if (bad) { ++nv; vmax = i; }
    }
    if (nv == 0) { rc = it; break; }
    if (it >= max_iter) { rc = OR_E_NOCONVERGE; break; }
    ++it;
    if (nv < beta) { /* progress: full exchange, reset backup counter */
      beta = nv;
      alpha = 3;
      for (int i = 0; i < k; ++i)
        if (passive[i] ? (x[i] < 0.0) : (!dead[i] && y[i] < -tau[i])) passive[i] = !passive[i];
    } else if (alpha >= 1) { /* no progress yet: full exchange, spend backup */
      alpha -= 1;
      for (int i = 0; i < k; ++i)
        if (passive[i] ? (x[i] < 0.0) : (!dead[i] && y[i] < -tau[i])) passive[i] = !passive[i];
    } else { /* backup rule: exchange only the largest infeasible index */
      passive[vmax] = !passive[vmax];
    }
    /* least squares on the passive set, complementary y on the active set */
    int nf = 0;
    for (int i = 0; i < k; ++i)
      if (passive[i]) F[nf++] = i;
    if (chol_solve_subset(G, k, F, nf, r, z, L) != 0) { rc = OR_E_NUMERIC; break; }
    for (int i = 0; i < k; ++i) x[i] = 0.0;
    for (int a = 0; a < nf; ++a) x[F[a]] = z[a];
    for (int i = 0; i < k; ++i) {
      if (passive[i]) { y[i] = 0.0; tau[i] = 0.0; continue; }
      double s = -r[i], mag = fabs(r[i]);
      for (int a = 0; a < nf; ++a) {
        s += G[i * k + F[a]] * z[a];
        mag += fabs(G[i * k + F[a]] * z[a]);
      }
      y[i] = s;
      tau[i] = BPP_YTOL * mag;
    }
  }
  free(L);
  return rc;
}

/* SolveBPP for the rows of W: W_r,: = argmin_{x>=0} ||H^T x - A_r,:^T||,
   i.e. G = H H^T and right-hand side (A H^T)_r,:.  Returns the total number
   of exchanges, or the first error. */
int64_t or_bpp_update_w(double *W, const double *PW, const double *GH, int64_t m, int k,
                        int max_iter) {
  int64_t total = 0;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
  for (int64_t r = 0; r < m; ++r) {
    const int rc = or_bpp_solve(GH, PW + r * k, k, W + r * k, max_iter);
    if (rc < 0) {
#pragma omp critical
      if (!err) err = rc;
    } else {
      total += rc;
    }
  }
  return err ? err : total;
}

/* SolveBPP for the columns of H: H_:,c = argmin_{x>=0} ||W x - A_:,c||,
   i.e. G = W^T W and right-hand side (W^T A)_:,c. */
int64_t or_bpp_update_h(double *H, const double *PH, const double *GW, int k, int64_t n,
                        int max_iter) {
  int64_t total = 0;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
  for (int64_t c = 0; c < n; ++c) {
    double rhs[1024], x[1024];
    for (int i = 0; i < k; ++i) rhs[i] = PH[i * n + c];
    const int rc = or_bpp_solve(GW, rhs, k, x, max_iter);
    for (int i = 0; i < k; ++i) H[i * n + c] = x[i];
    if (rc < 0) {
#pragma omp critical
      if (!err) err = rc;
    } else {
      total += rc;
    }
  }
  return err ? err : total;
}

/* ------------------------------------------------------------------------ */
/* Objective (Eq. original NMF) and relative error (Sec. 6.2; reading R5)   */
/* ------------------------------------------------------------------------ */

double or_norm2_a(const or_matrix *A) {
  double s = 0.0;
  if (A->dense) {
    for (int64_t t = 0; t < A->m * A->n; ++t) s += A->dense[t] * A->dense[t];
  } else {
    for (int64_t e = 0; e < A->rowptr[A->m]; ++e) s += A->val[e] * A->val[e];
  }
  return s;
}

/* ||A - W H||_F^2 formed entry by entry (WH one row at a time). */
double or_resid2_direct(const or_matrix *A, const double *W, const double *H, int k) {
  const int64_t m = A->m, n = A->n;
  double total = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : total)
  for (int64_t r = 0; r < m; ++r) {
    double *row = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t c = 0; c < n; ++c) {
      double s = 0.0;
      for (int i = 0; i < k; ++i) s += W[r * k + i] * H[i * n + c];
      row[c] = -s;
    }
    if (A->dense) {
      for (int64_t c = 0; c < n; ++c) row[c] += A->dense[r * n + c];
    } else {
      for (int64_t e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e) row[A->colidx[e]] += A->val[e];
    }
    double s = 0.0;
    for (int64_t c = 0; c < n; ++c) s += row[c] * row[c];
    total += s;
    free(row);
  }
  return total;
}

double or_relres_direct(const or_matrix *A, const double *W, const double *H, int k) {
  return sqrt(or_resid2_direct(A, W, H, k) / or_norm2_a(A));
}

/* The same quantity from the expansion
   ||A - WH||^2 = ||A||^2 - 2 <W^T A, H> + <W^T W, H H^T>,
   given P_H = W^T A (k x n), G_W = W^T W and G_H = H H^T. */
double or_relres_trace(double norm2_a, const double *PH, const double *H, const double *GW,
                       const double *GH, int k, int64_t n) {
  double cross = 0.0, quad = 0.0;
  for (int64_t t = 0; t < (int64_t)k * n; ++t) cross += PH[t] * H[t];
  for (int t = 0; t < k * k; ++t) quad += GW[t] * GH[t];
  double r2 = norm2_a - 2.0 * cross + quad;
  if (r2 < 0.0) r2 = 0.0;
  return sqrt(r2 / norm2_a);
}

/* ------------------------------------------------------------------------ */
/* Loss 0.5 ||A - W H||_F^2 and its gradient, from the residual R = W H - A: */
/* dL/dW = R H^T, dL/dH = W^T R (definition; no Gram identities used).       */
/* ------------------------------------------------------------------------ */
double or_loss_grad(const or_matrix *A, const double *W, const double *H, int k, double *dW,
                    double *dH) {
  const int64_t m = A->m, n = A->n;
  double *R = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
  if (!R) return NAN;
  for (int64_t r = 0; r < m; ++r)
    for (int64_t c = 0; c < n; ++c) {
      double s = 0.0;
      for (int i = 0; i < k; ++i) s += W[r * k + i] * H[i * n + c];
      R[r * n + c] = s;
    }
  if (A->dense) {
    for (int64_t t = 0; t < m * n; ++t) R[t] -= A->dense[t];
  } else {
    for (int64_t r = 0; r < m; ++r)
      for (int64_t e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e) R[r * n + A->colidx[e]] -= A->val[e];
  }
  double loss = 0.0;
  for (int64_t t = 0; t < m * n; ++t) loss += R[t] * R[t];
  loss *= 0.5;
  if (dW)
    for (int64_t r = 0; r < m; ++r)
      for (int i = 0; i < k; ++i) {
        double s = 0.0;
        for (int64_t c = 0; c < n; ++c) s += R[r * n + c] * H[i * n + c];
        dW[r * k + i] = s;
      }
  if (dH)
    for (int i = 0; i < k; ++i)
      for (int64_t c = 0; c < n; ++c) {
        double s = 0.0;
        for (int64_t r = 0; r < m; ++r) s += W[r * k + i] * R[r * n + c];
        dH[i * n + c] = s;
      }
  free(R);
  return loss;
}

/* One row of dL/dW and one column of dL/dH from the same definitions, for
   checks on matrices too large for or_loss_grad:
     (dL/dW)_r,: = sum_c R_rc H_:,c^T,   (dL/dH)_:,c = sum_r W_r,:^T R_rc,
   with R_rc = (W H)_rc - A_rc formed entry by entry. */
void or_grad_w_row(const or_matrix *A, const double *W, const double *H, int k, int64_t r,
                   double *out) {
  const int64_t n = A->n;
  for (int i = 0; i < k; ++i) out[i] = 0.0;
  for (int64_t c = 0; c < n; ++c) {
    double wh = 0.0;
    for (int i = 0; i < k; ++i) wh += W[r * k + i] * H[i * n + c];
    const double R = wh - A->dense[r * n + c];
    for (int i = 0; i < k; ++i) out[i] += R * H[i * n + c];
  }
}

void or_grad_h_col(const or_matrix *A, const double *W, const double *H, int k, int64_t c,
                   double *out) {
  const int64_t m = A->m, n = A->n;
  for (int i = 0; i < k; ++i) out[i] = 0.0;
  for (int64_t r = 0; r < m; ++r) {
    double wh = 0.0;
    for (int i = 0; i < k; ++i) wh += W[r * k + i] * H[i * n + c];
    const double R = wh - A->dense[r * n + c];
    for (int i = 0; i < k; ++i) out[i] += W[r * k + i] * R;
  }
}

/* ------------------------------------------------------------------------ */
/* AU-NMF driver (Alg. 1)                                                     */
/* ------------------------------------------------------------------------ */

/* Runs up to `iters` iterations of Alg. 1 from (W0, H0); W0 is ignored by ABPP
   (the paper initialises only H).  relres[t] is ||A - WH|| / ||A|| after
   iteration t's two updates.  hals_variant 1 takes Eq. halsupdate as printed
   (reading R9).  pgrad (may be NULL) receives, per iteration, the norm of the
   projected gradient of the state the iteration starts from (reading R10);
   with stop_tol > 0 the run ends after the first iteration whose entry is
   <= stop_tol times pgrad[0].  *iters_done (may be NULL) is the number of
   iterations run.  Returns OR_OK, or the first error; *pivots (may be NULL)
   receives the total number of BPP exchanges. */
int or_nmf_run_ex(const or_matrix *A, int k, int algo, int iters, const double *W0,
                  const double *H0, double *W, double *H, double *relres, double mu_eps,
                  int bpp_max_iter, int64_t *pivots, int hals_variant, double stop_tol,
                  double *pgrad, int *iters_done) {
  const int64_t m = A->m, n = A->n;
  if (k < 1 || k > 1024 || iters < 0 || algo < 0 || algo > 2) return OR_E_INVAL;
  if (hals_variant < 0 || hals_variant > 1 || !(stop_tol >= 0.0)) return OR_E_INVAL;
  const int track = pgrad != NULL || stop_tol > 0.0;
  double *GH = (double *)malloc(sizeof(double) * (size_t)k * k);
  double *GW = (double *)malloc(sizeof(double) * (size_t)k * k);
  double *PW = (double *)malloc(sizeof(double) * (size_t)m * k);
  double *PH = (double *)malloc(sizeof(double) * (size_t)k * n);
  if (!GH || !GW || !PW || !PH) { free(GH); free(GW); free(PW); free(PH); return OR_E_NOMEM; }
  if (W != W0) {
    if (algo == OR_ABPP || !W0) memset(W, 0, sizeof(double) * (size_t)m * k);
    else memcpy(W, W0, sizeof(double) * (size_t)m * k);
  }
  if (H != H0) memcpy(H, H0, sizeof(double) * (size_t)k * n);
  if (track) {
    /* W^T W and W^T A of the starting W, for the first iteration's measure */
    or_gram_w(W, m, k, GW);
    or_wta(A, W, k, PH);
  }
  int64_t piv = 0;
  int rc = OR_OK, done = 0;
  double pg0 = 0.0;
  for (int t = 0; t < iters && rc == OR_OK; ++t) {
    /* Alg. 1 line 3: update W using H H^T and A H^T */
    or_gram_h(H, k, n, GH);
    or_aht(A, H, k, PW);
    double pg = 0.0;
    if (track) {
      pg = sqrt(or_pgrad2(W, H, GH, PW, GW, PH, m, n, k));
      if (t == 0) pg0 = pg;
      if (pgrad) pgrad[t] = pg;
    }
    if (algo == OR_MU) {
      or_mu_update_w(W, PW, GH, m, k, mu_eps);
    } else if (algo == OR_HALS) {
      if (hals_variant == 1) or_hals_update_w_printed(W, PW, GH, m, k);
      else or_hals_update_w(W, PW, GH, m, k, H, n);
    } else {
      const int64_t p = or_bpp_update_w(W, PW, GH, m, k, bpp_max_iter);
      if (p < 0) rc = (int)p; else piv += p;
    }
    /* Alg. 1 line 4: update H using W^T W and W^T A */
    or_gram_w(W, m, k, GW);
    or_wta(A, W, k, PH);
    if (algo == OR_MU) {
      or_mu_update_h(H, PH, GW, k, n, mu_eps);
    } else if (algo == OR_HALS) {
      if (hals_variant == 1) or_hals_update_h_printed(H, PH, GW, k, n);
      else or_hals_update_h(H, PH, GW, k, n);
    } else {
      const int64_t p = or_bpp_update_h(H, PH, GW, k, n, bpp_max_iter);
      if (p < 0 && rc == OR_OK) rc = (int)p; else if (p >= 0) piv += p;
    }
    if (relres) relres[t] = or_relres_direct(A, W, H, k);
    done = t + 1;
    if (stop_tol > 0.0 && pg <= stop_tol * pg0) break;
  }
  if (pivots) *pivots = piv;
  if (iters_done) *iters_done = done;
  free(GH); free(GW); free(PW); free(PH);
  return rc;
}

/* Alg. 1 for exactly `iters` iterations with the default readings. */
int or_nmf_run(const or_matrix *A, int k, int algo, int iters, const double *W0,
               const double *H0, double *W, double *H, double *relres, double mu_eps,
               int bpp_max_iter, int64_t *pivots) {
  return or_nmf_run_ex(A, k, algo, iters, W0, H0, W, H, relres, mu_eps, bpp_max_iter, pivots, 0,
                       0.0, NULL, NULL);
}
