/*
 * aunmf.h -- C ABI of the GB300 (sm_103a) alternating-updating NMF library.
 *
 * Problem (Kannan, Ballard, Park, arXiv:1609.09154, Eq. "original NMF"):
 *     min_{W >= 0, H >= 0} || A - W H ||_F,   A m x n,  W m x k,  H k x n.
 * Solved by Alg. 1 (AU-NMF): repeat { update W from H H^T and A H^T;
 * update H from W^T W and W^T A } with one of three local updates:
 * MU (Sec. 4.1, Eq. muupdate), HALS (Sec. 4.2, Eq. halsupdate) or ANLS with
 * block principal pivoting (Sec. 4.3, SolveBPP).
 *
 * Conventions for every entry point:
 *   - All matrices are row-major float32 unless stated; W is m x k, H is k x n
 *     (the paper's shapes).  Pointers marked [device] must be CUDA device (or
 *     managed) memory on the handle's device; [host] pointers are host memory.
 *   - The caller owns every buffer it passes; the library never frees them.
 *     The handle owns its workspace (grown on demand, freed by
 *     aunmf_destroy).  Nothing is retained past a call except the workspace.
 *   - All work is enqueued on the handle's stream.  Entry points that return
 *     host results (relres, info, loss) synchronise that stream before
 *     returning; the step-level entry points (aunmf_gram_*, aunmf_aht, ...)
 *     do not synchronise.
 *   - Every call returns AUNMF_OK (0) or a negative status code; no C++
 *     exception crosses this boundary.  aunmf_strerror() names a code.
 *   - Rank limits: 1 <= k <= AUNMF_K_MAX; ABPP needs k <= AUNMF_BPP_K_MAX.
 */
#ifndef AUNMF_H
#define AUNMF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define AUNMF_OK 0
#define AUNMF_E_INVAL -1       /* bad argument: null pointer, k out of range, bad sizes */
#define AUNMF_E_NOMEM -2       /* workspace allocation failed */
#define AUNMF_E_CUDA -3        /* a CUDA runtime call failed (see aunmf_last_cuda_error) */
#define AUNMF_E_NUMERIC -4     /* non-finite value, or a non-positive Cholesky pivot in BPP */
#define AUNMF_E_NOCONVERGE -5  /* BPP hit its pivot cap on some right-hand side (results written) */
#define AUNMF_E_TIMEOUT -6     /* a bounded device-side wait expired */
#define AUNMF_E_UNSUPPORTED -7 /* valid request that the library does not implement */

/* ---- algorithms and precisions ---------------------------------------- */
#define AUNMF_MU 0   /* Sec. 4.1, Eq. muupdate */
#define AUNMF_HALS 1 /* Sec. 4.2, Eq. halsupdate */
#define AUNMF_ABPP 2 /* Sec. 4.3, SolveBPP on each row of W / column of H */

#define AUNMF_FP32 0 /* products with A on FP32 CUDA cores (FMA), FP32 accumulation */
#define AUNMF_TF32 1 /* products with A on tensor cores (tcgen05 kind::tf32), FP32 accumulation */
#define AUNMF_BF16 2 /* products with A on tensor cores from a BF16 copy of A, FP32 accumulation */

#define AUNMF_K_MAX 512
#define AUNMF_BPP_K_MAX 64

typedef struct aunmf_handle aunmf_handle;

/* Input matrix A (nonnegative, Eq. original NMF).  Exactly one form is set:
 *   dense: dense != NULL, row-major m x n, leading dimension lda >= n
 *          (elements), 16-byte aligned base and lda % 4 == 0 for the tensor
 *          paths.  [device]
 *   CSR:   dense == NULL; rowptr[m+1] (int64), colidx[nnz] (int32, sorted
 *          within a row), val[nnz] (float32).  [device]
 * Sizes use int64 throughout (the dense configurations exceed 2^31 entries). */
typedef struct {
  int64_t m, n;
  const float *dense;
  int64_t lda;
  const int64_t *rowptr;
  const int32_t *colidx;
  const float *val;
  int64_t nnz;
} aunmf_matrix;

/* Options (zero-initialised struct = defaults). */
typedef struct {
  int prec;           /* AUNMF_FP32 (default) / AUNMF_TF32 / AUNMF_BF16 */
  double mu_eps;      /* MU: added to the denominator of Eq. muupdate; 0 -> 1e-16 */
  int bpp_max_pivots; /* ABPP: exchange cap per right-hand side; 0 -> 10*k */
  int use_graph;      /* 1: capture one iteration as a CUDA graph and replay it */
  int profile;        /* 1: time product / update / Gram phases with CUDA events */
  int hals_variant;   /* HALS: 0 = exact coordinate steps, normalisation compensated in H;
                         1 = Eq. halsupdate as printed (see aunmf_run) */
  double stop_tol;    /* > 0: stop on the projected gradient (see aunmf_run); 0 = off */
  int validate;       /* 1: before the run, check that A >= 0 and finite (Sec. 2 poses NMF
                         for a nonnegative A), that a CSR A is well formed (rowptr from 0
                         to nnz and nondecreasing; column indices in [0, n) and increasing
                         within a row), and that W0 (MU, HALS) and H0 are >= 0 and finite;
                         any violation returns AUNMF_E_INVAL before other kernels read the
                         input.  Costs one pass over A (over the host link for a pinned
                         host A); 0 = the caller vouches for its input. */
  int bpp_cold_start; /* ABPP: 1 = every BPP solve starts from x = 0 (all indices active);
                         0 = from the previous iterate's support, the first iteration from
                         the signs of the unconstrained solution.  Each subproblem has one
                         solution when its Gram is positive definite, so both reach the
                         same x (to rounding); warm starts take fewer exchanges. */
} aunmf_options;

/* Per-call report, filled when the pointer is non-NULL. */
typedef struct {
  int64_t bpp_pivots;       /* total BPP exchanges over all right-hand sides and iterations */
  int64_t bpp_nonconverged; /* right-hand sides that hit the pivot cap */
  int64_t bpp_numeric;      /* right-hand sides with a non-positive Cholesky pivot */
  int iters_done;
  float ms_total;           /* device time of the whole call (CUDA events) */
  /* profile == 1 only: summed device time and launch count per phase */
  float ms_aht, ms_wta, ms_update, ms_gram, ms_other;
  int n_aht, n_wta;
  int64_t launches;         /* kernels this call launched (graph replays counted per kernel) */
  int tuned_bpp_warps;      /* aunmf_run_batched: autotuned BPP work tile (warps per block, */
  int tuned_bpp_rows;       /*   rows per warp per item)                                    */
  int64_t bpp_redone;       /* right-hand sides the fast BPP solver handed to the direct    */
                            /*   (cold-start, full-size Cholesky) fallback                  */
  double pgrad_first;       /* stop_tol > 0: projected-gradient norm of (W0, H0) ...        */
  double pgrad_last;        /*   ... and of the state the last iteration started from       */
  int tuned_gemm_stages_aht; /* aunmf_run_batched: autotuned pipeline stages of the grouped */
  int tuned_gemm_stages_wta; /*   A H^T and W^T A products (0: as many as fit)              */
} aunmf_info;

/* ---- handle -------------------------------------------------------------- */

/* Creates a handle bound to the current CUDA device and `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *h receives the handle. */
int aunmf_create(aunmf_handle **h, void *stream);
/* Rebinds the handle to another stream of the same device. */
int aunmf_set_stream(aunmf_handle *h, void *stream);
/* Frees the workspace and the handle (synchronises its stream first). */
int aunmf_destroy(aunmf_handle *h);

const char *aunmf_strerror(int code);
/* The last CUDA error string seen by this handle ("" if none). */
const char *aunmf_last_cuda_error(aunmf_handle *h);

/* ---- whole runs ---------------------------------------------------------- */

/* Alg. 1: `iters` iterations of AU-NMF with local update `algo` from (W0, H0).
 *   A        input matrix (dense or CSR) [device]
 *   W0, H0   initial factors, m x k and k x n [device]; W0 is read by MU and
 *            HALS only (ABPP starts from H0, as Alg. 1 initialises only H)
 *   W, H     outputs, m x k and k x n [device]; may alias W0, H0
 *   relres   [host] array of `iters` doubles (may be NULL): after iteration t's
 *            two updates, ||A - W H||_F / ||A||_F (Sec. 6.2), evaluated as
 *            sqrt(||A||^2 - 2 <W^T A, H> + <W^T W, H H^T>) / ||A|| with FP64
 *            reductions
 *   opt      options (NULL = defaults); info: report (may be NULL)
 * HALS takes each column step as the exact coordinate minimiser (the
 * correction divided by the Gram diagonal) and normalises W's columns after
 * the sweep while scaling H's rows by the same norms, which leaves W H
 * unchanged (Eq. halsupdate).  With opt->hals_variant = 1 it takes Eq.
 * halsupdate as printed instead: no division by the diagonal, and each
 * column of W normalised before the next is updated, H not rescaled (the W
 * sweep is then one cooperative launch with a grid-wide norm per column;
 * no CUDA graph).
 * Stopping (Sec. 6.2 names the projected gradient as a stopping measure):
 * with opt->stop_tol > 0 each iteration also forms ||P(grad f)||_F for the
 * state it starts from, f = 0.5 ||A - WH||_F^2, grad f = (W HH^T - AH^T,
 * W^T W H - W^T A), P keeping an entry where the factor's entry is > 0 and
 * min(0, entry) where it is 0 (FP32 entries, FP64 sum); the run ends after
 * the first iteration whose value is <= stop_tol times that of (W0, H0).
 * info->iters_done is then the iterations run, and relres holds that many
 * entries.  Synchronises the stream. */
int aunmf_run(aunmf_handle *h, const aunmf_matrix *A, int k, int algo, int iters,
              const float *W0, const float *H0, float *W, float *H, double *relres,
              const aunmf_options *opt, aunmf_info *info);

/* Same as aunmf_run with every array in HOST memory (A dense only): copies A,
 * W0, H0 to the device, runs, copies W, H back.  The device copies live in
 * the handle's workspace.  With opt->prec TF32 or BF16 and A in page-locked
 * host memory (cudaHostAlloc / cudaHostRegister, e.g. torch's pin_memory),
 * A is not copied: the run's one-off layout pass reads it over the host link
 * and writes the rounded device copies that the products stream, so A's
 * device footprint and staging copy disappear (A must stay valid and
 * unchanged until the call returns).  Otherwise A is copied first. */
int aunmf_run_host(aunmf_handle *h, const float *A, int64_t m, int64_t n, int64_t lda, int k,
                   int algo, int iters, const float *W0, const float *H0, float *W, float *H,
                   double *relres, const aunmf_options *opt, aunmf_info *info);

/* Many independent problems at once: `count` runs of Alg. 1 with ANLS/BPP
 * (Sec. 4.3), problem p on dense A[p] (m_p x n_p [device]) with rank k[p]
 * (1..64), from H0[p] (k_p x n_p [device]; W starts at 0 as in Alg. 1), into
 * W[p] (m_p x k_p) and H[p] (k_p x n_p) [device].  A, k, W0, H0, W, H are
 * HOST arrays of `count` entries (W0 is unused and may be NULL).
 * Every phase of an iteration -- both tensor-core products, the Gram
 * matrices, G^{-1}, the BPP solves, the residual -- is one launch covering
 * all problems; one iteration is captured as a CUDA graph (use_graph) and
 * replayed.  The BPP work tile and the grouped products' pipeline depth are
 * autotuned on the first call for a batch signature (count, sum m, sum n,
 * max k, precision), each candidate timed on the device, and cached in the
 * handle; info reports the choices.
 * Requires algo == AUNMF_ABPP and opt->prec TF32 or BF16.
 * relres [host] count x iters, row p = problem p (may be NULL).  Synchronises. */
int aunmf_run_batched(aunmf_handle *h, int count, const aunmf_matrix *A, const int *k, int algo,
                      int iters, const float *const *W0, const float *const *H0, float *const *W,
                      float *const *H, double *relres, const aunmf_options *opt,
                      aunmf_info *info);

/* ---- single steps of Alg. 1 (for step-by-step checks and custom drivers) -- */

/* G = W^T W (k x k) for W m x k [device in/out] (Alg. 1 line 4; Alg. 3 X). */
int aunmf_gram_w(aunmf_handle *h, const float *W, int64_t m, int k, float *G);
/* G = H H^T (k x k) for H k x n [device in/out] (Alg. 1 line 3; Alg. 3 U). */
int aunmf_gram_h(aunmf_handle *h, const float *H, int k, int64_t n, float *G);
/* P = A H^T (m x k) [device] (Alg. 1 line 3; Alg. 3 V), in precision `prec`. */
int aunmf_aht(aunmf_handle *h, const aunmf_matrix *A, const float *H, int k, int prec, float *P);
/* P = W^T A (k x n) [device] (Alg. 1 line 4; Alg. 3 Y), in precision `prec`. */
int aunmf_wta(aunmf_handle *h, const aunmf_matrix *A, const float *W, int k, int prec, float *P);

/* Local update of W (Alg. 1 line 3) in place: W m x k, PW = A H^T (m x k),
 * GH = H H^T (k x k) [device].  MU: Eq. muupdate with eps; HALS: the
 * column sweep of Eq. halsupdate, then unit-normalised columns with H's rows
 * (H k x n, may be NULL) scaled by the norms; ABPP: each row of W solves
 * SolveBPP(GH, row of PW) to FP64 accuracy from a cold start (GH widened from FP32;
 * aunmf_run forms its Grams in FP64 instead), and the call synchronises and
 * returns AUNMF_E_NUMERIC / AUNMF_E_NOCONVERGE if a row failed (W still
 * written).  eps <= 0 selects 1e-16. */
int aunmf_update_w(aunmf_handle *h, int algo, float *W, const float *PW, const float *GH,
                   int64_t m, int k, float *H, int64_t n, double eps);
/* Local update of H (Alg. 1 line 4) in place: H k x n, PH = W^T A (k x n),
 * GW = W^T W [device].  MU / HALS row sweep / ABPP on each column (ABPP
 * reports failures as aunmf_update_w does). */
int aunmf_update_h(aunmf_handle *h, int algo, float *H, const float *PH, const float *GW,
                   int k, int64_t n, double eps);

/* Batched NLS (Sec. 4.3, Eqs. single NLS and KKT): for each of `nrhs` rows r
 * of R (nrhs x k, float32 [device]) solves x = argmin_{x>=0} ||C x - b|| given
 * G = C^T C (k x k float32 [device]) and r = C^T b, to FP64 accuracy (FP32
 * solves refined with FP32-pair residuals, FP64 where they cannot finish); writes x as row r
 * of X (nrhs x k float32 [device]).  pivots/nonconv (may be NULL) [host]
 * receive the total exchanges and the number of right-hand sides that hit
 * max_pivots (0 -> 10*k).  Returns AUNMF_E_NOCONVERGE / AUNMF_E_NUMERIC if
 * any right-hand side failed (X still written).  Synchronises. */
int aunmf_nls_bpp(aunmf_handle *h, const float *G, const float *R, int64_t nrhs, int k, float *X,
                  int max_pivots, int64_t *pivots, int64_t *nonconv);

/* ||A - W H||_F / ||A||_F (Sec. 6.2) by the trace expansion with FP64
 * reductions; W m x k, H k x n [device]; *relres [host].  Synchronises.
 * Returns AUNMF_E_TIMEOUT if a bounded device wait of the product gave up. */
int aunmf_relres(aunmf_handle *h, const aunmf_matrix *A, const float *W, const float *H, int k,
                 double *relres);

/* ---- differentiable objective -------------------------------------------- */

/* L = 0.5 ||A - W H||_F^2, the squared objective of Eq. (original NMF),
 * halved, evaluated as 0.5 (||A||^2 - 2 <W^T A, H> + <W^T W, H H^T>) with the
 * products in precision `prec` and FP64 reductions.
 *   A [device], W m x k and H k x n [device]
 *   loss   [device] one double (written, not synchronised)
 *   WtA    [device] k x n, may be NULL: receives W^T A for aunmf_loss_bwd
 * The call enqueues work on the handle's stream and returns. */
int aunmf_loss_fwd(aunmf_handle *h, const aunmf_matrix *A, int k, const float *W, const float *H,
                   int prec, double *loss, float *WtA);

/* Gradient of L: dW = g (W H H^T - A H^T) (m x k) and dH = g (W^T W H - W^T A)
 * (k x n) -- the two terms whose ratio is Eq. (muupdate) -- with g = *grad_out
 * read on the device (grad_out NULL: g = 1).  WtA (k x n, from
 * aunmf_loss_fwd) may be NULL, in which case W^T A is recomputed.  dW or dH
 * may be NULL to skip that gradient.  All pointers [device]; enqueues only. */
int aunmf_loss_bwd(aunmf_handle *h, const aunmf_matrix *A, int k, const float *W, const float *H,
                   int prec, const float *WtA, const float *grad_out, float *dW, float *dH);

/* ---- measurement ------------------------------------------------------------ */

/* The gather roof of the sparse products (Sec. 5.2.1 products with a sparse
 * A): each nonzero of A H^T (W^T A) reads the k-vector of row idx[e] of H^T
 * (W), a row at a data-dependent address, so the products are bound by how
 * fast such rows can be gathered, not by their algorithmic HBM bytes.  This
 * call times nothing itself: it enqueues a kernel that loads row idx[e] of X
 * for every e < n (the same index stream a product walks: its column or row
 * indices) with the widest loads and does nothing else; the caller times it
 * with events on `stream`.  Not a step of the method.
 *   idx    n indices in [0, rows) [device]; X rows x k, leading dimension ld
 *          floats (ld % 4 == 0, 16-byte aligned base) [device]
 *   k      1..64; sink: one float [device] (never written in practice)
 * Returns AUNMF_OK, AUNMF_E_INVAL or AUNMF_E_CUDA. */
int aunmf_probe_gather(const int32_t *idx, int64_t n, const float *X, int64_t rows, int k,
                       int64_t ld, float *sink, void *stream);

/* ---- checked build -------------------------------------------------------- */

/* The library also builds as libaunmf_check.so (compiled with -DAUNMF_CHECK;
 * paper_1609_09154_gb300/build.py, build(check=True)), the stand-in for a
 * memory checker: device code tests each index it takes from data (CSR /
 * CSC structure, sorted positions, BPP index lists, batched work items,
 * TMA coordinates) and, where one is out of range, records the site and
 * skips the access instead of faulting.  aunmf_check_status() synchronises
 * the device, stores in *site the first site recorded since the last call
 * (0 = none, else an AUNMF_CHECK_* code) and clears the record.  The normal
 * build compiles no checks: *site = -1, and no device call is made.
 * Returns AUNMF_OK, or AUNMF_E_INVAL for a null site.  The paper has no
 * counterpart; this is test support of the library. */
#define AUNMF_CHECK_SPMM_COLUMN 1  /* SpMM: a gathered row index outside the factor */
#define AUNMF_CHECK_SPMM_RANGE 2   /* SpMM: a row's nonzero range outside [0, nnz] */
#define AUNMF_CHECK_CSC 3          /* CSR -> CSC: a position or column outside its array */
#define AUNMF_CHECK_BPP_LIST 4     /* BPP: a passive / active list position outside [0, k) */
#define AUNMF_CHECK_BATCHED_ITEM 5 /* batched: a work item's rows outside its problem */
#define AUNMF_CHECK_TMA_COORD 6    /* TMA: a copy coordinate negative or not 16-byte aligned */
int aunmf_check_status(int *site);

/* ---- fault injection for tests ---------------------------------------------- */

/* Every wait of a kernel on another thread, warp or block of the same launch
 * (the tensor-core products' and the FP32 products' mbarrier waits, the
 * printed HALS sweep's grid barrier) is bounded: after ~2 s it raises the
 * call's device error flag, the kernel drains the copies and tensor-core
 * operations it has in flight, frees its tensor memory and returns, and the
 * call returns AUNMF_E_TIMEOUT with the device context still usable (the
 * step-level entry points, which do not synchronise, leave their output
 * unwritten and report nothing).  aunmf_test_inject() makes those
 * paths run on purpose, for tests, without faulting or hanging the GPU: it
 * withholds one signal so that a bounded wait runs out.  The setting is
 * process-wide and applies to every launch made after the call, until it is
 * set back to AUNMF_INJECT_NONE; it is read when a kernel is launched (a CUDA
 * graph keeps the value seen at capture).
 *   site     AUNMF_INJECT_NONE          back to normal operation
 *            AUNMF_INJECT_TC_WAIT       tensor-core products (aunmf_run,
 *              aunmf_run_batched, aunmf_aht / aunmf_wta in TF32 / BF16): the
 *              MMA warp never signals that the first accumulator chunk is
 *              ready, so the epilogue's wait runs out
 *            AUNMF_INJECT_GRID_BARRIER  printed HALS sweep (hals_variant 1):
 *              block 0 never arrives at the first grid barrier
 *            AUNMF_INJECT_NOMEM         every workspace allocation fails with
 *              AUNMF_E_NOMEM (cudaMalloc is not called); buffers a handle
 *              already holds stay usable
 *            AUNMF_INJECT_SIMT_WAIT     the TMA-fed FP32 kernel: dense FP32
 *              products with k > 32 (aunmf_run, aunmf_relres, aunmf_aht /
 *              aunmf_wta in FP32) and the Gram matrices at k >= 96 (a
 *              multiple of 4, >= 1024 rows) in every precision: thread 0
 *              never arrives on the first stage's barrier, so every thread's
 *              wait for that stage runs out
 *   wait_ms  limit of the bounded waits while `site` is set, in milliseconds
 *            of the device's maximum SM clock (<= 0: the default ~2 s);
 *            ignored for AUNMF_INJECT_NONE, which restores the default.
 * Returns AUNMF_OK, or AUNMF_E_INVAL for an unknown site or wait_ms > 60000.
 * The paper has no counterpart; this is test support of the library. */
#define AUNMF_INJECT_NONE 0
#define AUNMF_INJECT_TC_WAIT 1
#define AUNMF_INJECT_GRID_BARRIER 2
#define AUNMF_INJECT_NOMEM 3
#define AUNMF_INJECT_SIMT_WAIT 4
int aunmf_test_inject(int site, double wait_ms);

/* ---- fixed-memory variant ------------------------------------------------ */

/* G = W^T W (k x k) for W m x k [device in/out], like aunmf_gram_w, for
 * callers that cannot allocate device memory: code running while another
 * framework's memory pool owns the device (a cudaMalloc there can fail or
 * upset the pool's accounting), or code held to a fixed memory budget.  The
 * paper has no counterpart; this is a service of the library.
 *   - Allocates nothing and needs no handle: the per-block partial sums live
 *     in a static device array of 4 MiB (256 partial 64 x 64 FP32 matrices)
 *     that every GPU loading the library holds until the process exits.
 *   - k must be in 1..64 (the array's limit); larger k returns
 *     AUNMF_E_INVAL without launching anything.  m is unlimited.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream); the call
 *     only enqueues work and does not synchronise.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.  After a device reset (a new CUDA context on
 *     the device) the next call looks the address up again.
 *   - Every call on a device shares the one array.  Nothing in it needs to
 *     start at zero (each call overwrites all it reads), but calls whose GPU
 *     work overlaps in time -- e.g. on two streams -- race on it: order them
 *     on one stream or with events.
 * Returns AUNMF_OK, AUNMF_E_INVAL, AUNMF_E_CUDA or AUNMF_E_UNSUPPORTED (device
 * ordinal >= 64). */
int aunmf_gram_w_noalloc(const float *W, int64_t m, int k, float *G, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* AUNMF_H */
