// aunmf_api.cu -- the C ABI (include/aunmf.h): handle, workspace, argument
// checks, and the AU-NMF driver of Alg. 1 that enqueues the hot-path kernels.
//
// One iteration (Alg. 1 lines 3-4, with H held as Ht = H^T, n x k):
//   P_W  = A Ht                       (product, Alg. 1 line 3)
//   W    = LUC(W, P_W, G_H)           (MU / HALS sweep / BPP)
//   G_W  = W^T W                      (Gram, Alg. 1 line 4)
//   HALS: W(:,i) /= s_i, Ht(:,i) *= s_i, G_W <- D^-1 G_W D^-1, s_i = sqrt(G_W,ii)
//   P_Ht = A^T W                      (product, Alg. 1 line 4)
//   Ht   = LUC(Ht, P_Ht, G_W)
//   G_H  = Ht^T Ht                    (Gram for the next iteration)
//   relres[t] = sqrt(||A||^2 - 2 <P_Ht, Ht> + <G_W, G_H>) / ||A||   (Sec. 6.2)
// Every step is a kernel of this library; the host only enqueues them.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "batched.cuh"
#include "internal.cuh"
#include "tc.cuh"

using namespace aunmf;

thread_local long long aunmf::g_launches = 0;

namespace {
std::atomic<int> g_inject_site{AUNMF_INJECT_NONE};
std::atomic<long long> g_inject_cycles{aunmf::fault::kDefaultWaitCycles};
}  // namespace

int aunmf::fault::site() { return g_inject_site.load(std::memory_order_relaxed); }

// Readers of the checked build's per-unit site words (registered while the
// library loads; none in the normal build).
static std::vector<int (*)()> &check_readers() {
  static std::vector<int (*)()> readers;
  return readers;
}
void aunmf::register_check_reader(int (*reader)()) { check_readers().push_back(reader); }
long long aunmf::fault::wait_cycles() { return g_inject_cycles.load(std::memory_order_relaxed); }

struct Buf {
  void *p = nullptr;
  size_t cap = 0;
};

struct aunmf_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
  std::string cuda_err;
  // workspace
  Buf Ht, PW, PHt, GH, GW, G64, gpart, dpart, n2a, ctr, relres, last;
  Buf Ax, At, Hk, Wt, parts, err;  // tensor-core path: layout copies, split partials, error flag
  Buf tcacc;                       // tensor-core path, k > 64: partial sums of wide products
  Buf colptr, rowidx, cval, cscratch;  // sparse path: CSC copy of A
  Buf bppq;                            // BPP: G^{-1} in FP64
  Buf dHt;                             // loss backward: (dL/dH)^T
  Buf batch, batch_meta;               // batched runs: arena, descriptors
  // autotuned BPP work tile per batch signature: (warps per block, rows per warp)
  std::map<std::tuple<int, int64_t, int64_t, int, int>, std::pair<int, int>> bpp_tuned;
  // autotuned pipeline stages of the grouped products per batch signature:
  // (A H^T, W^T A)
  std::map<std::tuple<int, int64_t, int64_t, int, int>, std::pair<int, int>> gemm_tuned;
  Buf hA, hW, hH;  // device copies for aunmf_run_host
  Buf aux;         // printed HALS sweep / projected gradient: partials, barrier, values
  Buf spl, splpart;  // sparse: long-row lists of the CSR and the CSC; their chunk partials
  int max_gram_blocks = 2 * 152;
  int n_dparts = 2 * 152;
};

namespace {

int fail_cuda(aunmf_handle *h, cudaError_t e, const char *what) {
  if (h) {
    h->cuda_err = std::string(what) + ": " + cudaGetErrorString(e);
  }
  return AUNMF_E_CUDA;
}

#define CK(h, call)                                      \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return fail_cuda(h, e_, #call); \
  } while (0)

// FP64 partial sums: residual partials, and the layout pass's per-block partials
size_t dpart_bytes(const aunmf_handle *h) {
  const size_t a = (size_t)h->n_dparts + 8, b = 2 * (size_t)tc::prepare_blocks();
  return sizeof(double) * (a > b ? a : b);
}

int ensure(aunmf_handle *h, Buf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return AUNMF_OK;
  if (fault::site() == AUNMF_INJECT_NOMEM) {
    h->cuda_err = "cudaMalloc: not called (allocation failure injected)";
    return AUNMF_E_NOMEM;
  }
  if (b.p) {
    cudaStreamSynchronize(h->stream);
    cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->cuda_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return AUNMF_E_NOMEM;
  }
  b.cap = bytes;
  return AUNMF_OK;
}

#define ENS(h, buf, bytes)                 \
  do {                                     \
    int rc_ = ensure(h, buf, (bytes));     \
    if (rc_ != AUNMF_OK) return rc_;       \
  } while (0)

template <class T>
T *P(Buf &b) {
  return reinterpret_cast<T *>(b.p);
}

bool valid_matrix(const aunmf_matrix *A) {
  if (!A || A->m < 1 || A->n < 1) return false;
  if (A->dense) return A->lda >= A->n;
  return A->rowptr && (A->nnz == 0 || (A->colidx && A->val));
}

struct RunCtx {
  const aunmf_matrix *A;
  int k, algo, prec;
  float mu_eps;
  int max_piv;
  int warm;        // BPP starts from the previous iterate's support
  void *bppq;      // BPP scratch (G^{-1})
  float *W, *Ht, *PW, *PHt, *GH, *GW, *gpart;
  double *GH64, *GW64;  // ABPP: the Grams in FP64 (GH / GW hold them rounded)
  double *dpart, *n2a, *relres_dev, *last;
  DevCounters *ctr;
  // tensor-core path (prec != FP32): X operands of the two products (A or its
  // BF16 copy, m x n; A^T copy, n x m), K-major factor copies (H as k x n,
  // W^T as k x m), split-K partials and the device error flag
  const void *Ax, *At;
  int64_t ldx, ldat;
  void *Hk, *Wt;
  int64_t ldh, ldw;
  float *parts;
  float *tcacc;  // k > 64: the products' per-CTA partial sums (null: added into parts)
  int *err;
  // sparse path: CSC form of A; the long rows of the CSR and the CSC
  const int64_t *colptr;
  const int32_t *rowidx;
  const float *cval;
  SpLongRows csr_long, csc_long;
  bool profile;
  int hals_variant;     // 1: Eq. halsupdate as printed
  bool track_pg;        // form the projected gradient each iteration
  double *sweep_part;   // printed W sweep: 2 x printed_sweep_blocks() partials
  unsigned *bar;        // its grid-barrier counter
  double *pg_part;      // projected gradient: 2 x pgrad_blocks() partials
  double *pg_dev;       // projected-gradient norm per iteration (slot ctr->iter)
  std::vector<cudaEvent_t> *ev;          // profile events (pairs)
  std::vector<int> *ev_phase;            // phase index per pair
};

// Events and the graph of one call, released on every return path (a
// failed call must not leak them).  Destroying an event or an executable
// graph whose work is still in flight is allowed: the driver frees it once
// that work completes.
struct CallResources {
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<cudaEvent_t> ev;  // profile events (pairs)
  CallResources() = default;
  CallResources(const CallResources &) = delete;
  CallResources &operator=(const CallResources &) = delete;
  ~CallResources() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
  }
};

enum Phase { kPhAht = 0, kPhWta = 1, kPhUpdate = 2, kPhGram = 3, kPhOther = 4 };

struct PhaseTimer {
  RunCtx &c;
  cudaStream_t s;
  int phase;
  cudaEvent_t b = nullptr;
  PhaseTimer(RunCtx &c_, cudaStream_t s_, int ph) : c(c_), s(s_), phase(ph) {
    if (!c.profile) return;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    c.ev->push_back(e0);
    c.ev->push_back(e1);
    c.ev_phase->push_back(ph);
    cudaEventRecord(e0, s);
    b = e1;
  }
  ~PhaseTimer() {
    if (b) cudaEventRecord(b, s);
  }
};

// The tensor-core products stream the fixed factor as a two-term split (hi +
// lo rows, MMA N = 2k) for k <= 64.  Beyond that the doubled N brings the
// tensor pipe near saturation at HBM speed (k = 100 at 172,800 x 115,200 ran
// the BF16 product at 91% of HBM with N = 208), and the factor's rounding
// averages out over more terms in the residual's cross term anyway.
bool use_split(int k) { return 2 * k <= 128; }

cudaError_t product_aht(aunmf_handle *h, RunCtx &c, cudaStream_t s) {
  const aunmf_matrix *A = c.A;
  (void)h;
  if (!A->dense) {
    PhaseTimer t(c, s, kPhAht);
    return launch_aht_csr(A->rowptr, A->colidx, A->val, A->m, A->n, A->nnz, c.Ht, c.k, c.PW,
                          &c.csr_long, s);
  }
  if (c.prec == AUNMF_FP32) {
    PhaseTimer t(c, s, kPhAht);
    return launch_aht_simt(A->dense, A->m, A->n, A->lda, c.Ht, c.k, c.PW, c.parts, c.err, s);
  }
  const bool bf = c.prec == AUNMF_BF16;
  const bool split = use_split(c.k);
  const int S = tc::splits_for(A->m, A->n, bf);
  cudaError_t e;
  {
    PhaseTimer t(c, s, kPhOther);
    e = split ? tc::launch_split_transpose(c.Ht, A->n, c.k, c.k, c.Hk, c.ldh, bf, s)
              : tc::launch_transpose_to(c.Ht, A->n, c.k, c.k, c.Hk, c.ldh, bf, s);
    if (e != cudaSuccess) return e;
  }
  {
    PhaseTimer t(c, s, kPhAht);
    e = tc::launch_gemm(c.Ax, A->m, A->n, c.ldx, c.Hk, c.k, c.ldh, split, bf,
                        S == 1 ? c.PW : c.parts, S, c.tcacc, c.err, s);
    if (e != cudaSuccess) return e;
  }
  if (S > 1) {
    PhaseTimer t(c, s, kPhOther);
    return tc::launch_sum_splits(c.parts, S, A->m * (int64_t)c.k, c.PW, s);
  }
  return cudaSuccess;
}

cudaError_t product_wta(aunmf_handle *h, RunCtx &c, cudaStream_t s) {
  const aunmf_matrix *A = c.A;
  (void)h;
  if (!A->dense) {
    PhaseTimer t(c, s, kPhWta);
    return launch_wta_csc(c.colptr, c.rowidx, c.cval, A->n, A->m, A->nnz, c.W, c.k, c.PHt,
                          &c.csc_long, s);
  }
  if (c.prec == AUNMF_FP32) {
    PhaseTimer t(c, s, kPhWta);
    return launch_wta_simt(A->dense, A->m, A->n, A->lda, c.W, c.k, c.PHt, c.parts, c.err, s);
  }
  const bool bf = c.prec == AUNMF_BF16;
  const bool split = use_split(c.k);
  const int S = tc::splits_for(A->n, A->m, bf);
  cudaError_t e;
  {
    PhaseTimer t(c, s, kPhOther);
    e = split ? tc::launch_split_transpose(c.W, A->m, c.k, c.k, c.Wt, c.ldw, bf, s)
              : tc::launch_transpose_to(c.W, A->m, c.k, c.k, c.Wt, c.ldw, bf, s);
    if (e != cudaSuccess) return e;
  }
  {
    PhaseTimer t(c, s, kPhWta);
    e = tc::launch_gemm(c.At, A->n, A->m, c.ldat, c.Wt, c.k, c.ldw, split, bf,
                        S == 1 ? c.PHt : c.parts, S, c.tcacc, c.err, s);
    if (e != cudaSuccess) return e;
  }
  if (S > 1) {
    PhaseTimer t(c, s, kPhOther);
    return tc::launch_sum_splits(c.parts, S, A->n * (int64_t)c.k, c.PHt, s);
  }
  return cudaSuccess;
}

// Workspace and one-off layout copies of A for the tensor-core products:
// X of A H^T is A and X of W^T A is A^T, both rounded to nearest TF32 (kept
// in FP32 containers) or BF16, with 16-byte aligned rows.
int prepare_tc(aunmf_handle *h, RunCtx &c, cudaStream_t s);
// CSC copy of a sparse A (setup of the W^T A product).
int prepare_sparse(aunmf_handle *h, RunCtx &c, cudaStream_t s);

cudaError_t update(RunCtx &c, float *X, const float *Pm, const float *G, const double *G64,
                   int64_t rows, cudaStream_t s) {
  switch (c.algo) {
    case AUNMF_MU: return launch_mu(X, Pm, G, rows, c.k, c.mu_eps, s);
    case AUNMF_HALS: return launch_hals(X, Pm, G, rows, c.k, s);
    default: return launch_bpp(G64, Pm, rows, c.k, X, c.max_piv, c.warm, c.ctr, c.bppq, s);
  }
}

// G = X^T X: FP32 for MU and HALS; for ABPP in FP64 (its solves need the
// small eigenvalues that an FP32 sum loses) with the FP32 rounding beside it.
cudaError_t gram(aunmf_handle *h, RunCtx &c, const float *X, int64_t rows, float *G32,
                 double *G64, cudaStream_t s) {
  if (c.algo == AUNMF_ABPP)
    return launch_gram_d(X, rows, c.k, c.k, G64, G32, reinterpret_cast<double *>(c.gpart),
                         h->max_gram_blocks, s);
  return launch_gram(X, rows, c.k, c.k, G32, c.gpart, h->max_gram_blocks, s, c.err);
}

// Projected-gradient norm of the current (W, H) into pg_dev[ctr->iter], from
// G_H, A H^T of H and G_W, W^T A of W (the last two held from the update of
// H that produced it).
cudaError_t projected_gradient(RunCtx &c, cudaStream_t s) {
  const int nb = pgrad_blocks();
  cudaError_t e = launch_pgrad_partial(c.W, c.PW, c.GH, c.A->m, c.k, c.pg_part, s);
  if (e == cudaSuccess) e = launch_pgrad_partial(c.Ht, c.PHt, c.GW, c.A->n, c.k, c.pg_part + nb, s);
  if (e == cudaSuccess) e = launch_pgrad_final(c.pg_part, 2 * nb, c.ctr, c.pg_dev, s);
  return e;
}

// One AU-NMF iteration (see the file header).
cudaError_t iterate(aunmf_handle *h, RunCtx &c, cudaStream_t s) {
  const int64_t m = c.A->m, n = c.A->n;
  const int k = c.k;
  const bool printed = c.algo == AUNMF_HALS && c.hals_variant == 1;
  cudaError_t e;
  if ((e = product_aht(h, c, s)) != cudaSuccess) return e;
  if (c.track_pg) {
    PhaseTimer t(c, s, kPhOther);
    if ((e = projected_gradient(c, s)) != cudaSuccess) return e;
  }
  {
    PhaseTimer t(c, s, kPhUpdate);
    e = printed ? launch_hals_w_printed(c.W, c.PW, c.GH, m, k, c.sweep_part, c.bar, c.err, s)
                : update(c, c.W, c.PW, c.GH, c.GH64, m, s);
    if (e != cudaSuccess) return e;
  }
  {
    PhaseTimer t(c, s, kPhGram);
    if ((e = gram(h, c, c.W, m, c.GW, c.GW64, s)) != cudaSuccess) return e;
  }
  if (c.algo == AUNMF_HALS && !printed) {
    PhaseTimer t(c, s, kPhUpdate);
    if ((e = launch_hals_normalise(c.W, m, c.Ht, n, c.GW, k, s)) != cudaSuccess) return e;
  }
  if ((e = product_wta(h, c, s)) != cudaSuccess) return e;
  {
    PhaseTimer t(c, s, kPhUpdate);
    e = printed ? launch_hals(c.Ht, c.PHt, c.GW, n, k, s, true)
                : update(c, c.Ht, c.PHt, c.GW, c.GW64, n, s);
    if (e != cudaSuccess) return e;
  }
  {
    PhaseTimer t(c, s, kPhGram);
    if ((e = gram(h, c, c.Ht, n, c.GH, c.GH64, s)) != cudaSuccess) return e;
  }
  {
    PhaseTimer t(c, s, kPhOther);
    e = launch_relres(c.PHt, c.Ht, n * (int64_t)k, c.GW, c.GH, k, c.n2a, c.dpart, h->n_dparts,
                      c.relres_dev, c.ctr, c.last, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int check_run_args(const aunmf_matrix *A, int k, int algo, int iters, const float *W0,
                   const float *H0, const float *W, const float *H, const aunmf_options *o) {
  if (!valid_matrix(A)) return AUNMF_E_INVAL;
  if (k < 1 || k > AUNMF_K_MAX || iters < 0) return AUNMF_E_INVAL;
  if (algo < AUNMF_MU || algo > AUNMF_ABPP) return AUNMF_E_INVAL;
  if (algo == AUNMF_ABPP && k > AUNMF_BPP_K_MAX) return AUNMF_E_INVAL;
  if (!H0 || !W || !H || (algo != AUNMF_ABPP && !W0)) return AUNMF_E_INVAL;
  const int prec = o ? o->prec : AUNMF_FP32;
  if (prec < AUNMF_FP32 || prec > AUNMF_BF16) return AUNMF_E_INVAL;
  if (o && (o->hals_variant < 0 || o->hals_variant > 1)) return AUNMF_E_INVAL;
  if (o && !(o->stop_tol >= 0.0 && o->stop_tol < 1e300)) return AUNMF_E_INVAL;
  if (prec != AUNMF_FP32) {
    if (!A->dense) return AUNMF_E_UNSUPPORTED;
    int rc = tc::check(A->m, A->n, A->lda, k, prec, A->dense);
    if (rc != AUNMF_OK) return rc;
  }
  return AUNMF_OK;
}

#define ENS_TC(h, buf, bytes)              \
  do {                                     \
    int rc_ = ensure(h, buf, (bytes));     \
    if (rc_ != AUNMF_OK) return rc_;       \
  } while (0)

int prepare_tc(aunmf_handle *h, RunCtx &c, cudaStream_t s) {
  const aunmf_matrix *A = c.A;
  const int64_t m = A->m, n = A->n;
  const int k = c.k;
  const bool bf = c.prec == AUNMF_BF16;
  const size_t esz = bf ? 2 : 4;
  c.ldh = tc::copy_ld(n);
  c.ldw = tc::copy_ld(m);
  c.ldat = tc::copy_ld(m);
  ENS_TC(h, h->Hk, esz * tc::factor_elems(n, k));
  ENS_TC(h, h->Wt, esz * tc::factor_elems(m, k));
  ENS_TC(h, h->At, esz * (size_t)n * c.ldat);
  const size_t parts = tc::parts_elems(m > n ? m : n, k);
  ENS_TC(h, h->parts, sizeof(float) * parts);
  ENS_TC(h, h->err, sizeof(int));
  if (!use_split(k)) {
    ENS_TC(h, h->tcacc, sizeof(float) * tc::scratch_elems());
    c.tcacc = P<float>(h->tcacc);
  }
  c.Hk = h->Hk.p;
  c.Wt = h->Wt.p;
  c.At = h->At.p;
  c.parts = P<float>(h->parts);
  c.err = P<int>(h->err);
  cudaError_t e = cudaMemsetAsync(c.err, 0, sizeof(int), s);
  if (e != cudaSuccess) return fail_cuda(h, e, "cudaMemsetAsync(err)");
  // X of A H^T: A rounded to nearest TF32 / BF16 with 16-byte aligned rows;
  // X of W^T A: the same, transposed; and ||A||^2, all in one pass over A
  c.ldx = tc::copy_ld(n);
  ENS_TC(h, h->Ax, esz * (size_t)m * c.ldx);
  ENS_TC(h, h->dpart, dpart_bytes(h));
  ENS_TC(h, h->n2a, 2 * sizeof(double));
  c.Ax = h->Ax.p;
  c.dpart = P<double>(h->dpart);
  if (!c.n2a) c.n2a = P<double>(h->n2a);
  e = tc::launch_prepare(A->dense, m, n, A->lda, h->Ax.p, c.ldx, h->At.p, c.ldat, bf, c.dpart,
                         c.n2a, s);
  if (e != cudaSuccess) return fail_cuda(h, e, "layout copies of A");
  return AUNMF_OK;
}

int prepare_sparse(aunmf_handle *h, RunCtx &c, cudaStream_t s) {
  const aunmf_matrix *A = c.A;
  ENS_TC(h, h->colptr, sizeof(int64_t) * (size_t)(A->n + 1));
  ENS_TC(h, h->rowidx, sizeof(int32_t) * (size_t)(A->nnz > 0 ? A->nnz : 1));
  ENS_TC(h, h->cval, sizeof(float) * (size_t)(A->nnz > 0 ? A->nnz : 1));
  ENS_TC(h, h->cscratch, csc_scratch_bytes(A->n, A->nnz));
  cudaError_t e = launch_csr_to_csc(A->rowptr, A->colidx, A->val, A->m, A->n, A->nnz,
                                    P<int64_t>(h->colptr), P<int32_t>(h->rowidx), P<float>(h->cval),
                                    h->cscratch.p, s);
  if (e != cudaSuccess) return fail_cuda(h, e, "csr_to_csc");
  c.colptr = P<int64_t>(h->colptr);
  c.rowidx = P<int32_t>(h->rowidx);
  c.cval = P<float>(h->cval);
  // rows of either form long enough to be split over several warps
  const int64_t cap = long_rows_capacity(A->nnz);
  ENS_TC(h, h->spl, sizeof(int64_t) * (size_t)(4 * cap + 2) + 2 * sizeof(unsigned long long));
  int64_t *L = P<int64_t>(h->spl);
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(L + 4 * cap + 2);
  e = find_long_rows(A->rowptr, A->m, A->nnz, L, L + cap, cnt, &c.csr_long, s);
  if (e == cudaSuccess)
    e = find_long_rows(c.colptr, A->n, A->nnz, L + 2 * cap + 1, L + 3 * cap + 1, cnt + 1,
                       &c.csc_long, s);
  if (e != cudaSuccess) return fail_cuda(h, e, "find_long_rows");
  const int64_t parts = c.csr_long.nchunks + c.csc_long.nchunks;
  if (parts > 0) {
    ENS_TC(h, h->splpart, sizeof(float) * (size_t)parts * c.k);
    c.csr_long.part = P<float>(h->splpart);
    c.csc_long.part = c.csr_long.part + (size_t)c.csr_long.nchunks * c.k;
  }
  return AUNMF_OK;
}

}  // namespace

// ============================================================ C ABI
extern "C" {

const char *aunmf_strerror(int code) {
  switch (code) {
    case AUNMF_OK: return "ok";
    case AUNMF_E_INVAL: return "invalid argument";
    case AUNMF_E_NOMEM: return "out of device memory";
    case AUNMF_E_CUDA: return "CUDA error";
    case AUNMF_E_NUMERIC: return "numerical failure (non-finite value or non-positive pivot)";
    case AUNMF_E_NOCONVERGE: return "BPP reached its pivot cap";
    case AUNMF_E_TIMEOUT: return "device wait timed out";
    case AUNMF_E_UNSUPPORTED: return "unsupported by the library";
    default: return "unknown status";
  }
}

int aunmf_create(aunmf_handle **out, void *stream) {
  if (!out) return AUNMF_E_INVAL;
  *out = nullptr;
  aunmf_handle *h = new (std::nothrow) aunmf_handle();
  if (!h) return AUNMF_E_NOMEM;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) { int rc = fail_cuda(h, e, "cudaGetDevice"); delete h; return rc; }
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { int rc = fail_cuda(h, e, "cudaStreamCreate"); delete h; return rc; }
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  // Gram partials: one per block of a single resident wave (two 256-thread
  // blocks per SM); fewer partials also shorten the FP64 reduction
  h->max_gram_blocks = 2 * sms;
  h->n_dparts = 2 * sms;
  *out = h;
  return AUNMF_OK;
}

int aunmf_set_stream(aunmf_handle *h, void *stream) {
  if (!h) return AUNMF_E_INVAL;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  return AUNMF_OK;
}

int aunmf_destroy(aunmf_handle *h) {
  if (!h) return AUNMF_E_INVAL;
  cudaStreamSynchronize(h->stream);
  Buf *bufs[] = {&h->Ht, &h->PW, &h->PHt, &h->GH, &h->GW, &h->G64, &h->gpart, &h->dpart, &h->n2a,
                 &h->ctr, &h->relres, &h->last, &h->Ax, &h->At, &h->Hk, &h->Wt, &h->parts,
                 &h->err, &h->tcacc, &h->aux, &h->spl, &h->splpart, &h->colptr, &h->rowidx, &h->cval, &h->cscratch, &h->bppq, &h->dHt,
                 &h->batch, &h->batch_meta, &h->hA, &h->hW, &h->hH};
  for (Buf *b : bufs)
    if (b->p) cudaFree(b->p);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
  return AUNMF_OK;
}

const char *aunmf_last_cuda_error(aunmf_handle *h) { return h ? h->cuda_err.c_str() : ""; }

int aunmf_test_inject(int site, double wait_ms) {
  if (site < AUNMF_INJECT_NONE || site > AUNMF_INJECT_SIMT_WAIT) return AUNMF_E_INVAL;
  if (!(wait_ms <= 60000.0)) return AUNMF_E_INVAL;  // also rejects NaN
  long long cycles = fault::kDefaultWaitCycles;
  if (site != AUNMF_INJECT_NONE && wait_ms > 0.0) {
    // the SM clock counted by clock64(); at most the device's maximum clock
    int dev = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) {
      cudaGetLastError();
      khz = 2100000;
    }
    cycles = (long long)(wait_ms * (double)khz);
    if (cycles < 1000) cycles = 1000;
  }
  g_inject_cycles.store(cycles, std::memory_order_relaxed);
  g_inject_site.store(site, std::memory_order_relaxed);
  return AUNMF_OK;
}

// aunmf_options.validate: A >= 0 and finite (and, for a CSR, a well-formed
// structure), W0 and H0 >= 0 and finite, checked before any other kernel
// reads them (Sec. 2 poses NMF for A >= 0; the updates of Sec. 4 keep the
// factors nonnegative only from a nonnegative start).  W0 may be null.
static int validate_inputs(aunmf_handle *h, const aunmf_matrix *A, int k, const float *W0,
                           const float *H0, cudaStream_t s) {
  ENS(h, h->err, sizeof(int));
  int *flag = P<int>(h->err);
  CK(h, cudaMemsetAsync(flag, 0, sizeof(int), s));
  if (A->dense)
    CK(h, launch_validate_dense(A->dense, A->m, A->n, A->lda, flag, s));
  else
    CK(h, launch_validate_csr(A->rowptr, A->colidx, A->val, A->m, A->n, A->nnz, flag, s));
  if (W0) CK(h, launch_validate_vec(W0, A->m * (int64_t)k, kValidateFactors, flag, s));
  if (H0) CK(h, launch_validate_vec(H0, (int64_t)k * A->n, kValidateFactors, flag, s));
  int hf = 0;
  CK(h, cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  return hf ? AUNMF_E_INVAL : AUNMF_OK;
}

int aunmf_check_status(int *site) {
  if (!site) return AUNMF_E_INVAL;
  if (check_readers().empty()) {
    *site = -1;
    return AUNMF_OK;
  }
  cudaDeviceSynchronize();
  int first = 0;
  for (int (*r)() : check_readers()) {
    const int v = r();
    if (!first) first = v;
  }
  *site = first;
  return AUNMF_OK;
}

int aunmf_run(aunmf_handle *h, const aunmf_matrix *A, int k, int algo, int iters,
              const float *W0, const float *H0, float *W, float *H, double *relres,
              const aunmf_options *opt, aunmf_info *info) {
  if (!h) return AUNMF_E_INVAL;
  int rc = check_run_args(A, k, algo, iters, W0, H0, W, H, opt);
  if (rc != AUNMF_OK) return rc;
  aunmf_options o{};
  if (opt) o = *opt;
  const int64_t m = A->m, n = A->n;
  cudaStream_t s = h->stream;
  if (o.validate) {
    rc = validate_inputs(h, A, k, algo == AUNMF_ABPP ? nullptr : W0, H0, s);
    if (rc != AUNMF_OK) return rc;
  }

  ENS(h, h->Ht, sizeof(float) * n * k);
  ENS(h, h->PW, sizeof(float) * m * k);
  ENS(h, h->PHt, sizeof(float) * n * k);
  ENS(h, h->GH, sizeof(float) * k * k);
  ENS(h, h->GW, sizeof(float) * k * k);
  ENS(h, h->G64, 2 * sizeof(double) * k * k);
  ENS(h, h->gpart, sizeof(double) * (size_t)h->max_gram_blocks * k * k);
  ENS(h, h->dpart, dpart_bytes(h));
  ENS(h, h->n2a, 2 * sizeof(double));
  ENS(h, h->ctr, sizeof(DevCounters));
  ENS(h, h->relres, sizeof(double) * (iters > 0 ? iters : 1));
  ENS(h, h->last, sizeof(double));
  ENS(h, h->bppq, bpp_scratch_bytes(k, m > n ? m : n));

  RunCtx c{};
  c.A = A;
  c.warm = o.bpp_cold_start ? 0 : 1;
  c.bppq = h->bppq.p;
  c.k = k;
  c.algo = algo;
  c.prec = o.prec;
  c.mu_eps = (float)(o.mu_eps > 0 ? o.mu_eps : 1e-16);
  c.max_piv = o.bpp_max_pivots > 0 ? o.bpp_max_pivots : 10 * k;
  c.W = W;
  c.Ht = P<float>(h->Ht);
  c.PW = P<float>(h->PW);
  c.PHt = P<float>(h->PHt);
  c.GH = P<float>(h->GH);
  c.GW = P<float>(h->GW);
  c.GH64 = P<double>(h->G64);
  c.GW64 = c.GH64 + (size_t)k * k;
  c.gpart = P<float>(h->gpart);
  c.dpart = P<double>(h->dpart);
  c.n2a = P<double>(h->n2a);
  c.relres_dev = P<double>(h->relres);
  c.last = P<double>(h->last);
  c.ctr = P<DevCounters>(h->ctr);
  CallResources R;
  std::vector<int> ev_phase;
  c.ev = &R.ev;
  c.ev_phase = &ev_phase;
  c.profile = o.profile != 0;
  c.hals_variant = algo == AUNMF_HALS ? o.hals_variant : 0;
  c.track_pg = o.stop_tol > 0.0;
  if (c.hals_variant == 1 || c.track_pg) {
    const size_t dbl = 2 * (size_t)printed_sweep_blocks() + 2 * (size_t)pgrad_blocks() +
                       (size_t)(iters > 0 ? iters : 1);
    ENS(h, h->aux, sizeof(double) * dbl + 256);
    c.sweep_part = P<double>(h->aux);
    c.pg_part = c.sweep_part + 2 * (size_t)printed_sweep_blocks();
    c.pg_dev = c.pg_part + 2 * (size_t)pgrad_blocks();
    c.bar = reinterpret_cast<unsigned *>(c.pg_dev + (iters > 0 ? iters : 1));
    ENS(h, h->err, sizeof(int));
    c.err = P<int>(h->err);
    CK(h, cudaMemsetAsync(c.err, 0, sizeof(int), s));
  }
  const long long launches0 = g_launches;
  long long graph_launches = 0;
  CK(h, cudaEventCreate(&R.t0));
  CK(h, cudaEventCreate(&R.t1));
  CK(h, cudaEventRecord(R.t0, s));
  CK(h, cudaMemsetAsync(c.ctr, 0, sizeof(DevCounters), s));
  // setup (a0): W0 -> W, H0 -> Ht, ||A||^2, BF16 copy of A, initial G_H
  if (algo != AUNMF_ABPP) {
    if (W != W0) CK(h, cudaMemcpyAsync(W, W0, sizeof(float) * m * k, cudaMemcpyDeviceToDevice, s));
  } else {
    CK(h, cudaMemsetAsync(W, 0, sizeof(float) * m * k, s));
  }
  CK(h, launch_transpose(H0, k, n, c.Ht, s));
  if (A->dense && o.prec != AUNMF_FP32) {
    // ||A||^2 comes out of the layout pass (prepare_tc below)
  } else if (A->dense) {
    CK(h, launch_norm2(A->dense, m, n, A->lda, c.dpart, h->n_dparts, c.n2a, s));
  } else {
    CK(h, launch_norm2_vec(A->val, A->nnz, c.dpart, h->n_dparts, c.n2a, s));
  }
  if (o.prec != AUNMF_FP32) {
    int prc = prepare_tc(h, c, s);
    if (prc != AUNMF_OK) return prc;
  } else if (A->dense) {
    ENS(h, h->parts, simt_parts_bytes(m > n ? m : n, k));
    c.parts = P<float>(h->parts);
    ENS(h, h->err, sizeof(int));
    c.err = P<int>(h->err);
    CK(h, cudaMemsetAsync(c.err, 0, sizeof(int), s));
  }
  if (!A->dense) {
    int prc = prepare_sparse(h, c, s);
    if (prc != AUNMF_OK) return prc;
  }
  if (!c.err) {  // the bounded waits of the wide-rank Gram report here too
    ENS(h, h->err, sizeof(int));
    c.err = P<int>(h->err);
    CK(h, cudaMemsetAsync(c.err, 0, sizeof(int), s));
  }
  CK(h, gram(h, c, c.Ht, n, c.GH, c.GH64, s));
  if (c.track_pg) {
    // W^T W and W^T A of the starting W, for the first iteration's measure
    CK(h, gram(h, c, c.W, m, c.GW, c.GW64, s));
    CK(h, product_wta(h, c, s));
  }

  // the printed HALS sweep is a cooperative launch: not captured
  const bool use_graph = o.use_graph && !o.profile && iters > 1 && c.hals_variant == 0;
  if (use_graph) {
    // capture one iteration on the private stream, replay on the caller's
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const long long lc0 = g_launches;
    cudaError_t ce = iterate(h, c, h->cap_stream);
    const long long per_iter = g_launches - lc0;
    g_launches = lc0;  // captured, not launched: counted per replay below
    graph_launches = per_iter;
    cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &R.graph);
    if (ce != cudaSuccess) return fail_cuda(h, ce, "iterate (capture)");
    if (ee != cudaSuccess) return fail_cuda(h, ee, "cudaStreamEndCapture");
    CK(h, cudaGraphInstantiate(&R.gexec, R.graph, 0));
  }
  // with a stop rule the host reads each iteration's measure before the next
  int done = 0;
  double pg0 = 0.0, pg_last = 0.0;
  for (int t = 0; t < iters; ++t) {
    if (R.gexec) {
      CK(h, cudaGraphLaunch(R.gexec, s));
    } else {
      cudaError_t e = iterate(h, c, s);
      if (e != cudaSuccess) return fail_cuda(h, e, "iterate");
    }
    done = t + 1;
    if (c.track_pg) {
      CK(h, cudaMemcpyAsync(&pg_last, c.pg_dev + t, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(h, cudaStreamSynchronize(s));
      if (t == 0) pg0 = pg_last;
      if (!(pg_last > o.stop_tol * pg0)) break;
    }
  }
  graph_launches *= done;
  CK(h, launch_transpose(c.Ht, n, k, H, s));
  CK(h, cudaEventRecord(R.t1, s));
  DevCounters hc{};
  int herr = 0;
  CK(h, cudaMemcpyAsync(&hc, c.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
  if (c.err) CK(h, cudaMemcpyAsync(&herr, c.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (relres && done > 0)
    CK(h, cudaMemcpyAsync(relres, c.relres_dev, sizeof(double) * done, cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  if (info) {
    memset(info, 0, sizeof(*info));
    info->bpp_pivots = hc.bpp_pivots;
    info->bpp_nonconverged = hc.bpp_nonconv;
    info->bpp_numeric = hc.bpp_numeric;
    info->bpp_redone = hc.bpp_redo;
    info->iters_done = done;
    info->pgrad_first = pg0;
    info->pgrad_last = pg_last;
    info->launches = g_launches - launches0 + graph_launches;
    cudaEventElapsedTime(&info->ms_total, R.t0, R.t1);
    for (size_t p = 0; p < ev_phase.size(); ++p) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, R.ev[2 * p], R.ev[2 * p + 1]);
      switch (ev_phase[p]) {
        case kPhAht: info->ms_aht += ms; info->n_aht += 1; break;
        case kPhWta: info->ms_wta += ms; info->n_wta += 1; break;
        case kPhUpdate: info->ms_update += ms; break;
        case kPhGram: info->ms_gram += ms; break;
        default: info->ms_other += ms; break;
      }
    }
  }
  if (herr) return AUNMF_E_TIMEOUT;
  if (hc.nonfinite) return AUNMF_E_NUMERIC;
  if (hc.bpp_numeric) return AUNMF_E_NUMERIC;
  if (hc.bpp_nonconv) return AUNMF_E_NOCONVERGE;
  return AUNMF_OK;
}

int aunmf_run_host(aunmf_handle *h, const float *A, int64_t m, int64_t n, int64_t lda, int k,
                   int algo, int iters, const float *W0, const float *H0, float *W, float *H,
                   double *relres, const aunmf_options *opt, aunmf_info *info) {
  if (!h || !A || m < 1 || n < 1 || lda < n || !H0 || !W || !H) return AUNMF_E_INVAL;
  if (algo != AUNMF_ABPP && !W0) return AUNMF_E_INVAL;
  if (k < 1 || k > AUNMF_K_MAX) return AUNMF_E_INVAL;
  cudaStream_t s = h->stream;
  const int prec = opt ? opt->prec : AUNMF_FP32;
  // The tensor-core forms read A only in the one-off layout pass, which
  // writes the rounded device copies the products stream.  When A is in
  // page-locked host memory that pass reads it over the host link directly
  // (no staging copy, no device buffer for A); otherwise, and for the FP32
  // form (whose products read A every iteration), A is copied first.
  const float *Ad = nullptr;
  int64_t ldd = n;
  if (prec == AUNMF_TF32 || prec == AUNMF_BF16) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, A) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer != nullptr) {
      Ad = static_cast<const float *>(at.devicePointer);
      ldd = lda;
    } else {
      cudaGetLastError();
    }
  }
  ENS(h, h->hW, sizeof(float) * m * k);
  ENS(h, h->hH, sizeof(float) * k * n);
  float *dW = P<float>(h->hW), *dH = P<float>(h->hH);
  if (!Ad) {
    ENS(h, h->hA, sizeof(float) * m * n);
    float *dA = P<float>(h->hA);
    if (lda == n)
      CK(h, cudaMemcpyAsync(dA, A, sizeof(float) * m * n, cudaMemcpyHostToDevice, s));
    else
      CK(h, cudaMemcpy2DAsync(dA, sizeof(float) * n, A, sizeof(float) * lda, sizeof(float) * n, m,
                              cudaMemcpyHostToDevice, s));
    Ad = dA;
  }
  if (algo != AUNMF_ABPP) CK(h, cudaMemcpyAsync(dW, W0, sizeof(float) * m * k, cudaMemcpyHostToDevice, s));
  CK(h, cudaMemcpyAsync(dH, H0, sizeof(float) * k * n, cudaMemcpyHostToDevice, s));
  aunmf_matrix M{};
  M.m = m;
  M.n = n;
  M.dense = Ad;
  M.lda = ldd;
  int rc = aunmf_run(h, &M, k, algo, iters, dW, dH, dW, dH, relres, opt, info);
  if (rc != AUNMF_OK && rc != AUNMF_E_NOCONVERGE) return rc;
  CK(h, cudaMemcpyAsync(W, dW, sizeof(float) * m * k, cudaMemcpyDeviceToHost, s));
  CK(h, cudaMemcpyAsync(H, dH, sizeof(float) * k * n, cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  return rc;
}

// ------------------------------------------------------------ single steps
int aunmf_gram_w(aunmf_handle *h, const float *W, int64_t m, int k, float *G) {
  if (!h || !W || !G || m < 1 || k < 1 || k > AUNMF_K_MAX) return AUNMF_E_INVAL;
  ENS(h, h->gpart, sizeof(float) * (size_t)h->max_gram_blocks * k * k);
  ENS(h, h->err, sizeof(int));
  CK(h, cudaMemsetAsync(h->err.p, 0, sizeof(int), h->stream));
  CK(h, launch_gram(W, m, k, k, G, P<float>(h->gpart), h->max_gram_blocks, h->stream,
                    P<int>(h->err)));
  return AUNMF_OK;
}

int aunmf_gram_h(aunmf_handle *h, const float *H, int k, int64_t n, float *G) {
  if (!h || !H || !G || n < 1 || k < 1 || k > AUNMF_K_MAX) return AUNMF_E_INVAL;
  ENS(h, h->Ht, sizeof(float) * n * k);
  ENS(h, h->gpart, sizeof(float) * (size_t)h->max_gram_blocks * k * k);
  ENS(h, h->err, sizeof(int));
  CK(h, cudaMemsetAsync(h->err.p, 0, sizeof(int), h->stream));
  CK(h, launch_transpose(H, k, n, P<float>(h->Ht), h->stream));
  CK(h, launch_gram(P<float>(h->Ht), n, k, k, G, P<float>(h->gpart), h->max_gram_blocks, h->stream,
                    P<int>(h->err)));
  return AUNMF_OK;
}

int aunmf_aht(aunmf_handle *h, const aunmf_matrix *A, const float *H, int k, int prec, float *Pout) {
  if (!h || !valid_matrix(A) || !H || !Pout || k < 1 || k > AUNMF_K_MAX) return AUNMF_E_INVAL;
  if (prec < AUNMF_FP32 || prec > AUNMF_BF16) return AUNMF_E_INVAL;
  if (!A->dense && prec != AUNMF_FP32) return AUNMF_E_UNSUPPORTED;
  if (prec != AUNMF_FP32) {
    int rc = tc::check(A->m, A->n, A->lda, k, prec, A->dense);
    if (rc != AUNMF_OK) return rc;
  }
  const int64_t n = A->n;
  ENS(h, h->Ht, sizeof(float) * n * k);
  RunCtx c{};
  c.A = A;
  c.k = k;
  c.prec = prec;
  c.Ht = P<float>(h->Ht);
  c.PW = Pout;
  CK(h, launch_transpose(H, k, n, c.Ht, h->stream));
  if (prec != AUNMF_FP32) {
    int rc = prepare_tc(h, c, h->stream);
    if (rc != AUNMF_OK) return rc;
  } else if (A->dense) {
    ENS(h, h->parts, simt_parts_bytes(A->m > A->n ? A->m : A->n, k));
    c.parts = P<float>(h->parts);
    ENS(h, h->err, sizeof(int));
    c.err = P<int>(h->err);
    CK(h, cudaMemsetAsync(c.err, 0, sizeof(int), h->stream));
  }
  CK(h, product_aht(h, c, h->stream));
  return AUNMF_OK;
}

int aunmf_wta(aunmf_handle *h, const aunmf_matrix *A, const float *W, int k, int prec, float *Pout) {
  if (!h || !valid_matrix(A) || !W || !Pout || k < 1 || k > AUNMF_K_MAX) return AUNMF_E_INVAL;
  if (prec < AUNMF_FP32 || prec > AUNMF_BF16) return AUNMF_E_INVAL;
  if (!A->dense && prec != AUNMF_FP32) return AUNMF_E_UNSUPPORTED;
  if (prec != AUNMF_FP32) {
    int rc = tc::check(A->m, A->n, A->lda, k, prec, A->dense);
    if (rc != AUNMF_OK) return rc;
  }
  const int64_t n = A->n;
  ENS(h, h->PHt, sizeof(float) * n * k);
  RunCtx c{};
  c.A = A;
  c.k = k;
  c.prec = prec;
  c.W = const_cast<float *>(W);
  c.PHt = P<float>(h->PHt);
  if (prec != AUNMF_FP32) {
    int rc = prepare_tc(h, c, h->stream);
    if (rc != AUNMF_OK) return rc;
  } else if (A->dense) {
    ENS(h, h->parts, simt_parts_bytes(A->m > n ? A->m : n, k));
    c.parts = P<float>(h->parts);
    ENS(h, h->err, sizeof(int));
    c.err = P<int>(h->err);
    CK(h, cudaMemsetAsync(c.err, 0, sizeof(int), h->stream));
  }
  if (!A->dense) {
    int rc = prepare_sparse(h, c, h->stream);
    if (rc != AUNMF_OK) return rc;
  }
  CK(h, product_wta(h, c, h->stream));
  CK(h, launch_transpose(c.PHt, n, k, Pout, h->stream));
  return AUNMF_OK;
}

namespace {
// ABPP step calls: the caller's FP32 Gram widened into the handle's FP64 slot.
int widen_gram(aunmf_handle *h, const float *G, int k, double **G64) {
  ENS(h, h->G64, 2 * sizeof(double) * k * k);
  *G64 = P<double>(h->G64);
  CK(h, launch_widen(G, k, *G64, h->stream));
  return AUNMF_OK;
}
// Status of an ABPP step from the device counters (synchronises).
int bpp_status(aunmf_handle *h, DevCounters *ctr) {
  DevCounters hc{};
  CK(h, cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  if (hc.bpp_numeric) return AUNMF_E_NUMERIC;
  if (hc.bpp_nonconv) return AUNMF_E_NOCONVERGE;
  return AUNMF_OK;
}
}  // namespace

int aunmf_update_w(aunmf_handle *h, int algo, float *W, const float *PW, const float *GH,
                   int64_t m, int k, float *H, int64_t n, double eps) {
  if (!h || !W || !PW || !GH || m < 1 || k < 1 || k > AUNMF_K_MAX) return AUNMF_E_INVAL;
  if (algo < AUNMF_MU || algo > AUNMF_ABPP) return AUNMF_E_INVAL;
  if (algo == AUNMF_ABPP && k > AUNMF_BPP_K_MAX) return AUNMF_E_INVAL;
  cudaStream_t s = h->stream;
  ENS(h, h->ctr, sizeof(DevCounters));
  ENS(h, h->bppq, bpp_scratch_bytes(k, m));
  RunCtx c{};
  c.k = k;
  c.algo = algo;
  c.mu_eps = (float)(eps > 0 ? eps : 1e-16);
  c.max_piv = 10 * k;
  c.ctr = P<DevCounters>(h->ctr);
  c.bppq = h->bppq.p;
  double *G64 = nullptr;
  if (algo == AUNMF_ABPP) {
    int rc = widen_gram(h, GH, k, &G64);
    if (rc != AUNMF_OK) return rc;
  }
  CK(h, cudaMemsetAsync(c.ctr, 0, sizeof(DevCounters), s));
  CK(h, update(c, W, PW, GH, G64, m, s));
  if (algo == AUNMF_ABPP) return bpp_status(h, c.ctr);
  if (algo == AUNMF_HALS) {
    ENS(h, h->GW, sizeof(float) * k * k);
    ENS(h, h->gpart, sizeof(float) * (size_t)h->max_gram_blocks * k * k);
    CK(h, launch_gram(W, m, k, k, P<float>(h->GW), P<float>(h->gpart), h->max_gram_blocks, s));
    if (H && n > 0) {
      ENS(h, h->Ht, sizeof(float) * n * k);
      CK(h, launch_transpose(H, k, n, P<float>(h->Ht), s));
      CK(h, launch_hals_normalise(W, m, P<float>(h->Ht), n, P<float>(h->GW), k, s));
      CK(h, launch_transpose(P<float>(h->Ht), n, k, H, s));
    } else {
      CK(h, launch_hals_normalise(W, m, nullptr, 0, P<float>(h->GW), k, s));
    }
  }
  return AUNMF_OK;
}

int aunmf_update_h(aunmf_handle *h, int algo, float *H, const float *PH, const float *GW, int k,
                   int64_t n, double eps) {
  if (!h || !H || !PH || !GW || n < 1 || k < 1 || k > AUNMF_K_MAX) return AUNMF_E_INVAL;
  if (algo < AUNMF_MU || algo > AUNMF_ABPP) return AUNMF_E_INVAL;
  if (algo == AUNMF_ABPP && k > AUNMF_BPP_K_MAX) return AUNMF_E_INVAL;
  cudaStream_t s = h->stream;
  ENS(h, h->Ht, sizeof(float) * n * k);
  ENS(h, h->PHt, sizeof(float) * n * k);
  ENS(h, h->ctr, sizeof(DevCounters));
  ENS(h, h->bppq, bpp_scratch_bytes(k, n));
  RunCtx c{};
  c.k = k;
  c.algo = algo;
  c.mu_eps = (float)(eps > 0 ? eps : 1e-16);
  c.max_piv = 10 * k;
  c.ctr = P<DevCounters>(h->ctr);
  c.bppq = h->bppq.p;
  double *G64 = nullptr;
  if (algo == AUNMF_ABPP) {
    int rc = widen_gram(h, GW, k, &G64);
    if (rc != AUNMF_OK) return rc;
  }
  CK(h, cudaMemsetAsync(c.ctr, 0, sizeof(DevCounters), s));
  CK(h, launch_transpose(H, k, n, P<float>(h->Ht), s));
  CK(h, launch_transpose(PH, k, n, P<float>(h->PHt), s));
  CK(h, update(c, P<float>(h->Ht), P<float>(h->PHt), GW, G64, n, s));
  CK(h, launch_transpose(P<float>(h->Ht), n, k, H, s));
  if (algo == AUNMF_ABPP) return bpp_status(h, c.ctr);
  return AUNMF_OK;
}

int aunmf_nls_bpp(aunmf_handle *h, const float *G, const float *R, int64_t nrhs, int k, float *X,
                  int max_pivots, int64_t *pivots, int64_t *nonconv) {
  if (!h || !G || !R || !X || nrhs < 0 || k < 1 || k > AUNMF_BPP_K_MAX) return AUNMF_E_INVAL;
  cudaStream_t s = h->stream;
  ENS(h, h->ctr, sizeof(DevCounters));
  ENS(h, h->bppq, bpp_scratch_bytes(k, nrhs));
  DevCounters *ctr = P<DevCounters>(h->ctr);
  double *G64 = nullptr;
  int rc = widen_gram(h, G, k, &G64);
  if (rc != AUNMF_OK) return rc;
  CK(h, cudaMemsetAsync(ctr, 0, sizeof(DevCounters), s));
  CK(h, launch_bpp(G64, R, nrhs, k, X, max_pivots > 0 ? max_pivots : 10 * k, 0, ctr, h->bppq.p, s));
  DevCounters hc{};
  CK(h, cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  if (pivots) *pivots = hc.bpp_pivots;
  if (nonconv) *nonconv = hc.bpp_nonconv;
  if (hc.bpp_numeric) return AUNMF_E_NUMERIC;
  if (hc.bpp_nonconv) return AUNMF_E_NOCONVERGE;
  return AUNMF_OK;
}

int aunmf_relres(aunmf_handle *h, const aunmf_matrix *A, const float *W, const float *H, int k,
                 double *relres) {
  if (!h || !valid_matrix(A) || !W || !H || !relres || k < 1 || k > AUNMF_K_MAX) return AUNMF_E_INVAL;
  const int64_t m = A->m, n = A->n;
  cudaStream_t s = h->stream;
  ENS(h, h->Ht, sizeof(float) * n * k);
  ENS(h, h->PHt, sizeof(float) * n * k);
  ENS(h, h->GH, sizeof(float) * k * k);
  ENS(h, h->GW, sizeof(float) * k * k);
  ENS(h, h->gpart, sizeof(float) * (size_t)h->max_gram_blocks * k * k);
  ENS(h, h->dpart, dpart_bytes(h));
  ENS(h, h->n2a, 2 * sizeof(double));
  ENS(h, h->ctr, sizeof(DevCounters));
  ENS(h, h->last, sizeof(double));
  float *Ht = P<float>(h->Ht), *PHt = P<float>(h->PHt);
  double *dp = P<double>(h->dpart);
  ENS(h, h->err, sizeof(int));
  CK(h, cudaMemsetAsync(h->ctr.p, 0, sizeof(DevCounters), s));
  CK(h, cudaMemsetAsync(h->err.p, 0, sizeof(int), s));
  CK(h, launch_transpose(H, k, n, Ht, s));
  if (A->dense) {
    CK(h, launch_norm2(A->dense, m, n, A->lda, dp, h->n_dparts, P<double>(h->n2a), s));
    ENS(h, h->parts, simt_parts_bytes(A->m > n ? A->m : n, k));
    CK(h, launch_wta_simt(A->dense, m, n, A->lda, W, k, PHt, P<float>(h->parts), P<int>(h->err),
                          s));
  } else {
    CK(h, launch_norm2_vec(A->val, A->nnz, dp, h->n_dparts, P<double>(h->n2a), s));
    RunCtx c{};
    c.A = A;
    int rc = prepare_sparse(h, c, s);
    if (rc != AUNMF_OK) return rc;
    CK(h, launch_wta_csc(c.colptr, c.rowidx, c.cval, n, m, A->nnz, W, k, PHt, &c.csc_long, s));
  }
  CK(h, launch_gram(W, m, k, k, P<float>(h->GW), P<float>(h->gpart), h->max_gram_blocks, s,
                    P<int>(h->err)));
  CK(h, launch_gram(Ht, n, k, k, P<float>(h->GH), P<float>(h->gpart), h->max_gram_blocks, s,
                    P<int>(h->err)));
  CK(h, launch_relres(PHt, Ht, n * (int64_t)k, P<float>(h->GW), P<float>(h->GH), k,
                      P<double>(h->n2a), dp, h->n_dparts, nullptr, P<DevCounters>(h->ctr),
                      P<double>(h->last), s));
  int herr = 0;
  CK(h, cudaMemcpyAsync(&herr, h->err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(h, cudaMemcpyAsync(relres, h->last.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  return herr ? AUNMF_E_TIMEOUT : AUNMF_OK;
}

// ------------------------------------------------------------ loss / gradient
namespace {
int loss_setup(aunmf_handle *h, const aunmf_matrix *A, int k, const float *W, const float *H,
               int prec, RunCtx &c) {
  if (!valid_matrix(A) || !W || !H || k < 1 || k > AUNMF_K_MAX) return AUNMF_E_INVAL;
  if (prec < AUNMF_FP32 || prec > AUNMF_BF16) return AUNMF_E_INVAL;
  if (!A->dense && prec != AUNMF_FP32) return AUNMF_E_UNSUPPORTED;
  if (prec != AUNMF_FP32) {
    int rc = tc::check(A->m, A->n, A->lda, k, prec, A->dense);
    if (rc != AUNMF_OK) return rc;
  }
  const int64_t m = A->m, n = A->n;
  ENS(h, h->Ht, sizeof(float) * n * k);
  ENS(h, h->PW, sizeof(float) * m * k);
  ENS(h, h->PHt, sizeof(float) * n * k);
  ENS(h, h->GH, sizeof(float) * k * k);
  ENS(h, h->GW, sizeof(float) * k * k);
  ENS(h, h->gpart, sizeof(float) * (size_t)h->max_gram_blocks * k * k);
  ENS(h, h->dpart, dpart_bytes(h));
  ENS(h, h->n2a, 2 * sizeof(double));
  c.A = A;
  c.k = k;
  c.prec = prec;
  c.W = const_cast<float *>(W);
  c.Ht = P<float>(h->Ht);
  c.PW = P<float>(h->PW);
  c.PHt = P<float>(h->PHt);
  c.GH = P<float>(h->GH);
  c.GW = P<float>(h->GW);
  c.gpart = P<float>(h->gpart);
  c.dpart = P<double>(h->dpart);
  c.n2a = P<double>(h->n2a);
  cudaStream_t s = h->stream;
  CK(h, launch_transpose(H, k, n, c.Ht, s));
  if (prec != AUNMF_FP32) {
    int rc = prepare_tc(h, c, s);  // also writes ||A||^2
    if (rc != AUNMF_OK) return rc;
  } else if (A->dense) {
    CK(h, launch_norm2(A->dense, m, n, A->lda, c.dpart, h->n_dparts, c.n2a, s));
    ENS(h, h->parts, simt_parts_bytes(m > n ? m : n, k));
    c.parts = P<float>(h->parts);
    ENS(h, h->err, sizeof(int));
    c.err = P<int>(h->err);
    CK(h, cudaMemsetAsync(c.err, 0, sizeof(int), s));
  } else {
    CK(h, launch_norm2_vec(A->val, A->nnz, c.dpart, h->n_dparts, c.n2a, s));
  }
  if (!A->dense) {
    int rc = prepare_sparse(h, c, s);
    if (rc != AUNMF_OK) return rc;
  }
  return AUNMF_OK;
}
}  // namespace

int aunmf_loss_fwd(aunmf_handle *h, const aunmf_matrix *A, int k, const float *W, const float *H,
                   int prec, double *loss, float *WtA) {
  if (!h || !loss) return AUNMF_E_INVAL;
  RunCtx c{};
  int rc = loss_setup(h, A, k, W, H, prec, c);
  if (rc != AUNMF_OK) return rc;
  cudaStream_t s = h->stream;
  const int64_t m = A->m, n = A->n;
  CK(h, product_wta(h, c, s));
  CK(h, launch_gram(c.W, m, k, k, c.GW, c.gpart, h->max_gram_blocks, s, c.err));
  CK(h, launch_gram(c.Ht, n, k, k, c.GH, c.gpart, h->max_gram_blocks, s, c.err));
  CK(h, launch_loss(c.PHt, c.Ht, n * (int64_t)k, c.GW, c.GH, k, c.n2a, c.dpart, h->n_dparts, loss,
                    s));
  if (WtA) CK(h, launch_transpose(c.PHt, n, k, WtA, s));
  return AUNMF_OK;
}

int aunmf_loss_bwd(aunmf_handle *h, const aunmf_matrix *A, int k, const float *W, const float *H,
                   int prec, const float *WtA, const float *grad_out, float *dW, float *dH) {
  if (!h || (!dW && !dH)) return AUNMF_E_INVAL;
  RunCtx c{};
  int rc = loss_setup(h, A, k, W, H, prec, c);
  if (rc != AUNMF_OK) return rc;
  cudaStream_t s = h->stream;
  const int64_t m = A->m, n = A->n;
  if (dW) {  // dL/dW = W (H H^T) - A H^T
    CK(h, launch_gram(c.Ht, n, k, k, c.GH, c.gpart, h->max_gram_blocks, s, c.err));
    CK(h, product_aht(h, c, s));
    CK(h, launch_xg_minus_p(c.W, c.PW, c.GH, m, k, grad_out, dW, s));
  }
  if (dH) {  // dL/dH = (W^T W) H - W^T A, formed transposed
    ENS(h, h->dHt, sizeof(float) * n * k);
    CK(h, launch_gram(c.W, m, k, k, c.GW, c.gpart, h->max_gram_blocks, s, c.err));
    if (WtA) {
      CK(h, launch_transpose(WtA, k, n, c.PHt, s));
    } else {
      CK(h, product_wta(h, c, s));
    }
    CK(h, launch_xg_minus_p(c.Ht, c.PHt, c.GW, n, k, grad_out, P<float>(h->dHt), s));
    CK(h, launch_transpose(P<float>(h->dHt), n, k, dH, s));
  }
  return AUNMF_OK;
}

}  // extern "C"

// ------------------------------------------------------------ batched runs
namespace {
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Host bytes starting on a 64-byte boundary (tensor-map descriptors).
struct alignas(64) Block64 {
  uint8_t b[64];
};
struct DescBytes {
  std::vector<Block64> v;
  size_t n = 0;
  void assign(size_t bytes, uint8_t) {
    v.assign((bytes + 63) / 64, Block64{});
    n = bytes;
  }
  uint8_t *data() { return reinterpret_cast<uint8_t *>(v.data()); }
  size_t size() const { return n; }
  uint8_t &operator[](size_t i) { return data()[i]; }
};

struct BatchPlan {
  std::vector<batched::BInst> inst;
  std::vector<batched::Item> rows_w, rows_h, gram_w, gram_h, dot;
  std::vector<int64_t> tiles_a, tiles_fh, tiles_fw, rows_mx;
  DescBytes probs_aht, probs_wta;  // grouped GEMM descriptors
  int64_t units_aht = 0, units_wta = 0;
  int bn_aht = 16, bn_wta = 16;
  int kmax = 1;
  // device copies (offsets into the meta buffer)
  size_t o_inst, o_rw, o_rh, o_gw, o_gh, o_dot, o_ta, o_tfh, o_tfw, o_rmx, o_pa, o_pw, o_h0, o_h, o_end;
};

// Items of up to `chunk` rows per problem (rows(b) rows); chunk index counts
// the problem's items.
template <class F>
void make_items(std::vector<batched::Item> &out, const std::vector<batched::BInst> &inst,
                int64_t chunk, F rows) {
  out.clear();
  for (int p = 0; p < (int)inst.size(); ++p) {
    const int64_t R = rows(inst[p]);
    int c = 0;
    for (int64_t r = 0; r < R; r += chunk, ++c) {
      batched::Item it;
      it.p = p;
      it.chunk = c;
      it.r0 = r;
      it.r1 = r + chunk < R ? r + chunk : R;
      out.push_back(it);
    }
  }
}

template <class F>
std::vector<int64_t> prefix_of(const std::vector<batched::BInst> &inst, F count) {
  std::vector<int64_t> pre(inst.size() + 1, 0);
  for (size_t p = 0; p < inst.size(); ++p) pre[p + 1] = pre[p] + count(inst[p]);
  return pre;
}
}  // namespace

extern "C" {

int aunmf_run_batched(aunmf_handle *h, int count, const aunmf_matrix *A, const int *k, int algo,
                      int iters, const float *const *W0, const float *const *H0, float *const *W,
                      float *const *H, double *relres, const aunmf_options *opt,
                      aunmf_info *info) {
  (void)W0;
  if (!h || count < 1 || !A || !k || iters < 0 || !H0 || !W || !H) return AUNMF_E_INVAL;
  aunmf_options o{};
  if (opt) o = *opt;
  if (algo != AUNMF_ABPP) return AUNMF_E_UNSUPPORTED;
  if (o.prec != AUNMF_TF32 && o.prec != AUNMF_BF16) return AUNMF_E_UNSUPPORTED;
  const bool bf = o.prec == AUNMF_BF16;
  const size_t esz = bf ? 2 : 4;
  for (int p = 0; p < count; ++p) {
    if (!A[p].dense || A[p].m < 1 || A[p].n < 1 || A[p].lda < A[p].n) return AUNMF_E_INVAL;
    if (k[p] < 1 || k[p] > batched::kMaxK || !W[p] || !H0[p] || !H[p]) return AUNMF_E_INVAL;
    if (A[p].m > 0x7fffffffLL || A[p].n > 0x7fffffffLL) return AUNMF_E_UNSUPPORTED;
  }
  if (tc::check(1, 1, 1, 1, o.prec, nullptr) != AUNMF_OK) return AUNMF_E_UNSUPPORTED;
  cudaStream_t s = h->stream;
  if (o.validate) {
    for (int p = 0; p < count; ++p) {
      const int rc = validate_inputs(h, &A[p], k[p], nullptr, H0[p], s);
      if (rc != AUNMF_OK) return rc;
    }
  }
  const int max_piv_opt = o.bpp_max_pivots;
  const int bpp_cold = o.bpp_cold_start ? 1 : 0;
  constexpr int64_t kGramChunk = 256, kDotChunk = 16384;

  // ---- arena layout
  BatchPlan pl;
  pl.inst.resize(count);
  std::vector<size_t> off(count * 20);
  size_t top = 0;
  auto take = [&](size_t bytes) { const size_t at = top; top += al256(bytes ? bytes : 16); return at; };
  const size_t relres_off = take(sizeof(double) * (size_t)count * (iters > 0 ? iters : 1));
  for (int p = 0; p < count; ++p) {
    batched::BInst &b = pl.inst[p];
    b.m = A[p].m;
    b.n = A[p].n;
    b.k = k[p];
    pl.kmax = b.k > pl.kmax ? b.k : pl.kmax;
    b.lda = A[p].lda;
    b.ldx = tc::copy_ld(b.n);
    b.ldat = tc::copy_ld(b.m);
    b.ldh = tc::copy_ld(b.n);
    b.ldw = tc::copy_ld(b.m);
    b.ngw = (int)((b.m + kGramChunk - 1) / kGramChunk);
    b.ngh = (int)((b.n + kGramChunk - 1) / kGramChunk);
    b.nr = (int)((b.n * b.k + kDotChunk - 1) / kDotChunk);
    const size_t kk = (size_t)b.k * b.k, mx = (size_t)(b.m > b.n ? b.m : b.n);
    size_t *o_ = &off[p * 20];
    o_[0] = take(sizeof(float) * b.n * b.k);            // Ht
    o_[1] = take(sizeof(float) * b.m * b.k);            // PW
    o_[2] = take(sizeof(float) * b.n * b.k);            // PHt
    o_[3] = take(sizeof(double) * kk);                  // GH
    o_[4] = take(sizeof(double) * kk);                  // GW
    o_[5] = take(sizeof(double) * kk * b.ngw);          // Gram partials (W)
    o_[6] = take(sizeof(double) * kk * b.ngh);          // Gram partials (Ht)
    o_[7] = take(esz * (size_t)b.m * b.ldx);            // Ax
    o_[8] = take(esz * (size_t)b.n * b.ldat);           // At
    o_[9] = take(esz * 2 * (size_t)b.k * b.ldh);        // Hk
    o_[10] = take(esz * 2 * (size_t)b.k * b.ldw);       // Wt
    o_[11] = take(sizeof(double) * kk);                 // Q
    o_[12] = take(2 * sizeof(int));                     // q_ok, factorisation flag
    o_[16] = take(sizeof(double) * (kk + 2 * b.k));     // L, 1 / diag(L), column sums
    o_[13] = take(mx);                                  // redo
    o_[14] = take(2 * sizeof(double));                  // n2a
    o_[15] = take(sizeof(double) * b.nr);               // residual partials
  }
  std::vector<int64_t> tiles_prep;
  pl.tiles_a = prefix_of(pl.inst, [](const batched::BInst &b) {
    return ((b.m + 31) / 32) * ((b.n + 31) / 32);
  });
  const size_t tsq_off = take(2 * sizeof(double) * (size_t)pl.tiles_a[count]);
  ENS(h, h->batch, top);
  uint8_t *base = P<uint8_t>(h->batch);
  for (int p = 0; p < count; ++p) {
    batched::BInst &b = pl.inst[p];
    const size_t *o_ = &off[p * 20];
    b.A = A[p].dense;
    b.W = W[p];
    b.Ht = reinterpret_cast<float *>(base + o_[0]);
    b.PW = reinterpret_cast<float *>(base + o_[1]);
    b.PHt = reinterpret_cast<float *>(base + o_[2]);
    b.GH = reinterpret_cast<double *>(base + o_[3]);
    b.GW = reinterpret_cast<double *>(base + o_[4]);
    b.gpart_w = reinterpret_cast<double *>(base + o_[5]);
    b.gpart_h = reinterpret_cast<double *>(base + o_[6]);
    b.Ax = base + o_[7];
    b.At = base + o_[8];
    b.Hk = base + o_[9];
    b.Wt = base + o_[10];
    b.Q = reinterpret_cast<double *>(base + o_[11]);
    b.q_ok = reinterpret_cast<int *>(base + o_[12]);
    b.Lq = reinterpret_cast<double *>(base + o_[16]);
    b.redo = base + o_[13];
    b.n2a = reinterpret_cast<double *>(base + o_[14]);
    b.rpart = reinterpret_cast<double *>(base + o_[15]);
    b.relres = reinterpret_cast<double *>(base + relres_off) + (size_t)p * (iters > 0 ? iters : 1);
  }
  double *tile_sq = reinterpret_cast<double *>(base + tsq_off);

  // ---- work lists and tile prefixes
  make_items(pl.gram_w, pl.inst, kGramChunk, [](const batched::BInst &b) { return b.m; });
  make_items(pl.gram_h, pl.inst, kGramChunk, [](const batched::BInst &b) { return b.n; });
  make_items(pl.dot, pl.inst, kDotChunk, [](const batched::BInst &b) { return b.n * b.k; });
  pl.tiles_fh = prefix_of(pl.inst, [](const batched::BInst &b) { return ((b.n + 31) / 32) * ((b.k + 31) / 32); });
  pl.tiles_fw = prefix_of(pl.inst, [](const batched::BInst &b) { return ((b.m + 31) / 32) * ((b.k + 31) / 32); });
  pl.rows_mx = prefix_of(pl.inst, [](const batched::BInst &b) { return (b.m > b.n ? b.m : b.n) * b.k; });

  // ---- grouped GEMM descriptors
  const size_t pb = tc::problem_bytes();
  pl.probs_aht.assign(pb * count, 0);
  pl.probs_wta.assign(pb * count, 0);
  for (int p = 0; p < count; ++p) {
    const batched::BInst &b = pl.inst[p];
    int64_t u = 0;
    int bn = 0;
    if (!tc::fill_group_problem(&pl.probs_aht[pb * p], b.Ax, b.m, b.n, b.ldx, b.Hk, b.k, b.ldh,
                                true, bf, b.PW, pl.units_aht, &u, &bn))
      return AUNMF_E_UNSUPPORTED;
    pl.units_aht += u;
    pl.bn_aht = bn > pl.bn_aht ? bn : pl.bn_aht;
    if (!tc::fill_group_problem(&pl.probs_wta[pb * p], b.At, b.n, b.m, b.ldat, b.Wt, b.k, b.ldw,
                                true, bf, b.PHt, pl.units_wta, &u, &bn))
      return AUNMF_E_UNSUPPORTED;
    pl.units_wta += u;
    pl.bn_wta = bn > pl.bn_wta ? bn : pl.bn_wta;
  }

  // ---- BPP work tile (autotuned once per batch signature)
  int64_t sum_m = 0, sum_n = 0;
  for (const auto &b : pl.inst) { sum_m += b.m; sum_n += b.n; }
  const auto sig = std::make_tuple(count, sum_m, sum_n, pl.kmax, o.prec);
  const int wmax = batched::bpp_max_warps(pl.kmax);
  auto tune_it = h->bpp_tuned.find(sig);
  std::pair<int, int> tile = tune_it != h->bpp_tuned.end() ? tune_it->second
                                                           : std::make_pair(wmax, 4);
  auto gtune_it = h->gemm_tuned.find(sig);
  std::pair<int, int> gstages =
      gtune_it != h->gemm_tuned.end() ? gtune_it->second : std::make_pair(0, 0);

  // ---- descriptors to the device: one staging copy
  auto stage_meta = [&](std::vector<uint8_t> &buf) {
    buf.clear();
    auto put = [&](const void *src, size_t bytes) {
      const size_t at = al256(buf.size());
      buf.resize(at + al256(bytes ? bytes : 16), 0);
      if (bytes) memcpy(&buf[at], src, bytes);
      return at;
    };
    make_items(pl.rows_w, pl.inst, (int64_t)tile.first * tile.second,
               [](const batched::BInst &b) { return b.m; });
    make_items(pl.rows_h, pl.inst, (int64_t)tile.first * tile.second,
               [](const batched::BInst &b) { return b.n; });
    pl.o_inst = put(pl.inst.data(), sizeof(batched::BInst) * count);
    pl.o_rw = put(pl.rows_w.data(), sizeof(batched::Item) * pl.rows_w.size());
    pl.o_rh = put(pl.rows_h.data(), sizeof(batched::Item) * pl.rows_h.size());
    pl.o_gw = put(pl.gram_w.data(), sizeof(batched::Item) * pl.gram_w.size());
    pl.o_gh = put(pl.gram_h.data(), sizeof(batched::Item) * pl.gram_h.size());
    pl.o_dot = put(pl.dot.data(), sizeof(batched::Item) * pl.dot.size());
    pl.o_ta = put(pl.tiles_a.data(), sizeof(int64_t) * pl.tiles_a.size());
    pl.o_tfh = put(pl.tiles_fh.data(), sizeof(int64_t) * pl.tiles_fh.size());
    pl.o_tfw = put(pl.tiles_fw.data(), sizeof(int64_t) * pl.tiles_fw.size());
    pl.o_rmx = put(pl.rows_mx.data(), sizeof(int64_t) * pl.rows_mx.size());
    pl.o_pa = put(pl.probs_aht.data(), pl.probs_aht.size());
    pl.o_pw = put(pl.probs_wta.data(), pl.probs_wta.size());
    pl.o_h0 = put(H0, sizeof(float *) * count);
    pl.o_h = put(H, sizeof(float *) * count);
    pl.o_end = buf.size();
  };
  std::vector<uint8_t> meta;
  {  // size the device copy for the most items any candidate tile produces
    const std::pair<int, int> keep = tile;
    tile = {8, 2};
    stage_meta(meta);
    const size_t most = meta.size();
    tile = keep;
    stage_meta(meta);
    ENS(h, h->batch_meta, (most > meta.size() ? most : meta.size()) + 1024);
  }
  uint8_t *mb = P<uint8_t>(h->batch_meta);
  CK(h, cudaMemcpyAsync(mb, meta.data(), meta.size(), cudaMemcpyHostToDevice, s));
  auto D = [&](size_t o) { return mb + o; };
  auto inst_d = [&]() { return reinterpret_cast<const batched::BInst *>(D(pl.o_inst)); };

  ENS(h, h->ctr, sizeof(DevCounters));
  ENS(h, h->err, sizeof(int));
  DevCounters *ctr = P<DevCounters>(h->ctr);
  int *err = P<int>(h->err);
  const int max_piv = max_piv_opt > 0 ? max_piv_opt : 10 * pl.kmax;
  const long long launches0 = g_launches;
  long long graph_launches = 0;
  CallResources R;
  CK(h, cudaEventCreate(&R.t0));
  CK(h, cudaEventCreate(&R.t1));
  CK(h, cudaEventRecord(R.t0, s));
  CK(h, cudaMemsetAsync(ctr, 0, sizeof(DevCounters), s));
  CK(h, cudaMemsetAsync(err, 0, sizeof(int), s));

  // ---- setup: layout copies and norms, Ht = H0^T, W = 0, G_H
  CK(h, batched::launch_prepare(inst_d(), reinterpret_cast<const int64_t *>(D(pl.o_ta)), count,
                                pl.tiles_a[count], bf, tile_sq, s));
  CK(h, batched::launch_init(inst_d(), reinterpret_cast<const float *const *>(D(pl.o_h0)),
                             reinterpret_cast<const int64_t *>(D(pl.o_rmx)), count,
                             pl.rows_mx[count], s));
  CK(h, batched::launch_gram(inst_d(), reinterpret_cast<const batched::Item *>(D(pl.o_gh)),
                             (int)pl.gram_h.size(), count, 0, s));

  auto w_half = [&](cudaStream_t st, const batched::BInst *I, const batched::Item *rw, int nrw) {
    cudaError_t e;
    if ((e = batched::launch_split_transpose(I, reinterpret_cast<const int64_t *>(D(pl.o_tfh)),
                                             count, pl.tiles_fh[count], 0, bf, st)) != cudaSuccess)
      return e;
    if ((e = tc::launch_gemm_group(D(pl.o_pa), pl.probs_aht.data(), count, pl.units_aht,
                                   pl.bn_aht, bf, err, st, gstages.first)) != cudaSuccess)
      return e;
    return batched::launch_bpp(I, rw, nrw, count, 0, pl.kmax, max_piv, bpp_cold, ctr, tile.first,
                               st);
  };
  auto h_half = [&](cudaStream_t st, const batched::BInst *I, const batched::Item *rh, int nrh) {
    cudaError_t e;
    if ((e = batched::launch_gram(I, reinterpret_cast<const batched::Item *>(D(pl.o_gw)),
                                  (int)pl.gram_w.size(), count, 1, st)) != cudaSuccess)
      return e;
    if ((e = batched::launch_split_transpose(I, reinterpret_cast<const int64_t *>(D(pl.o_tfw)),
                                             count, pl.tiles_fw[count], 1, bf, st)) != cudaSuccess)
      return e;
    if ((e = tc::launch_gemm_group(D(pl.o_pw), pl.probs_wta.data(), count, pl.units_wta,
                                   pl.bn_wta, bf, err, st, gstages.second)) != cudaSuccess)
      return e;
    if ((e = batched::launch_bpp(I, rh, nrh, count, 1, pl.kmax, max_piv, bpp_cold, ctr, tile.first,
                                 st)) !=
        cudaSuccess)
      return e;
    if ((e = batched::launch_gram(I, reinterpret_cast<const batched::Item *>(D(pl.o_gh)),
                                  (int)pl.gram_h.size(), count, 0, st)) != cudaSuccess)
      return e;
    return batched::launch_relres(I, reinterpret_cast<const batched::Item *>(D(pl.o_dot)),
                                  (int)pl.dot.size(), count, ctr, iters, st);
  };

  // timing events of the autotuners (freed with the call's resources)
  auto tune_events = [&]() -> int {
    if (R.ev.size() >= 2) return AUNMF_OK;
    R.ev.assign(2, nullptr);
    CK(h, cudaEventCreate(&R.ev[0]));
    CK(h, cudaEventCreate(&R.ev[1]));
    return AUNMF_OK;
  };

  // ---- autotune the grouped products' pipeline depth: every stage count
  // from 2 to as many as fit, each product timed twice (their inputs are the
  // split copies of H^T and of W = 0; only P is written, and every iteration
  // forms it again)
  if (gtune_it == h->gemm_tuned.end() && iters > 0) {
    int rc = tune_events();
    if (rc != AUNMF_OK) return rc;
    cudaEvent_t a0 = R.ev[0], a1 = R.ev[1];
    CK(h, batched::launch_split_transpose(inst_d(), reinterpret_cast<const int64_t *>(D(pl.o_tfh)),
                                          count, pl.tiles_fh[count], 0, bf, s));
    CK(h, batched::launch_split_transpose(inst_d(), reinterpret_cast<const int64_t *>(D(pl.o_tfw)),
                                          count, pl.tiles_fw[count], 1, bf, s));
    auto tune = [&](const void *dp, DescBytes &probs, int64_t units, int bn,
                    int *chosen) -> int {
      const int smax = tc::group_max_stages(probs.data(), count, units, bn);
      float best = 1e30f;
      *chosen = 0;
      for (int st = 2; st <= smax; ++st) {
        CK(h, cudaEventRecord(a0, s));
        for (int rep = 0; rep < 2; ++rep)
          CK(h, tc::launch_gemm_group(dp, probs.data(), count, units, bn, bf, err, s, st));
        CK(h, cudaEventRecord(a1, s));
        CK(h, cudaEventSynchronize(a1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a0, a1);
        if (ms < best) { best = ms; *chosen = st; }
      }
      return AUNMF_OK;
    };
    rc = tune(D(pl.o_pa), pl.probs_aht, pl.units_aht, pl.bn_aht, &gstages.first);
    if (rc != AUNMF_OK) return rc;
    rc = tune(D(pl.o_pw), pl.probs_wta, pl.units_wta, pl.bn_wta, &gstages.second);
    if (rc != AUNMF_OK) return rc;
    h->gemm_tuned[sig] = gstages;
  }

  // ---- autotune the BPP work tile on the first W update (factors restored)
  if (tune_it == h->bpp_tuned.end() && iters > 0) {
    std::vector<std::pair<int, int>> cand;
    for (int wp : {8, 16})
      for (int rpw : {2, 8})
        if (wp <= wmax) cand.push_back({wp, rpw});
    if (cand.empty()) cand.push_back({wmax, 4});
    float best = 1e30f;
    std::pair<int, int> best_tile = cand[0];
    int rc = tune_events();
    if (rc != AUNMF_OK) return rc;
    cudaEvent_t a0 = R.ev[0], a1 = R.ev[1];
    for (const auto &c : cand) {
      tile = c;
      stage_meta(meta);
      CK(h, cudaMemcpyAsync(mb, meta.data(), meta.size(), cudaMemcpyHostToDevice, s));
      for (const auto &b : pl.inst)  // W is all zero before the first update: restore it
        CK(h, cudaMemsetAsync(b.W, 0, sizeof(float) * b.m * b.k, s));
      CK(h, cudaEventRecord(a0, s));
      CK(h, w_half(s, inst_d(), reinterpret_cast<const batched::Item *>(D(pl.o_rw)),
                   (int)pl.rows_w.size()));
      CK(h, cudaEventRecord(a1, s));
      CK(h, cudaEventSynchronize(a1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a0, a1);
      if (ms < best) { best = ms; best_tile = c; }
    }
    tile = best_tile;
    h->bpp_tuned[sig] = tile;
    for (const auto &b : pl.inst) CK(h, cudaMemsetAsync(b.W, 0, sizeof(float) * b.m * b.k, s));
    CK(h, cudaMemsetAsync(ctr, 0, sizeof(DevCounters), s));
    stage_meta(meta);
    CK(h, cudaMemcpyAsync(mb, meta.data(), meta.size(), cudaMemcpyHostToDevice, s));
  }

  // ---- iterations: one captured iteration, replayed
  if (iters > 0) {
    const batched::Item *rw = reinterpret_cast<const batched::Item *>(D(pl.o_rw));
    const batched::Item *rh = reinterpret_cast<const batched::Item *>(D(pl.o_rh));
    if (o.use_graph && iters > 1) {
      CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      const long long lc0 = g_launches;
      cudaError_t ce = w_half(h->cap_stream, inst_d(), rw, (int)pl.rows_w.size());
      if (ce == cudaSuccess) ce = h_half(h->cap_stream, inst_d(), rh, (int)pl.rows_h.size());
      const long long per_iter = g_launches - lc0;
      g_launches = lc0;
      cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &R.graph);
      if (ce != cudaSuccess) return fail_cuda(h, ce, "batched iteration (capture)");
      if (ee != cudaSuccess) return fail_cuda(h, ee, "cudaStreamEndCapture");
      CK(h, cudaGraphInstantiate(&R.gexec, R.graph, 0));
      graph_launches = per_iter * iters;
      for (int t = 0; t < iters; ++t) CK(h, cudaGraphLaunch(R.gexec, s));
    } else {
      for (int t = 0; t < iters; ++t) {
        CK(h, w_half(s, inst_d(), rw, (int)pl.rows_w.size()));
        CK(h, h_half(s, inst_d(), rh, (int)pl.rows_h.size()));
      }
    }
  }
  CK(h, batched::launch_finish(inst_d(), reinterpret_cast<float *const *>(D(pl.o_h)),
                               reinterpret_cast<const int64_t *>(D(pl.o_rmx)), count,
                               pl.rows_mx[count], s));
  CK(h, cudaEventRecord(R.t1, s));
  DevCounters hc{};
  int herr = 0;
  CK(h, cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, s));
  CK(h, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (relres && iters > 0)
    CK(h, cudaMemcpyAsync(relres, base + relres_off, sizeof(double) * (size_t)count * iters,
                          cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  if (info) {
    memset(info, 0, sizeof(*info));
    info->bpp_pivots = hc.bpp_pivots;
    info->bpp_nonconverged = hc.bpp_nonconv;
    info->bpp_numeric = hc.bpp_numeric;
    info->bpp_redone = hc.bpp_redo;
    info->iters_done = iters;
    cudaEventElapsedTime(&info->ms_total, R.t0, R.t1);
    info->launches = g_launches - launches0 + graph_launches;
    info->tuned_bpp_warps = tile.first;
    info->tuned_bpp_rows = tile.second;
    info->tuned_gemm_stages_aht = gstages.first;
    info->tuned_gemm_stages_wta = gstages.second;
  }
  if (herr) return AUNMF_E_TIMEOUT;
  if (hc.bpp_numeric) return AUNMF_E_NUMERIC;
  if (hc.bpp_nonconv) return AUNMF_E_NOCONVERGE;
  return AUNMF_OK;
}

}  // extern "C"
