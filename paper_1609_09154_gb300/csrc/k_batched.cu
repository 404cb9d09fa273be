// k_batched.cu -- many independent AU-NMF problems (Alg. 1 per problem, ANLS
// with block principal pivoting, Sec. 4.3) advanced together: every phase of
// an iteration is ONE launch over all problems.  Work is described by item
// lists built once on the host (problem, row range) or by per-problem prefix
// counts of tiles; kernels are persistent (grid-stride over items).
//
// Phases per iteration (see aunmf_run_batched in aunmf_api.cu):
//   split-transpose Ht -> H copy, grouped tensor-core A H^T, G^{-1} of H H^T,
//   BPP rows of W, Gram W^T W, split-transpose W -> W^T copy, grouped A^T W,
//   G^{-1} of W^T W, BPP rows of H^T, Gram H H^T, relative residual.
#include <cuda_bf16.h>

#include "batched.cuh"
#include "bpp_core.cuh"

namespace aunmf {
namespace batched {
namespace {

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
template <class T>
__device__ __forceinline__ T rnd(float x);
template <>
__device__ __forceinline__ float rnd<float>(float x) { return round_tf32(x); }
template <>
__device__ __forceinline__ uint16_t rnd<uint16_t>(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
template <class T>
__device__ __forceinline__ float wid(T x);
template <>
__device__ __forceinline__ float wid<float>(float x) { return x; }
template <>
__device__ __forceinline__ float wid<uint16_t>(uint16_t x) {
  return __bfloat162float(__ushort_as_bfloat16(x));
}

// problem p with prefix[p] <= idx < prefix[p + 1]
__device__ __forceinline__ int locate(const int64_t *prefix, int count, int64_t idx) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= idx) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ double block_sum(double v, double *ws) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
  return s;
}

// ---------------------------------------------------------------- setup
// Rounded copy Ax, rounded transposed copy At and per-tile sums of a_ij^2
// and of a_ij (round(a_ij) - a_ij) of each problem's A (tile_sq[2 g],
// tile_sq[2 g + 1]), 32 x 32 tiles numbered across problems by tile_prefix.
template <class T>
__global__ void __launch_bounds__(256)
    g_prepare(const BInst *__restrict__ P, const int64_t *__restrict__ tile_prefix, int count,
              double *__restrict__ tile_sq) {
  __shared__ float t[32][33];
  __shared__ double ws[8];
  const int64_t total = tile_prefix[count];
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int p = locate(tile_prefix, count, g);
    const BInst &b = P[p];
    const int64_t tl = g - tile_prefix[p];
    const int64_t tcn = (b.n + 31) / 32;
    const int64_t r0 = (tl / tcn) * 32, c0 = (tl % tcn) * 32;
    T *X = reinterpret_cast<T *>(b.Ax);
    T *Xt = reinterpret_cast<T *>(b.At);
    float sq = 0.f, sd = 0.f;  // this thread's 4 terms of each sum, in FP32
    __syncthreads();
    for (int y = threadIdx.x >> 5; y < 32; y += 8) {
      const int64_t r = r0 + y, c = c0 + (threadIdx.x & 31);
      float v = 0.f;
      if (r < b.m && c < b.n) {
        v = b.A[r * b.lda + c];
        const T rv = rnd<T>(v);
        X[r * b.ldx + c] = rv;
        sd = fmaf(v, wid<T>(rv) - v, sd);
      }
      sq = fmaf(v, v, sq);
      t[y][threadIdx.x & 31] = v;
    }
    const double acc = (double)sq, acc_d = (double)sd;
    __syncthreads();
    for (int y = threadIdx.x >> 5; y < 32; y += 8) {
      const int64_t c = c0 + y, r = r0 + (threadIdx.x & 31);
      if (r < b.m && c < b.n) Xt[c * b.ldat + r] = rnd<T>(t[threadIdx.x & 31][y]);
    }
    const double s = block_sum(acc, ws);
    const double d = block_sum(acc_d, ws);
    if (threadIdx.x == 0) {
      tile_sq[2 * g] = s;
      tile_sq[2 * g + 1] = d;
    }
  }
}

// n2a = {||A_p||^2, 2 <round(A_p) - A_p, A_p>}: sums of the problem's tile
// partials in tile order (one block per problem).
__global__ void g_norm_final(const BInst *__restrict__ P, const int64_t *__restrict__ tile_prefix,
                             const double *__restrict__ tile_sq) {
  __shared__ double ws[8];
  const int p = blockIdx.x;
  double s = 0.0, d = 0.0;
  for (int64_t g = tile_prefix[p] + threadIdx.x; g < tile_prefix[p + 1]; g += blockDim.x) {
    s += tile_sq[2 * g];
    d += tile_sq[2 * g + 1];
  }
  s = block_sum(s, ws);
  d = block_sum(d, ws);
  if (threadIdx.x == 0) {
    P[p].n2a[0] = s;
    P[p].n2a[1] = 2.0 * d;
  }
}

// Ht = H0^T (n x k) and W = 0 for each problem (ABPP starts from H only).
__global__ void g_init(const BInst *__restrict__ P, const float *const *__restrict__ H0,
                       const int64_t *__restrict__ row_prefix, int count) {
  const int64_t total = row_prefix[count];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int p = locate(row_prefix, count, g);
    const BInst &b = P[p];
    const int64_t e = g - row_prefix[p];  // element of max(m, n) x k
    const int64_t r = e / b.k;
    const int j = (int)(e % b.k);
    if (r < b.n) b.Ht[r * b.k + j] = H0[p][(int64_t)j * b.n + r];
    if (r < b.m) b.W[r * b.k + j] = 0.f;
  }
}

// H = Ht^T for each problem (k x n into the caller's arrays).
__global__ void g_finish(const BInst *__restrict__ P, float *const *__restrict__ H,
                         const int64_t *__restrict__ row_prefix, int count) {
  const int64_t total = row_prefix[count];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int p = locate(row_prefix, count, g);
    const BInst &b = P[p];
    const int64_t e = g - row_prefix[p];
    const int64_t r = e / b.k;
    const int j = (int)(e % b.k);
    if (r < b.n) H[p][(int64_t)j * b.n + r] = b.Ht[r * b.k + j];
  }
}

// ---------------------------------------------------------------- per iteration
// Two-term split, transposed: rows (2c, 2c+1) of the copy = hi, lo of column
// c of the factor (rows x k).  side 0: factor Ht (n rows) -> Hk; side 1:
// factor W (m rows) -> Wt.
template <class T>
__global__ void __launch_bounds__(256)
    g_split_transpose(const BInst *__restrict__ P, const int64_t *__restrict__ tile_prefix,
                      int count, int side) {
  __shared__ float t[32][33];
  const int64_t total = tile_prefix[count];
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int p = locate(tile_prefix, count, g);
    const BInst &b = P[p];
    const int64_t rows = side ? b.m : b.n;
    const float *in = side ? b.W : b.Ht;
    T *out = reinterpret_cast<T *>(side ? b.Wt : b.Hk);
    const int64_t ldo = side ? b.ldw : b.ldh;
    const int k = b.k;
    const int64_t tl = g - tile_prefix[p];
    const int64_t tcn = (k + 31) / 32;
    const int64_t r0 = (tl / tcn) * 32, c0 = (tl % tcn) * 32;
    __syncthreads();
    for (int y = threadIdx.x >> 5; y < 32; y += 8) {
      const int64_t r = r0 + y, c = c0 + (threadIdx.x & 31);
      if (r < rows && c < k) t[y][threadIdx.x & 31] = in[r * k + c];
    }
    __syncthreads();
    for (int y = threadIdx.x >> 5; y < 32; y += 8) {
      const int64_t c = c0 + y, r = r0 + (threadIdx.x & 31);
      if (r < rows && c < k) {
        const float x = t[threadIdx.x & 31][y];
        const T hi = rnd<T>(x);
        out[(2 * c) * ldo + r] = hi;
        out[(2 * c + 1) * ldo + r] = rnd<T>(x - wid<T>(hi));
      }
    }
  }
}

// Gram partials: item (p, chunk, r0, r1) adds X^T X over rows [r0, r1) of
// the problem's X (side 0: Ht, side 1: W) into partial slot `chunk`.  Each
// thread owns a 4 x 4 tile of the upper triangle (mirrored on output); each
// 32-row slab's exact products are summed in FP32 pairs (two_fma_acc) and
// added to FP64 sums, so the Gram keeps the small eigenvalues that the BPP
// solves need when the factor is ill-conditioned (an FP32 sum would leave
// them as rounding noise).
__global__ void __launch_bounds__(256)
    g_gram_partial(const BInst *__restrict__ P, const Item *__restrict__ items, int nitems,
                   int side) {
  __shared__ float sX[32 * kMaxK];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const Item I = items[it];
    const BInst &b = P[I.p];
    const int k = b.k;
    if (!AUNMF_BOUND(I.r0 >= 0 && I.r0 <= I.r1 && I.r1 <= (side ? b.m : b.n) && k >= 1 &&
                         k <= kMaxK,
                     AUNMF_CHECK_BATCHED_ITEM))
      continue;
    const float *X = side ? b.W : b.Ht;
    double *out = (side ? b.gpart_w : b.gpart_h) + (int64_t)I.chunk * k * k;
    const int kp = (k + 3) & ~3;
    const int nt = kp / 4, ntiles = nt * (nt + 1) / 2;
    for (int tb = 0; tb < ntiles; tb += blockDim.x) {
      const int tt = tb + threadIdx.x;
      const bool act = tt < ntiles;
      int ti = 0, tj = 0;
      if (act) {
        int rem = tt;
        while (rem >= nt - ti) { rem -= nt - ti; ++ti; }
        tj = ti + rem;
      }
      double acc[4][4] = {};
      for (int64_t c0 = I.r0; c0 < I.r1; c0 += 32) {
        const int nr = (int)min((int64_t)32, I.r1 - c0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < 32 * kp; idx += blockDim.x) {
          const int rr = idx / kp, cc = idx % kp;
          sX[idx] = (rr < nr && cc < k) ? X[(c0 + rr) * k + cc] : 0.f;
        }
        __syncthreads();
        if (act) {
          float hi[4][4] = {}, lo[4][4] = {};
          for (int rr = 0; rr < nr; ++rr) {
            float av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              av[u] = sX[rr * kp + 4 * ti + u];
              bv[u] = sX[rr * kp + 4 * tj + u];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) two_fma_acc(av[a], bv[c], hi[a][c], lo[a][c]);
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] += (double)hi[a][c] + (double)lo[a][c];
        }
      }
      if (act)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int i = 4 * ti + a, j = 4 * tj + c;
            if (i < k && j < k) {
              out[i * k + j] = acc[a][c];
              out[j * k + i] = acc[a][c];
            }
          }
    }
  }
}

// G = sum of the problem's partials in chunk order, FP64 (block per problem).
__global__ void g_gram_reduce(const BInst *__restrict__ P, int side) {
  const BInst &b = P[blockIdx.x];
  const int k = b.k;
  const int nparts = side ? b.ngw : b.ngh;
  const double *part = side ? b.gpart_w : b.gpart_h;
  double *G = side ? b.GW : b.GH;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * k * k + e];
    G[e] = s;
  }
}

// G^{-1} (FP64) per problem (side 0: of H H^T; 1: of W^T W): Cholesky, one
// block per problem; column solves, one warp per (problem, column); check.
__global__ void __launch_bounds__(256) g_chol(const BInst *__restrict__ P, int side) {
  extern __shared__ double sm[];
  const BInst &b = P[blockIdx.x];
  const int k = b.k;
  bpp::chol_block(side ? b.GW : b.GH, k, b.Lq, b.Lq + (size_t)k * k, b.q_ok + 1, sm);
}

__global__ void g_inv_cols(const BInst *__restrict__ P, int kmax) {
  const BInst &b = P[blockIdx.x / kmax];
  const int j = blockIdx.x % kmax, k = b.k;
  if (j >= k) return;
  const double *L = b.Lq, *invd = b.Lq + (size_t)k * k;
  bpp::inv_col_warp(L, invd, k, j, reinterpret_cast<float *>(b.Q), b.Lq + (size_t)k * k + k);
}

__global__ void g_inv_check(const BInst *__restrict__ P, int side) {
  const BInst &b = P[blockIdx.x];
  const int k = b.k;
  bpp::inv_check(side ? b.GW : b.GH, b.Lq + (size_t)k * k + k, k, b.q_ok + 1, b.q_ok);
}

// BPP: items (p, -, r0, r1) of rows of W (side 0: against H H^T, R = A H^T)
// or of Ht (side 1: against W^T W, R = (W^T A)^T); warm start from the
// current values; rows that need the direct fallback are flagged.
template <int KT>
__global__ void __launch_bounds__(32 * bpp::kBppWarps, 1)
    g_bpp(const BInst *__restrict__ P, const Item *__restrict__ items, int nitems, int side,
          int max_piv, int cold, DevCounters *ctr) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  long long piv_total = 0, nonconv = 0;
  // the first iteration starts each solve from the signs of the unconstrained
  // solution (W = 0 and the random H0 say nothing about the solution), later
  // ones from the previous iterate's support; cold: every solve from x = 0
  const int warm = cold ? 0 : (ctr->iter == 0 ? 2 : 1);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const Item I = items[it];
    const BInst &b = P[I.p];
    const int k = b.k;
    if (!AUNMF_BOUND(I.r0 >= 0 && I.r0 <= I.r1 && I.r1 <= (side ? b.n : b.m) && k >= 1 &&
                         k <= kMaxK,
                     AUNMF_CHECK_BATCHED_ITEM))
      continue;
    __syncthreads();
    const bpp::BppWarp w =
        bpp::bpp_stage(side ? b.GW : b.GH, reinterpret_cast<const float *>(b.Q), b.q_ok, k, sm, wib);
    __syncthreads();
    const float *R = side ? b.PHt : b.PW;
    float *X = side ? b.Ht : b.W;
    for (int64_t row = I.r0 + wib; row < I.r1; row += nwb) {
      bool fnum, fcap;
      // problems with k <= 32 take the one-index-per-lane form even in a
      // launch sized for larger ranks (fewer instructions per exchange)
      const int n_ex = (KT > 1 && k <= 32)
                           ? bpp::bpp_row_fast<1>(w, R, row, k, X, warm, max_piv, &fnum, &fcap)
                           : bpp::bpp_row_fast<KT>(w, R, row, k, X, warm, max_piv, &fnum, &fcap);
      if (lane == 0) b.redo[row] = fnum ? 1 : 0;
      if (!fnum) {
        piv_total += n_ex;
        nonconv += fcap;
      }
      __syncwarp();
    }
  }
  if (lane == 0) {
    if (piv_total) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->bpp_pivots),
                             (unsigned long long)piv_total);
    if (nonconv) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->bpp_nonconv),
                           (unsigned long long)nonconv);
  }
}

template <int KT>
__global__ void __launch_bounds__(256)
    g_bpp_direct(const BInst *__restrict__ P, const Item *__restrict__ items, int nitems,
                 int side, int max_piv, int cold, DevCounters *ctr) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  long long piv_total = 0, nonconv = 0, numeric = 0, redone = 0;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const Item I = items[it];
    const BInst &b = P[I.p];
    const int k = b.k;
    if (!AUNMF_BOUND(I.r0 >= 0 && I.r0 <= I.r1 && I.r1 <= (side ? b.n : b.m) && k >= 1 &&
                         k <= kMaxK,
                     AUNMF_CHECK_BATCHED_ITEM))
      continue;
    bool any = false;
    for (int64_t r = I.r0 + threadIdx.x; r < I.r1; r += blockDim.x) any |= b.redo[r] != 0;
    if (!__syncthreads_or(any)) continue;
    const int ldl = k | 1;
    double *G = sm;
    const double *Gd = side ? b.GW : b.GH;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) G[e] = Gd[e];
    __syncthreads();
    double *L = sm + (size_t)k * k + (size_t)wib * ((size_t)k * ldl + 3 * (size_t)k);
    double *v = L + (size_t)k * ldl;
    double *rs = v + k;
    int *Fl = reinterpret_cast<int *>(rs + k);
    const float *R = side ? b.PHt : b.PW;
    float *X = side ? b.Ht : b.W;
    for (int64_t row = I.r0 + wib; row < I.r1; row += nwb) {
      if (!b.redo[row]) continue;
      bool fnum, fcap;
      const int n_ex = bpp::bpp_row_direct<KT>(G, L, v, rs, Fl, R, row, k, X, cold ? 0 : 1, max_piv,
                                                    &fnum, &fcap);
      piv_total += n_ex;
      nonconv += fcap;
      numeric += fnum;
      redone += 1;
      __syncwarp();
    }
    __syncthreads();
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

// Residual partials: item (p, chunk, e0, e1) sums PHt * Ht over elements
// [e0, e1) of the problem's n x k arrays into slot `chunk`.
__global__ void g_dot_partial(const BInst *__restrict__ P, const Item *__restrict__ items,
                              int nitems) {
  __shared__ double ws[8];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const Item I = items[it];
    const BInst &b = P[I.p];
    if (!AUNMF_BOUND(I.r0 >= 0 && I.r0 <= I.r1 && I.r1 <= b.n * (int64_t)b.k,
                     AUNMF_CHECK_BATCHED_ITEM))
      continue;
    double s = 0.0;
    for (int64_t e = I.r0 + threadIdx.x; e < I.r1; e += blockDim.x)
      s = fma((double)b.PHt[e], (double)b.Ht[e], s);
    s = block_sum(s, ws);
    if (threadIdx.x == 0) b.rpart[I.chunk] = s;
    __syncthreads();
  }
}

// relres[iter] = sqrt(max(0, ||A||^2 + d - 2 <P, Ht> + <GW, GH>) / ||A||^2),
// FP64, with d = 2 <round(A) - A, A> correcting for the rounded copy the
// products read (as in the single-problem residual); one block per problem;
// the iteration index is read from the counters.
__global__ void g_relres_final(const BInst *__restrict__ P, DevCounters *ctr, int iters) {
  __shared__ double ws[8];
  const BInst &b = P[blockIdx.x];
  double cross = 0.0;
  for (int c = threadIdx.x; c < b.nr; c += blockDim.x) cross += b.rpart[c];
  cross = block_sum(cross, ws);
  const int k = b.k;
  double quad = 0.0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) quad = fma(b.GW[e], b.GH[e], quad);
  quad = block_sum(quad, ws);
  if (threadIdx.x == 0) {
    const double a2 = b.n2a[0];
    double r2 = (a2 + b.n2a[1]) - 2.0 * cross + quad;
    if (r2 < 0.0) r2 = 0.0;
    const long long t = ctr->iter;
    if (t < iters) b.relres[t] = a2 > 0.0 ? sqrt(r2 / a2) : 0.0;
  }
}

__global__ void g_iter_tick(DevCounters *ctr) { ctr->iter += 1; }

int sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

}  // namespace

cudaError_t launch_prepare(const BInst *P, const int64_t *tile_prefix, int count, int64_t tiles,
                           bool bf16, double *tile_sq, cudaStream_t s) {
  const int grid = (int)(tiles < (int64_t)sms() * 16 ? tiles : (int64_t)sms() * 16);
  if (bf16)
    g_prepare<uint16_t><<<grid, 256, 0, s>>>(P, tile_prefix, count, tile_sq);
  else
    g_prepare<float><<<grid, 256, 0, s>>>(P, tile_prefix, count, tile_sq);
  g_norm_final<<<count, 256, 0, s>>>(P, tile_prefix, tile_sq);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_init(const BInst *P, const float *const *H0, const int64_t *row_prefix,
                        int count, int64_t total, cudaStream_t s) {
  int64_t nb = (total + 255) / 256;
  if (nb > (int64_t)sms() * 16) nb = (int64_t)sms() * 16;
  g_init<<<(unsigned)(nb < 1 ? 1 : nb), 256, 0, s>>>(P, H0, row_prefix, count);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_finish(const BInst *P, float *const *H, const int64_t *row_prefix, int count,
                          int64_t total, cudaStream_t s) {
  int64_t nb = (total + 255) / 256;
  if (nb > (int64_t)sms() * 16) nb = (int64_t)sms() * 16;
  g_finish<<<(unsigned)(nb < 1 ? 1 : nb), 256, 0, s>>>(P, H, row_prefix, count);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_split_transpose(const BInst *P, const int64_t *tile_prefix, int count,
                                   int64_t tiles, int side, bool bf16, cudaStream_t s) {
  const int grid = (int)(tiles < (int64_t)sms() * 16 ? tiles : (int64_t)sms() * 16);
  if (bf16)
    g_split_transpose<uint16_t><<<grid, 256, 0, s>>>(P, tile_prefix, count, side);
  else
    g_split_transpose<float><<<grid, 256, 0, s>>>(P, tile_prefix, count, side);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_gram(const BInst *P, const Item *items, int nitems, int count, int side,
                        cudaStream_t s) {
  const int grid = nitems < sms() * 8 ? nitems : sms() * 8;
  g_gram_partial<<<grid, 256, 0, s>>>(P, items, nitems, side);
  g_gram_reduce<<<count, 256, 0, s>>>(P, side);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_bpp(const BInst *P, const Item *items, int nitems, int count, int side,
                       int kmax, int max_piv, int cold, DevCounters *ctr, int wpb, cudaStream_t s) {
  const size_t chol_smem = sizeof(double) * (size_t)kmax * kmax;
  cudaFuncSetAttribute(g_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chol_smem);
  g_chol<<<count, 256, chol_smem, s>>>(P, side);
  g_inv_cols<<<count * kmax, 32, 0, s>>>(P, kmax);
  g_inv_check<<<count, 32, 0, s>>>(P, side);
  const bpp::BppLayout lay = bpp::bpp_layout(kmax);
  const size_t smem = sizeof(double) * (lay.shared_dbl + (size_t)wpb * lay.warp_dbl);
  const int grid = nitems < sms() * 2 ? nitems : sms() * 2;
  const size_t fb_warp = (size_t)kmax * (kmax | 1) + 3 * (size_t)kmax;
  int fbw = (int)((200 * 1024 / sizeof(double) - (size_t)kmax * kmax) / fb_warp);
  fbw = fbw > 8 ? 8 : (fbw < 1 ? 1 : fbw);
  const size_t fb_smem = sizeof(double) * ((size_t)kmax * kmax + (size_t)fbw * fb_warp);
  if (kmax <= 32) {
    cudaFuncSetAttribute(g_bpp<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    g_bpp<1><<<grid, 32 * wpb, smem, s>>>(P, items, nitems, side, max_piv, cold, ctr);
    cudaFuncSetAttribute(g_bpp_direct<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem);
    g_bpp_direct<1><<<grid, 32 * fbw, fb_smem, s>>>(P, items, nitems, side, max_piv, cold, ctr);
  } else {
    cudaFuncSetAttribute(g_bpp<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    g_bpp<2><<<grid, 32 * wpb, smem, s>>>(P, items, nitems, side, max_piv, cold, ctr);
    cudaFuncSetAttribute(g_bpp_direct<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem);
    g_bpp_direct<2><<<grid, 32 * fbw, fb_smem, s>>>(P, items, nitems, side, max_piv, cold, ctr);
  }
  g_launches += 5;
  return cudaGetLastError();
}

int bpp_max_warps(int kmax) {
  const bpp::BppLayout lay = bpp::bpp_layout(kmax);
  int wpb = (int)((200 * 1024 / sizeof(double) - lay.shared_dbl) / lay.warp_dbl);
  if (wpb > bpp::kBppWarps) wpb = bpp::kBppWarps;
  return wpb < 1 ? 1 : wpb;
}

cudaError_t launch_relres(const BInst *P, const Item *items, int nitems, int count,
                          DevCounters *ctr, int iters, cudaStream_t s) {
  const int grid = nitems < sms() * 8 ? nitems : sms() * 8;
  g_dot_partial<<<grid, 256, 0, s>>>(P, items, nitems);
  g_relres_final<<<count, 256, 0, s>>>(P, ctr, iters);
  g_iter_tick<<<1, 1, 0, s>>>(ctr);
  g_launches += 3;
  return cudaGetLastError();
}

}  // namespace batched
}  // namespace aunmf
