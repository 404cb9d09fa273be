// k_simt.cu -- FP32/FP64 CUDA-core kernels of the AU-NMF hot path:
//   * Gram matrices X^T X (Alg. 1 lines 3-4: H H^T, W^T W; the all-reduce of
//     Alg. 3 becomes a fixed-order FP64 reduction of per-block partials)
//   * the two products with A on CUDA cores (Alg. 1: A H^T, W^T A)
//   * transposes, ||A||^2 and the relative residual of Sec. 6.2 from the
//     expansion ||A||^2 - 2 <W^T A, H> + <W^T W, H H^T>.
// Internally H is held transposed (Ht, n x k) so that both factors are
// row-major "rows x k" and share the same update kernels.
#include <math.h>

#include <type_traits>

#include "internal.cuh"
#include "ptx.cuh"

namespace aunmf {

// ------------------------------------------------------------------ Gram
// Block b accumulates X^T X over rows [b*chunk, (b+1)*chunk) into
// partials[b] (k x k).  Each thread owns a 4x4 tile of G's upper triangle;
// rows are staged in shared memory 64 at a time.  There are only
// nt (nt + 1) / 2 tiles (91 at k = 50), so the block's threads form
// ngrp = 256 / tiles groups (2 at k = 50, 7 at k = 32), each covering every
// tile for its share of the staged rows (row g, g + ngrp, ...) with running
// sums of its own; the groups' sums are added in group order at the end, so
// the result does not depend on scheduling.
namespace {
constexpr int kGramRows = 64;
constexpr int kGramThreads = 256;
// rows of a group summed in a fresh register before they join the running
// sum (FP32 path) or the FP64 sum (FP64-accurate path)
constexpr int kGramSlab = 32;

__device__ __forceinline__ int gram_groups(int ntiles) {
  return ntiles >= kGramThreads ? 1 : kGramThreads / ntiles;
}

// The per-block partial of G = X^T X over the block's rows.
//   FP64 = false: each group's slab of up to 32 rows is summed in a fresh
//     FP32 register and added to an FP32 running sum with Kahan's
//     compensation (the residual's expansion <W^T W, H H^T> needs the Grams
//     to ~1e-7; FP64 additions, at ~2 per SM per clock on this part, would
//     bound the kernel).
//   FP64 = true: within a slab each product is formed exactly and summed in
//     an FP32 pair (hi, lo) (two_fma_acc), and the slab's pair is added to
//     an FP64 running sum: ~1e-14 relative, so a Gram whose smallest
//     eigenvalues sit below FP32's resolution of its largest (condition
//     beyond ~1e7, which ABPP's factors reach on uniform low-rank data) stays
//     positive definite.
// The next 64-row slab is loaded into registers while the current one is
// consumed from shared memory.  Dynamic shared memory: gram_smem_bytes().
template <bool FP64>
__global__ void __launch_bounds__(kGramThreads, 2)
    k_gram_part(const float *__restrict__ X, int64_t rows, int k, int64_t ldx, int64_t chunk,
                typename std::conditional<FP64, double, float>::type *__restrict__ partials) {
  using T = typename std::conditional<FP64, double, float>::type;
  extern __shared__ __align__(16) float sX[];  // [kGramRows][kp], then the group sums
  constexpr int kPre = (kGramRows * 64 + kGramThreads - 1) / kGramThreads;  // k <= 64 prefetch
  const int kp = (k + 3) & ~3;
  const int nt = kp / 4, ntiles = nt * (nt + 1) / 2;
  const int ngrp = gram_groups(ntiles);
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(rows, r0 + chunk);
  T *out = partials + (int64_t)blockIdx.x * k * k;
  const int slab = kGramRows * kp;
  const bool pre = slab <= kPre * kGramThreads;
  T *gsum = reinterpret_cast<T *>(sX + ((slab + 3) & ~3));  // [ngrp][ntiles][16]
  for (int tb = 0; tb < ntiles; tb += kGramThreads) {
    const int g = ngrp > 1 ? (int)threadIdx.x / ntiles : 0;
    const int t = tb + (ngrp > 1 ? (int)threadIdx.x % ntiles : (int)threadIdx.x);
    const bool act = g < ngrp && t < ntiles;
    // t -> (ti, tj), ti <= tj, row-major over the upper triangle
    int ti = 0, tj = 0;
    if (act) {
      int rem = t;
      while (rem >= nt - ti) { rem -= nt - ti; ++ti; }
      tj = ti + rem;
    }
    T sum[4][4];
    float cmp[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        sum[a][b] = T(0);
        cmp[a][b] = 0.f;
      }
    float nxt[kPre];
    // slab index idx -> (row, column) = (idx / kp, idx % kp) by a float
    // reciprocal: idx < 4096 and kp <= 64 keep (idx + 0.5) / kp at least
    // 1 / 128 away from an integer, far beyond the product's rounding, so the
    // truncation is exact (an integer division costs ~20 instructions, and
    // took most of the kernel's issue slots)
    const float inv_kp = 1.f / (float)kp;
    auto fetch = [&](int64_t c0) {
      const int nr = (int)min((int64_t)kGramRows, r1 - c0);
#pragma unroll
      for (int q = 0; q < kPre; ++q) {
        const int idx = threadIdx.x + q * kGramThreads;
        const int rr = __float2int_rz(((float)idx + 0.5f) * inv_kp), cc = idx - rr * kp;
        nxt[q] = (idx < slab && rr < nr && cc < k) ? X[(c0 + rr) * ldx + cc] : 0.f;
      }
    };
    if (pre && r0 < r1) fetch(r0);
    for (int64_t c0 = r0; c0 < r1; c0 += kGramRows) {
      const int nr = (int)min((int64_t)kGramRows, r1 - c0);
      __syncthreads();
      if (pre) {
#pragma unroll
        for (int q = 0; q < kPre; ++q) {
          const int idx = threadIdx.x + q * kGramThreads;
          if (idx < slab) sX[idx] = nxt[q];
        }
        if (c0 + kGramRows < r1) fetch(c0 + kGramRows);
      } else {
        for (int idx = threadIdx.x; idx < slab; idx += kGramThreads) {
          const int rr = __float2int_rz(((float)idx + 0.5f) * inv_kp), cc = idx - rr * kp;
          sX[idx] = (rr < nr && cc < k) ? X[(c0 + rr) * ldx + cc] : 0.f;
        }
      }
      __syncthreads();
      if (act) {
        // the group's rows of this stage, kGramSlab at a time
        for (int s0 = g; s0 < nr; s0 += kGramSlab * ngrp) {
          const int s1 = min(nr, s0 + kGramSlab * ngrp);
          float hi[4][4] = {}, lo[4][4] = {};
          for (int rr = s0; rr < s1; rr += ngrp) {
            const float4 a = *reinterpret_cast<const float4 *>(&sX[rr * kp + 4 * ti]);
            const float4 b = *reinterpret_cast<const float4 *>(&sX[rr * kp + 4 * tj]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                if constexpr (FP64)
                  two_fma_acc(av[p], bv[q], hi[p][q], lo[p][q]);
                else
                  hi[p][q] = fmaf(av[p], bv[q], hi[p][q]);
              }
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if constexpr (FP64) {
                sum[p][q] += (double)hi[p][q] + (double)lo[p][q];
              } else {
                const float y = hi[p][q] - cmp[p][q];
                const float tt = sum[p][q] + y;
                cmp[p][q] = (tt - sum[p][q]) - y;
                sum[p][q] = tt;
              }
            }
        }
      }
    }
    // the groups' sums, added in group order
    __syncthreads();
    if (act && ngrp > 1) {
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          gsum[((size_t)g * ntiles + t) * 16 + 4 * p + q] = FP64 ? sum[p][q] : sum[p][q] - cmp[p][q];
    }
    __syncthreads();
    if (act && g == 0) {
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          T v = FP64 ? sum[p][q] : sum[p][q] - cmp[p][q];
          for (int h = 1; h < ngrp; ++h) v += gsum[((size_t)h * ntiles + t) * 16 + 4 * p + q];
          const int i = 4 * ti + p, j = 4 * tj + q;
          if (i < k && j < k) {
            out[i * k + j] = v;
            out[j * k + i] = v;
          }
        }
    }
  }
}

// k_gram8: the FP32 Gram of a factor with contiguous rows (ldx == k, k <= 64,
// 16-byte aligned), with 8 x 8 register tiles.  A block (one per SM) walks
// its rows in stages of kG8Rows: each stage is one contiguous span of the
// factor, copied with 16-byte loads at the span's own offsets into shared
// memory (no index arithmetic) while the previous stage is consumed.
// Thread (g, t): tile t = (ti, tj), ti <= tj, of the upper triangle in 8 x 8
// blocks (28 tiles at k = 50, 36 at 64), row group g of ngrp = 256 / tiles
// (rows g, g + ngrp, ... of each stage).  Each row costs a thread 16 values
// (float2 loads for even k) and 64 FFMAs, against 8 values and 16 FFMAs per
// row in k_gram_part's 4 x 4 tiles.  As there, slabs are summed in fresh
// registers and folded into Kahan-compensated running sums (~64 rows a
// slab; the sums in registers, the corrections in shared memory), and the
// groups' sums are added in group order, so the result does not depend on
// scheduling.
constexpr int kG8Threads = 256, kG8Rows = 128, kG8MaxK = 64;
constexpr int kG8Buf = kG8Rows * kG8MaxK + 8;  // floats per stage buffer (+ tail pad)
constexpr int kG8Ldc = 68;                     // floats per thread row of corrections
constexpr int kG8Pre = kG8Rows * kG8MaxK / 4 / kG8Threads;  // float4 prefetch per thread
constexpr size_t kG8Smem = sizeof(float) * (2 * (size_t)kG8Buf + (size_t)kG8Threads * kG8Ldc);

template <bool EVEN>
__global__ void __launch_bounds__(kG8Threads, 1)
    k_gram8(const float *__restrict__ X, int64_t rows, int k, int64_t chunk,
            float *__restrict__ partials) {
  extern __shared__ __align__(16) float sg[];
  float *buf0 = sg, *buf1 = sg + kG8Buf;
  float *corr = sg + 2 * kG8Buf;
  const int tid = threadIdx.x;
  const int nt = (k + 7) >> 3, ntiles = nt * (nt + 1) / 2;
  const int ngrp = kG8Threads / ntiles;
  const int g = tid / ntiles, t = tid - g * ntiles;
  const bool act = g < ngrp;
  int ti = 0, tj = 0;
  if (act) {
    int rem = t;
    while (rem >= nt - ti) { rem -= nt - ti; ++ti; }
    tj = ti + rem;
  }
  // stages per slab: ~64 of the thread's own rows between folds
  const int fold_every = max(1, (64 * ngrp + kG8Rows / 2) / kG8Rows);
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  float *kc = corr + (size_t)tid * kG8Ldc;
#pragma unroll
  for (int e = 0; e < 64; e += 4) *reinterpret_cast<float4 *>(kc + e) = make_float4(0.f, 0.f, 0.f, 0.f);
  float acc[8][8], hi[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = hi[i][j] = 0.f;

  // stage c0: the span X[c0 k, (c0 + nr) k), float4 groups then <= 3 floats
  float4 pre[kG8Pre];
  float tailv = 0.f;
  auto fetch = [&](int64_t c0) {
    const int nr = (int)min((int64_t)kG8Rows, r1 - c0);
    const int len = nr * k, n4 = len >> 2;
    const float4 *src = reinterpret_cast<const float4 *>(X + c0 * k);
#pragma unroll
    for (int q = 0; q < kG8Pre; ++q) {
      const int i4 = tid + q * kG8Threads;
      pre[q] = i4 < n4 ? __ldcs(src + i4) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    tailv = tid < (len & 3) ? X[c0 * k + (n4 << 2) + tid] : 0.f;
  };
  auto store = [&](float *b, int64_t c0) {
    const int nr = (int)min((int64_t)kG8Rows, r1 - c0);
    const int len = nr * k, n4 = len >> 2;
#pragma unroll
    for (int q = 0; q < kG8Pre; ++q) {
      const int i4 = tid + q * kG8Threads;
      if (i4 < n4) *reinterpret_cast<float4 *>(b + 4 * i4) = pre[q];
    }
    if (tid < (len & 3)) b[(n4 << 2) + tid] = tailv;
  };
  auto fold = [&]() {
#pragma unroll
    for (int e4 = 0; e4 < 64; e4 += 4) {
      float4 cv = *reinterpret_cast<const float4 *>(kc + e4);
      float *c = &cv.x;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e4 + u, i = e >> 3, j = e & 7;
        const float y = acc[i][j] - c[u];
        const float tt = hi[i][j] + y;
        c[u] = (tt - hi[i][j]) - y;
        hi[i][j] = tt;
        acc[i][j] = 0.f;
      }
      *reinterpret_cast<float4 *>(kc + e4) = cv;
    }
  };
  auto load8 = [&](const float *p, float (&v)[8]) {
    if constexpr (EVEN) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2 w = *reinterpret_cast<const float2 *>(p + 2 * u);
        v[2 * u] = w.x;
        v[2 * u + 1] = w.y;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = p[u];
    }
  };

  if (r0 < r1) {
    fetch(r0);
    store(buf0, r0);
  }
  __syncthreads();
  int stage = 0;
  float *cur = buf0, *nxt = buf1;
  for (int64_t c0 = r0; c0 < r1; c0 += kG8Rows, ++stage) {
    const int nr = (int)min((int64_t)kG8Rows, r1 - c0);
    const bool more = c0 + kG8Rows < r1;
    if (more) fetch(c0 + kG8Rows);
    if (act) {
      for (int rr = g; rr < nr; rr += ngrp) {
        const float *row = cur + rr * k;
        float a[8], b[8];
        load8(row + 8 * ti, a);
        load8(row + 8 * tj, b);
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
          for (int i = 0; i < 8; ++i) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      if ((stage + 1) % fold_every == 0 || !more) fold();
    }
    if (more) store(nxt, c0 + kG8Rows);
    __syncthreads();
    float *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  // the groups' sums (hi - c), added in group order by group 0
  float *gs = sg;  // ngrp x ntiles x 64 floats, over the stage buffers
  __syncthreads();
  if (act && g > 0) {
#pragma unroll
    for (int e = 0; e < 64; ++e) gs[((size_t)g * ntiles + t) * 64 + e] = hi[e >> 3][e & 7] - kc[e];
  }
  __syncthreads();
  if (act && g == 0) {
    float *out = partials + (int64_t)blockIdx.x * k * k;
#pragma unroll
    for (int e = 0; e < 64; ++e) {
      float v = hi[e >> 3][e & 7] - kc[e];
      for (int h = 1; h < ngrp; ++h) v += gs[((size_t)h * ntiles + t) * 64 + e];
      const int i = 8 * ti + (e >> 3), j = 8 * tj + (e & 7);
      if (i < k && j < k) {
        out[i * k + j] = v;
        out[j * k + i] = v;
      }
    }
  }
}

template <bool FP64>
size_t gram_smem_bytes(int k) {
  const int kp = (k + 3) & ~3, nt = kp / 4, ntiles = nt * (nt + 1) / 2;
  const int ngrp = ntiles >= kGramThreads ? 1 : kGramThreads / ntiles;
  const size_t slab = (size_t)((kGramRows * kp + 3) & ~3) * sizeof(float);
  const size_t grp = ngrp > 1 ? (size_t)ngrp * ntiles * 16 * (FP64 ? sizeof(double) : sizeof(float)) : 0;
  return slab + grp;
}

__global__ void __launch_bounds__(256)
    k_gram_reduce_d(const double *__restrict__ partials, int nb, int k, double *__restrict__ G64,
                    float *__restrict__ G32) {
  __shared__ double sw[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int kk = k * k;
  const int e = blockIdx.x * 32 + lane;
  const int per = (nb + 7) / 8;
  const int b0 = w * per, b1 = min(nb, b0 + per);
  // four independent chains (loads in flight, FP64 latency overlapped),
  // combined in a fixed order
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  if (e < kk) {
    int b = b0;
    for (; b + 4 <= b1; b += 4) {
      a0 += partials[(int64_t)b * kk + e];
      a1 += partials[(int64_t)(b + 1) * kk + e];
      a2 += partials[(int64_t)(b + 2) * kk + e];
      a3 += partials[(int64_t)(b + 3) * kk + e];
    }
    for (; b < b1; ++b) a0 += partials[(int64_t)b * kk + e];
  }
  sw[w][lane] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  if (w == 0 && e < kk) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += sw[q][lane];
    G64[e] = s;
    if (G32) G32[e] = (float)s;
  }
}

__global__ void k_widen(const float *__restrict__ G32, int kk, double *__restrict__ G64) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kk; e += gridDim.x * blockDim.x)
    G64[e] = (double)G32[e];
}

// G_e = sum_b partials[b]_e in FP64: 32 entries per block; warp w sums the
// w-th eighth of the blocks in four interleaved chains (b ascending within
// each), and the chains and then the eight warp sums are added in a fixed
// order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(256)
    k_gram_reduce(const float *__restrict__ partials, int nb, int k, float *__restrict__ G) {
  __shared__ double sw[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int kk = k * k;
  const int e = blockIdx.x * 32 + lane;
  const int per = (nb + 7) / 8;
  const int b0 = w * per, b1 = min(nb, b0 + per);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  if (e < kk) {
    int b = b0;
    for (; b + 4 <= b1; b += 4) {
      a0 += (double)partials[(int64_t)b * kk + e];
      a1 += (double)partials[(int64_t)(b + 1) * kk + e];
      a2 += (double)partials[(int64_t)(b + 2) * kk + e];
      a3 += (double)partials[(int64_t)(b + 3) * kk + e];
    }
    for (; b < b1; ++b) a0 += (double)partials[(int64_t)b * kk + e];
  }
  sw[w][lane] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  if (w == 0 && e < kk) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += sw[i][lane];
    G[e] = (float)t;
  }
}
}  // namespace

int gram_partial_blocks(int64_t rows, int max_blocks) {
  int64_t nb = (rows + 127) / 128;  // at least 128 rows per block
  if (nb > max_blocks) nb = max_blocks;
  if (nb < 1) nb = 1;
  return (int)nb;
}

namespace {
bool gram_via_gemm(const float *X, int64_t rows, int k, float *G, float *partials, int max_blocks,
                   int *err, cudaStream_t s, cudaError_t *status);
}  // namespace

cudaError_t launch_gram(const float *X, int64_t rows, int k, int64_t ldx, float *G,
                        float *partials, int max_blocks, cudaStream_t s, int *err) {
  // wide ranks: the TMA-fed FP32 product kernel on X^T X (below)
  if (ldx == k && err) {
    cudaError_t st = cudaSuccess;
    if (gram_via_gemm(X, rows, k, G, partials, max_blocks, err, s, &st)) return st;
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 148;
  // k_gram8 needs >= 16 stages per block to repay its fixed costs: on the
  // sparse workload's 10^6 / 5 10^5 rows it takes the Grams from 0.320 to
  // 0.242 ms per iteration; on the dense one's 96,000 / 64,000 rows it was
  // slower (0.109 against 0.077 ms), so those keep k_gram_part
  if (ldx == k && k <= kG8MaxK && k >= 8 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
      rows >= 16LL * kG8Rows * sms) {
    // one block per SM (its chunk a whole number of stages, so every span
    // starts on a 16-byte boundary), partials reduced as for k_gram_part
    int64_t nb = (rows + kG8Rows - 1) / kG8Rows;
    const int64_t cap = min((int64_t)max_blocks, (int64_t)sms);
    if (nb > cap) nb = cap;
    const int64_t chunk = ((rows + nb - 1) / nb + kG8Rows - 1) / kG8Rows * kG8Rows;
    nb = (rows + chunk - 1) / chunk;
    auto kern = (k & 1) ? k_gram8<false> : k_gram8<true>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kG8Smem);
    kern<<<(unsigned)nb, kG8Threads, kG8Smem, s>>>(X, rows, k, chunk, partials);
    k_gram_reduce<<<(k * k + 31) / 32, 256, 0, s>>>(partials, (int)nb, k, G);
    g_launches += 2;
    return cudaGetLastError();
  }
  const int nb = gram_partial_blocks(rows, max_blocks);
  const int64_t chunk = (rows + nb - 1) / nb;
  const size_t smem = gram_smem_bytes<false>(k);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_gram_part<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_gram_part<false><<<nb, kGramThreads, smem, s>>>(X, rows, k, ldx, chunk, partials);
  k_gram_reduce<<<(k * k + 31) / 32, 256, 0, s>>>(partials, nb, k, G);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_gram_d(const float *X, int64_t rows, int k, int64_t ldx, double *G64,
                          float *G32, double *partials, int max_blocks, cudaStream_t s) {
  const int nb = gram_partial_blocks(rows, max_blocks);
  const int64_t chunk = (rows + nb - 1) / nb;
  const size_t smem = gram_smem_bytes<true>(k);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_gram_part<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_gram_part<true><<<nb, kGramThreads, smem, s>>>(X, rows, k, ldx, chunk, partials);
  k_gram_reduce_d<<<(k * k + 31) / 32, 256, 0, s>>>(partials, nb, k, G64, G32);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_widen(const float *G32, int k, double *G64, cudaStream_t s) {
  k_widen<<<(k * k + 255) / 256, 256, 0, s>>>(G32, k * k, G64);
  g_launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ SIMT GEMM
// C (M x N, ld ldc) = Aop (M x K) * B (K x N, ld ldb), FP32 FMA.
//   AK = true : Aop(mm, kk) = A[mm * lda + kk]   (A H^T: A is K-contiguous)
//   AK = false: Aop(mm, kk) = A[kk * lda + mm]   (W^T A as (A^T W): M-contiguous)
// 256 threads as 16 x 16; thread (ty, tx) owns rows ty*TM .. ty*TM+TM-1 and
// columns tx*TN .. tx*TN+TN-1 of the block tile.  (A layout of 8 threads
// along N with BN = 56 at k = 50, which wastes fewer FMAs on padding columns,
// measured 11 % slower even with its shared-memory reads free of bank
// conflicts: 20.4 against 18.3 ms per product at 96000 x 64000.)  The next K-slab is
// prefetched into registers while the current one is consumed from shared
// memory.  Accumulation is compensated: each 32-long K-slab is summed in a
// fresh FP32 register and added to the running sum with Kahan's correction,
// so the error does not grow with K (the residual expansion of Sec. 6.2
// subtracts nearly equal terms and needs the products close to FP32
// rounding).
namespace {
// two resident blocks per SM (at most 128 registers a thread): measured 8-12 %
// faster than one at 96000 x 64000, k = 50, despite a few spilled registers
#ifndef AUNMF_SIMT_MINB
#define AUNMF_SIMT_MINB 2
#endif
#ifndef AUNMF_SIMT_BM
#define AUNMF_SIMT_BM 128
#endif
template <int BM, int BN, int BK, bool AK>
__global__ void __launch_bounds__(256, AUNMF_SIMT_MINB)
    k_gemm_simt(const float *__restrict__ A, int64_t lda, int64_t M, int64_t K,
                const float *__restrict__ B, int ldb, int N, float *__restrict__ C, int ldc,
                int64_t kchunk, int vec) {
  // blockIdx.z: K split [kz0, kz1) (kchunk a multiple of the slab); its
  // partial C goes to C + z * M * ldc.  vec: A is 16-byte aligned with lda % 4
  // == 0, so its tile is read as float4 groups along A's contiguous axis.
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int GA = BM * BK / 4 / 256;  // float4 groups of the A tile per thread
  constexpr int LA = BM * BK / 256, LB = BK * BN / 256;
  constexpr int PADA = 4;  // row pad: spreads the transposed stores over banks
  constexpr int SLAB = 128;  // K elements per compensated partial
  constexpr int LDK = TM * TN + 1;  // odd row stride of the per-thread running sums
  static_assert(GA >= 1 && GA * 4 == LA && LB >= 1 && TM % 4 == 0, "tile too small");
  static_assert(SLAB % BK == 0, "slab must be a multiple of BK");
  __shared__ __align__(16) float sA[2][BK][BM + PADA];
  __shared__ __align__(16) float sB[2][BK][BN];
  // Kahan running sum and correction of each thread's TM x TN outputs, in a
  // row of its own (touched once per slab): keeping them in registers would
  // triple the accumulator registers and halve the resident warps
  extern __shared__ float sKahan[];
  float *kh = sKahan + (size_t)threadIdx.x * LDK * 2, *kc = kh + LDK;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int64_t kz0 = (int64_t)blockIdx.z * kchunk, kz1 = min(K, kz0 + kchunk);

  // Per-thread tile coordinates, pointers and edge predicates, fixed for the
  // whole K range (the loads of a full K step do no index arithmetic).
  //   AK:  group q is row am[q] of the tile, K offsets ak[q] .. ak[q] + 3
  //   !AK: group q is K offset ak[q], rows am[q] .. am[q] + 3
  // va: 1 all four elements inside A, 2 some (M edge, !AK), 0 none.
  int am[GA], ak[GA], va[GA];
  const float *pa[GA];
#pragma unroll
  for (int q = 0; q < GA; ++q) {
    const int f = tid + 256 * q;
    if (AK) {
      am[q] = f / (BK / 4);
      ak[q] = 4 * (f % (BK / 4));
      va[q] = m0 + am[q] < M ? 1 : 0;
      pa[q] = A + (va[q] ? (m0 + am[q]) : 0) * lda + kz0 + ak[q];
    } else {
      ak[q] = f / (BM / 4);
      am[q] = 4 * (f % (BM / 4));
      va[q] = m0 + am[q] + 3 < M ? 1 : (m0 + am[q] < M ? 2 : 0);
      pa[q] = A + (kz0 + ak[q]) * lda + (va[q] ? m0 + am[q] : 0);
    }
  }
  int bk[LB], bn[LB];
  bool vb[LB];
  const float *pb[LB];
#pragma unroll
  for (int q = 0; q < LB; ++q) {
    const int idx = tid + 256 * q;
    bn[q] = idx % BN;
    bk[q] = idx / BN;
    vb[q] = n0 + bn[q] < N;
    pb[q] = B + (kz0 + bk[q]) * ldb + (vb[q] ? n0 + bn[q] : 0);
  }

  float4 ra[GA];
  float rb[LB];
  // K step [k0, k0 + BK): a full step inside [kz0, kz1) with vec takes the
  // pointers as they stand; the last, partial step (and !vec) checks each
  // element's K index as well.
  auto load = [&](int64_t k0, bool full) {
#pragma unroll
    for (int q = 0; q < GA; ++q) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (full && vec && va[q] == 1) {
        v = __ldg(reinterpret_cast<const float4 *>(pa[q]));
      } else if (va[q]) {
        float e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t gm = m0 + am[q] + (AK ? 0 : u), gk = k0 + ak[q] + (AK ? u : 0);
          e[u] = (gm < M && gk < kz1) ? __ldg(&A[AK ? gm * lda + gk : gk * lda + gm]) : 0.f;
        }
        v = make_float4(e[0], e[1], e[2], e[3]);
      }
      ra[q] = v;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q)
      rb[q] = (vb[q] && (full || k0 + bk[q] < kz1)) ? __ldg(pb[q]) : 0.f;
  };
  auto advance = [&]() {
#pragma unroll
    for (int q = 0; q < GA; ++q) pa[q] += AK ? (int64_t)BK : (int64_t)BK * lda;
#pragma unroll
    for (int q = 0; q < LB; ++q) pb[q] += (int64_t)BK * ldb;
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < GA; ++q) {
      if (AK) {
        sA[buf][ak[q] + 0][am[q]] = ra[q].x;
        sA[buf][ak[q] + 1][am[q]] = ra[q].y;
        sA[buf][ak[q] + 2][am[q]] = ra[q].z;
        sA[buf][ak[q] + 3][am[q]] = ra[q].w;
      } else {
        *reinterpret_cast<float4 *>(&sA[buf][ak[q]][am[q]]) = ra[q];
      }
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) sB[buf][bk[q]][bn[q]] = rb[q];
  };

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  for (int e = 0; e < TM * TN; ++e) kh[e] = kc[e] = 0.f;
  auto fold = [&]() {  // hi += acc with Kahan's compensation; acc = 0
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int e = i * TN + j;
        const float hi = kh[e], cor = kc[e];
        const float y = acc[i][j] - cor;
        const float t = hi + y;
        kc[e] = (t - hi) - y;
        kh[e] = t;
        acc[i][j] = 0.f;
      }
  };

  C += (int64_t)blockIdx.z * M * ldc;
  load(kz0, kz0 + BK <= kz1);
  advance();
  store(0);
  __syncthreads();
  int buf = 0, slab_left = SLAB / BK;
  for (int64_t k0 = kz0; k0 < kz1; k0 += BK) {
    const bool more = k0 + BK < kz1;
    if (more) {
      load(k0 + BK, k0 + 2 * BK <= kz1);
      advance();
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; i += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(&sA[buf][kk][ty * TM + i]);
        a[i] = v.x; a[i + 1] = v.y; a[i + 2] = v.z; a[i + 3] = v.w;
      }
      if constexpr (TN == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(&sB[buf][kk][tx * TN]);
        b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
      } else if constexpr (TN == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(&sB[buf][kk][tx * TN]);
        b[0] = v.x; b[1] = v.y;
      } else {
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = sB[buf][kk][tx * TN + j];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    // fold once per slab of K (kz0 is a multiple of the slab) and at the end
    if (--slab_left == 0 || !more) {
      fold();
      slab_left = SLAB / BK;
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gm = m0 + ty * TM + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx * TN + j;
      if (gn < N) C[gm * ldc + gn] = kh[i * TN + j] - kc[i * TN + j];
    }
  }
}

// ---------------------------------------------------------------- TMA-fed form
// k_gemm_simt_tma: the same product and the same compensated summation as
// k_gemm_simt, for N > 32 (column tiles of 64) when A's rows are 16-byte
// aligned.  A's tiles and the fixed factor's 16 x 64 tiles arrive by TMA in
// a seven-stage shared-memory ring with mbarriers (full: one arrival + the
// copies' bytes; empty: all 256 threads).  The factor is read from a copy
// whose rows are padded to a multiple of 4 floats (TMA needs 16-byte row
// strides; N = 50 floats is not one); staging its tiles with 4-byte
// asynchronous copies instead measured 3x slower than the whole product
// should take (11.5 ms for the copies alone at 96,000 x 64,000).  Eight warps compute, 8 x 8 outputs per thread (256 x 64 per
// block, one block per SM), four 16-byte fragment loads per 64 FFMAs, with
// the running sums in registers (two warps per SM sub-partition may hold
// up to 255 registers each; a ninth, producer-only warp would cap them at
// 168).  Thread 0 also fills the ring: steps 0 .. 6 first, then at the top
// of step s it waits until every thread has released the stage read at
// step s - 1 (warp 0 trails the others, so the wait is short) and issues
// the two copies of step s + 6 into it.
//   Thread (ty, tx), ty = 0..31, tx = 0..7 (a warp: 4 ty x 8 tx): columns
//   tx*4 + {0..3} and 32 + tx*4 + {0..3}; rows ty + 32 i (AK) or
//   ty*4 + {0..3} and 128 + ty*4 + {0..3} (!AK).
// AK (A K-contiguous): the tile is 256 rows of 16 K (64 bytes), copied with
// the 64-byte swizzle (16-byte chunk c of row r lands at chunk
// c ^ ((r >> 1) & 3)), so the four rows a warp reads at once (ty .. ty+3)
// sit in four different bank groups.  !AK: 16 K-rows of 256 (one kilobyte):
// a warp's four row fragments are consecutive.  Either way a warp's 16-byte
// loads of the factor tile read 8 consecutive chunks, with no bank conflict.
// Slab sums are folded every 128 K into the running sums with Kahan's
// corrections, which sit in shared memory (one row per thread).  Every wait
// is bounded; on expiry the kernel raises *err, writes nothing and returns
// (thread 0 first waits, bounded, for the copies it has in flight).  The K
// steps of a split are whole (its length is a multiple of 128); rows and
// columns past either matrix are zero-filled by the copies.
constexpr int kTBM = 256, kTBN = 64, kTBK = 16, kTStages = 7;
constexpr int kTThreads = 256;
constexpr int kTSlabSteps = 8;  // K steps per compensated slab (128 K, as k_gemm_simt)
constexpr int kTLdc = 68;       // floats per thread row of corrections (64 + pad)
constexpr size_t kTStageA = (size_t)kTBM * kTBK * 4, kTStageB = (size_t)kTBK * kTBN * 4;
constexpr size_t kTSmem = 1024 + kTStages * (kTStageA + kTStageB) +
                          (size_t)kTThreads * kTLdc * 4 + 2 * kTStages * 8;

template <bool AK>
__global__ void __launch_bounds__(kTThreads, 1)
    k_gemm_simt_tma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                    int64_t M, int64_t K, int N, float *__restrict__ C, int ldc, int64_t kchunk,
                    int *err, long long limit, int inject) {
  // inject (test hook): thread 0 never arrives on the first stage's barrier,
  // so every thread's bounded wait runs out
  using namespace aunmf::ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  float *sA = reinterpret_cast<float *>(smem);
  float *sB = reinterpret_cast<float *>(smem + kTStages * kTStageA);
  float *corr = reinterpret_cast<float *>(smem + kTStages * (kTStageA + kTStageB));
  uint64_t *full = reinterpret_cast<uint64_t *>(corr + kTThreads * kTLdc);
  uint64_t *empty = full + kTStages;
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.x * kTBM;
  const int n0 = blockIdx.y * kTBN;
  const int64_t kz0 = (int64_t)blockIdx.z * kchunk, kz1 = min(K, kz0 + kchunk);
  const int nsteps = kz1 > kz0 ? (int)((kz1 - kz0 + kTBK - 1) / kTBK) : 0;
  const bool producer = tid < 32;
  if (tid == 0) {
    for (int st = 0; st < kTStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kTThreads);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // thread 0: fill stage st with step s
  const uint64_t pol_a = policy_evict_first(), pol_b = policy_evict_last();  // A streams once
  int issued = 0;
  auto fill = [&](int s) {
    const int st = s % kTStages;
    const int k0 = (int)(kz0 + (int64_t)s * kTBK);
    const uint32_t bytes = (uint32_t)(kTStageA + kTStageB);
    if (inject && s == 0)
      mbar_expect_tx_only(&full[st], bytes);
    else
      mbar_expect_tx(&full[st], bytes);
    // x coordinates (k0 for AK and the factor, m0 otherwise) are multiples
    // of 16 floats; the checked build tests it and skips bad copies
    if (!AUNMF_BOUND(k0 >= 0 && (k0 & 3) == 0 && (m0 & 3) == 0 && (n0 & 3) == 0,
                     AUNMF_CHECK_TMA_COORD))
      return;
    if (AK)
      tma_load_2d(sA + (size_t)st * kTBM * kTBK, &mapA, &full[st], k0, (int)m0, pol_a);
    else
      tma_load_2d(sA + (size_t)st * kTBM * kTBK, &mapA, &full[st], (int)m0, k0, pol_a);
    tma_load_2d(sB + (size_t)st * kTBK * kTBN, &mapB, &full[st], n0, k0, pol_b);
    ++issued;
  };
  if (tid == 0)  // every stage starts empty: steps 0 .. kTStages - 1
    for (int s = 0; s < kTStages && s < nsteps; ++s) fill(s);

  const int w = tid >> 5, l = tid & 31, tx = l & 7, ty = w * 4 + (l >> 3);
  float *kc = corr + (size_t)tid * kTLdc;  // Kahan corrections of the 64 sums
#pragma unroll
  for (int e = 0; e < 64; e += 4) *reinterpret_cast<float4 *>(kc + e) = make_float4(0.f, 0.f, 0.f, 0.f);
  float acc[8][8], hi[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = hi[i][j] = 0.f;
  auto fold = [&]() {  // hi += acc with Kahan's compensation; acc = 0
#pragma unroll
    for (int e4 = 0; e4 < 64; e4 += 4) {
      float4 cv = *reinterpret_cast<const float4 *>(kc + e4);
      float *c = &cv.x;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e4 + u, i = e >> 3, j = e & 7;
        const float y = acc[i][j] - c[u];
        const float t = hi[i][j] + y;
        c[u] = (t - hi[i][j]) - y;
        hi[i][j] = t;
        acc[i][j] = 0.f;
      }
      *reinterpret_cast<float4 *>(kc + e4) = cv;
    }
  };
  // column-major issue order (each b[j] for 8 FFMAs in a row): 2-3 % faster
  // than row-major at 96000 x 64000 (fewer operand dispatch stalls)
  auto fma8x8 = [&](const float (&a)[8], const float4 b0, const float4 b1) {
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  };
  // AK: rows ty + 32 i share their swizzle (r >> 1) & 3 (32 i leaves those bits alone)
  const int sw = (ty >> 1) & 3;

  bool ok = true;
  int slab = 0;
  for (int s = 0; s < nsteps; ++s) {
    const int st = s % kTStages;
    if (producer && s >= 1 && s - 1 + kTStages < nsteps) {
      // refill the stage read at step s - 1 (use (s - 1) / kTStages of it)
      const int sp = s - 1;
      int okp = 1;
      if (tid == 0)
        okp = mbar_wait(&empty[sp % kTStages], (uint32_t)(sp / kTStages) & 1u, err, limit) ? 1 : 0;
      if (!__shfl_sync(0xffffffffu, okp, 0)) {
        ok = false;
        break;
      }
      if (tid == 0) fill(sp + kTStages);
    }
    if (!mbar_wait(&full[st], (uint32_t)(s / kTStages) & 1u, err, limit)) {
      ok = false;
      break;
    }
    const float *a = sA + (size_t)st * kTBM * kTBK;
    const float *b = sB + (size_t)st * kTBK * kTBN + tx * 4;
    if (AK) {  // a: [256 rows][16 K], 64-byte swizzle
#pragma unroll
      for (int kq = 0; kq < kTBK / 4; ++kq) {
        float4 av[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
          av[i] = *reinterpret_cast<const float4 *>(a + (ty + 32 * i) * kTBK + ((kq ^ sw) << 2));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float *br = b + (kq * 4 + u) * kTBN;
          const float4 b0 = *reinterpret_cast<const float4 *>(br);
          const float4 b1 = *reinterpret_cast<const float4 *>(br + 32);
          float af[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) af[i] = (&av[i].x)[u];
          fma8x8(af, b0, b1);
        }
      }
    } else {  // a: [16 K][256 rows]
#pragma unroll
      for (int kk = 0; kk < kTBK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4 *>(a + kk * kTBM + ty * 4);
        const float4 a1 = *reinterpret_cast<const float4 *>(a + kk * kTBM + 128 + ty * 4);
        const float *br = b + kk * kTBN;
        const float4 b0 = *reinterpret_cast<const float4 *>(br);
        const float4 b1 = *reinterpret_cast<const float4 *>(br + 32);
        const float af[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        fma8x8(af, b0, b1);
      }
    }
    mbar_arrive(&empty[st]);
    if (++slab == kTSlabSteps || s + 1 == nsteps) {
      fold();
      slab = 0;
    }
  }
  if (tid == 0) {
    // the copies thread 0 has put in flight land before the block exits
    for (int st = 0; st < kTStages && st < issued; ++st) {
      const int cnt = (issued - st + kTStages - 1) / kTStages;
      mbar_wait_drain(&full[st], (uint32_t)(cnt - 1) & 1u, limit);
    }
  }
  if (!ok) return;
  C += (int64_t)blockIdx.z * M * ldc;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gm = m0 + (AK ? ty + 32 * i : (i < 4 ? ty * 4 + i : 128 + ty * 4 + i - 4));
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gn = n0 + (j < 4 ? tx * 4 + j : 32 + tx * 4 + j - 4);
      if (gn < N) C[gm * ldc + gn] = hi[i][j] - kc[i * 8 + j];
    }
  }
}

// Tensor map of A's tiles for k_gemm_simt_tma: AK, a box of 16 K x 256 rows
// over A (M x K, ld lda), 64-byte swizzle; !AK, 256 rows x 16 K over A
// stored K x M, no swizzle.  FP32, zero fill outside the matrix.
// Tensor map of the factor's tiles: 64 columns x 16 K rows over the padded
// copy (K x N, ld ldp), no swizzle, zero fill past N and K.
bool simt_factor_map(CUtensorMap *map, const float *Bp, int64_t K, int N, int ldp) {
  ptx::EncodeTiledFn fn = ptx::encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)K};
  cuuint64_t strides[1] = {(cuuint64_t)ldp * 4};
  cuuint32_t box[2] = {(cuuint32_t)kTBN, (cuuint32_t)kTBK};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(Bp), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool simt_map(CUtensorMap *map, const float *A, int64_t lda, int64_t M, int64_t K, bool AK) {
  ptx::EncodeTiledFn fn = ptx::encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)(AK ? K : M), (cuuint64_t)(AK ? M : K)};
  cuuint64_t strides[1] = {(cuuint64_t)(lda * 4)};
  cuuint32_t box[2] = {(cuuint32_t)(AK ? kTBK : kTBM), (cuuint32_t)(AK ? kTBM : kTBK)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(A), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            AK ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BM, int BN>
constexpr size_t simt_kahan_bytes() {
  return sizeof(float) * 256 * 2 * ((BM / 16) * (BN / 16) + 1);
}

// K splits: the smallest S in 1..4 whose block count fills the resident
// slots (`per_sm` blocks per SM) most evenly, each split at least 8 slabs long.
int simt_splits(int64_t tiles, int64_t K, int per_sm) {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t slots = (int64_t)per_sm * (sms > 0 ? sms : 148);
  int best = 1;
  double best_eff = 0.0;
  for (int S = 1; S <= 4; ++S) {
    if (S > 1 && K / S < 8 * 128) break;
    const int64_t u = tiles * S;
    const double eff = ((double)u / slots) / (double)((u + slots - 1) / slots);
    if (eff > best_eff + 0.02) { best_eff = eff; best = S; }
  }
  return best;
}

__global__ void k_sum_parts(const float *__restrict__ parts, int S, int64_t len,
                            float *__restrict__ C) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += parts[z * len + e];
    C[e] = s;
  }
}

template <bool AK>
cudaError_t gemm_simt(const float *A, int64_t lda, int64_t M, int64_t K, const float *B, int N,
                      float *C, float *parts, int *err, cudaStream_t s) {
  constexpr int BM = AUNMF_SIMT_BM, BK = 16, SLAB = 128;
  const int vec = (reinterpret_cast<uintptr_t>(A) % 16 == 0 && lda % 4 == 0) ? 1 : 0;
  // TMA-fed form: N > 32, 16-byte aligned rows, coordinates within int32
  // (parts holds the split partials, then the factor's padded copy)
  CUtensorMap mapA, mapB;
  const int ldp = (N + 3) & ~3;
  float *Bp = parts ? parts + ((4 * M * (int64_t)N + 63) & ~63LL) : nullptr;
  if (N > 32 && vec && err && parts && M < (1LL << 31) && K < (1LL << 31) &&
      simt_map(&mapA, A, lda, M, K, AK) && simt_factor_map(&mapB, Bp, K, N, ldp)) {
    const unsigned gx = (unsigned)((M + kTBM - 1) / kTBM), gy = (unsigned)((N + kTBN - 1) / kTBN);
    const int S = simt_splits((int64_t)gx * gy, K, 1);
    const int64_t kchunk = ((K + S - 1) / S + SLAB - 1) / SLAB * SLAB;
    cudaError_t e = launch_copy2d(B, N, Bp, ldp, K, N, s);
    if (e != cudaSuccess) return e;
    auto kern = k_gemm_simt_tma<AK>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTSmem);
    kern<<<dim3(gx, gy, (unsigned)S), kTThreads, kTSmem, s>>>(
        mapA, mapB, M, K, N, S > 1 ? parts : C, N, kchunk, err, fault::wait_cycles(),
        fault::site() == AUNMF_INJECT_SIMT_WAIT ? 1 : 0);
    g_launches += 1;
    if (S > 1) {
      const int64_t len = M * (int64_t)N;
      int64_t nb = (len + 255) / 256;
      if (nb > 152 * 16) nb = 152 * 16;
      k_sum_parts<<<(unsigned)nb, 256, 0, s>>>(parts, S, len, C);
      g_launches += 1;
    }
    return cudaGetLastError();
  }
  const unsigned gx = (unsigned)((M + BM - 1) / BM);
  const int BN = N <= 16 ? 16 : (N <= 32 ? 32 : 64);
  const unsigned gy = (unsigned)((N + BN - 1) / BN);
  const int S = parts ? simt_splits((int64_t)gx * gy, K, 2) : 1;
  const int64_t kchunk = ((K + S - 1) / S + SLAB - 1) / SLAB * SLAB;
  float *out = S > 1 ? parts : C;
  const dim3 grid(gx, gy, (unsigned)S);
  auto go = [&](auto kern, size_t sm) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<grid, 256, sm, s>>>(A, lda, M, K, B, N, N, out, N, kchunk, vec);
  };
  switch (BN) {
    case 16: go(k_gemm_simt<BM, 16, BK, AK>, simt_kahan_bytes<BM, 16>()); break;
    case 32: go(k_gemm_simt<BM, 32, BK, AK>, simt_kahan_bytes<BM, 32>()); break;
    default: go(k_gemm_simt<BM, 64, BK, AK>, simt_kahan_bytes<BM, 64>()); break;
  }
  g_launches += 1;
  if (S > 1) {
    const int64_t len = M * (int64_t)N;
    int64_t nb = (len + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    k_sum_parts<<<(unsigned)nb, 256, 0, s>>>(parts, S, len, C);
    g_launches += 1;
  }
  return cudaGetLastError();
}
// G = X^T X for X (rows x k, contiguous rows, k >= 96 and a multiple of 4,
// 16-byte aligned) with the TMA-fed FP32 product kernel: C (k x k) = Aop
// (k x rows) B (rows x k) with Aop(i, r) = X[r][i] (A stored K x M) and B =
// X.  The whole square is formed (twice the flops of the upper triangle), in
// Kahan-compensated slabs like every product, over S K splits chosen to fill
// the SMs, whose partials (S x k x k in `partials`) are added in FP64 in
// split order.  At k = 512 on 96,000 / 64,000 rows this replaces k_gram_part,
// whose 4 x 4 tiles need 8,256 tiles per row and so re-stage every row 33
// times.  Returns false (nothing launched) when the shape does not qualify.
bool gram_via_gemm(const float *X, int64_t rows, int k, float *G, float *partials, int max_blocks,
                   int *err, cudaStream_t s, cudaError_t *status) {
  if (k < 96 || (k & 3) || (reinterpret_cast<uintptr_t>(X) & 15) || rows < 1024 ||
      rows >= (1LL << 31))
    return false;
  CUtensorMap mapA, mapB;
  if (!simt_map(&mapA, X, k, k, rows, false) || !simt_factor_map(&mapB, X, rows, k, k)) return false;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 148;
  const unsigned gx = (unsigned)((k + kTBM - 1) / kTBM), gy = (unsigned)((k + kTBN - 1) / kTBN);
  int64_t S = (sms + (int64_t)gx * gy - 1) / ((int64_t)gx * gy);
  S = min(S, (int64_t)max_blocks);
  S = min(S, rows / 512);
  if (S < 1) S = 1;
  const int64_t kchunk = ((rows + S - 1) / S + 127) / 128 * 128;
  S = (rows + kchunk - 1) / kchunk;
  auto kern = k_gemm_simt_tma<false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTSmem);
  kern<<<dim3(gx, gy, (unsigned)S), kTThreads, kTSmem, s>>>(
      mapA, mapB, k, rows, k, partials, k, kchunk, err, fault::wait_cycles(),
      fault::site() == AUNMF_INJECT_SIMT_WAIT ? 1 : 0);
  k_gram_reduce<<<(k * k + 31) / 32, 256, 0, s>>>(partials, (int)S, k, G);
  g_launches += 2;
  *status = cudaGetLastError();
  return true;
}
}  // namespace

cudaError_t launch_aht_simt(const float *A, int64_t m, int64_t n, int64_t lda, const float *Ht,
                            int k, float *P, float *parts, int *err, cudaStream_t s) {
  return gemm_simt<true>(A, lda, m, n, Ht, k, P, parts, err, s);
}

cudaError_t launch_wta_simt(const float *A, int64_t m, int64_t n, int64_t lda, const float *W,
                            int k, float *P, float *parts, int *err, cudaStream_t s) {
  return gemm_simt<false>(A, lda, n, m, W, k, P, parts, err, s);
}

size_t simt_parts_bytes(int64_t rows, int k) {
  return sizeof(float) * (((4 * (size_t)rows * k + 63) & ~(size_t)63) + (size_t)rows * ((k + 3) & ~3));
}

// ------------------------------------------------------------------ transpose
namespace {
__global__ void k_transpose(const float *__restrict__ in, int64_t rows, int64_t cols,
                            float *__restrict__ out) {
  __shared__ float t[32][33];
  const int64_t tr = (rows + 31) / 32, tc = (cols + 31) / 32;
  for (int64_t tile = blockIdx.x; tile < tr * tc; tile += gridDim.x) {
    const int64_t r0 = (tile / tc) * 32, c0 = (tile % tc) * 32;
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      const int64_t r = r0 + y, c = c0 + threadIdx.x;
      if (r < rows && c < cols) t[y][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      const int64_t c = c0 + y, r = r0 + threadIdx.x;
      if (r < rows && c < cols) out[c * rows + r] = t[threadIdx.x][y];
    }
  }
}

__global__ void k_copy2d(const float *__restrict__ in, int64_t ld_in, float *__restrict__ out,
                         int64_t ld_out, int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    out[r * ld_out + c] = in[r * ld_in + c];
  }
}
}  // namespace

cudaError_t launch_transpose(const float *in, int64_t rows, int64_t cols, float *out,
                             cudaStream_t s) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  int64_t tiles = ((rows + 31) / 32) * ((cols + 31) / 32);
  if (tiles > 152 * 64) tiles = 152 * 64;
  k_transpose<<<(unsigned)tiles, dim3(32, 8), 0, s>>>(in, rows, cols, out);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_copy2d(const float *in, int64_t ld_in, float *out, int64_t ld_out,
                          int64_t rows, int64_t cols, cudaStream_t s) {
  if (rows * cols == 0) return cudaSuccess;
  int64_t nb = (rows * cols + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  k_copy2d<<<(unsigned)nb, 256, 0, s>>>(in, ld_in, out, ld_out, rows, cols);
  g_launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ reductions
namespace {
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide FP64 sum in a fixed tree order; result valid in thread 0.
__device__ double block_sum_d(double v) {
  __shared__ double sw[32];
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sw[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sw[lane] : 0.0;
    r = warp_sum_d(r);
  }
  return r;
}

// partials[b] = sum of squares over rows r = b, b + nb, ... of A (m x n, lda)
__global__ void k_norm2_partial(const float *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                                double *__restrict__ partials) {
  // squares of one row are summed in FP32 by each thread (<= n/256 terms),
  // then added in FP64: FP64 adds at every element would bound the pass by
  // the FP64 rate instead of HBM
  // With 16-byte aligned rows the row is read as float4 groups, four groups
  // in flight per thread (scalar loads left the pass at ~1/3 of HBM speed).
  double s = 0.0;
  const bool vec = (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (lda & 3) == 0;
  for (int64_t r = blockIdx.x; r < m; r += gridDim.x) {
    const float *row = A + r * lda;
    float sr = 0.f;
    int64_t c0 = 0;
    if (vec) {
      const float4 *row4 = reinterpret_cast<const float4 *>(row);
      const int64_t n4 = n >> 2;
      float s4[4] = {0.f, 0.f, 0.f, 0.f};
      int64_t g = threadIdx.x;
      for (; g + 3 * (int64_t)blockDim.x < n4; g += 4 * (int64_t)blockDim.x) {
        float4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = __ldcs(row4 + g + u * blockDim.x);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          s4[u] = fmaf(q[u].w, q[u].w, fmaf(q[u].z, q[u].z, fmaf(q[u].y, q[u].y, fmaf(q[u].x, q[u].x, s4[u]))));
      }
      for (; g < n4; g += blockDim.x) {
        const float4 q = __ldcs(row4 + g);
        s4[0] = fmaf(q.w, q.w, fmaf(q.z, q.z, fmaf(q.y, q.y, fmaf(q.x, q.x, s4[0]))));
      }
      sr = (s4[0] + s4[1]) + (s4[2] + s4[3]);
      c0 = n4 << 2;
    }
    for (int64_t c = c0 + threadIdx.x; c < n; c += blockDim.x) sr = fmaf(row[c], row[c], sr);
    s += (double)sr;
  }
  s = block_sum_d(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_norm2_vec_partial(const float *__restrict__ v, int64_t len,
                                    double *__restrict__ partials) {
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)v[e];
    s = fma(x, x, s);
  }
  s = block_sum_d(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out[0] = ||A||^2 from the partials; out[1] = 0: the products read A itself.
__global__ void k_sum_partials(const double *__restrict__ partials, int nparts,
                               double *__restrict__ out) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += partials[b];
  s = block_sum_d(s);
  if (threadIdx.x == 0) {
    out[0] = s;
    out[1] = 0.0;
  }
}

// <P, Q> partials.  With 16-byte aligned arrays, four products at a time are
// formed and summed in FP32 (round-to-nearest: unbiased, ~1e-7 relative per
// group, averaging out over the groups) and the group joins an FP64 sum; an
// FP64 FMA per element bound the pass by the FP64 rate (0.14 ms on the sparse
// workload's 2.5e7 entries, ~5x its memory time).
__global__ void k_dot_partial(const float *__restrict__ P, const float *__restrict__ Q,
                              int64_t len, double *__restrict__ partials) {
  double s = 0.0;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  int64_t tail = 0;
  if (((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(Q)) & 15) == 0) {
    const float4 *P4 = reinterpret_cast<const float4 *>(P), *Q4 = reinterpret_cast<const float4 *>(Q);
    const int64_t n4 = len >> 2;
    for (int64_t g = t0; g < n4; g += nt) {
      const float4 p = P4[g], q = Q4[g];
      s += (double)fmaf(p.w, q.w, fmaf(p.z, q.z, fmaf(p.y, q.y, p.x * q.x)));
    }
    tail = n4 << 2;
  }
  for (int64_t e = tail + t0; e < len; e += nt) s = fma((double)P[e], (double)Q[e], s);
  s = block_sum_d(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// relres = sqrt(max(0, ||A||^2 + d - 2 <P, Ht> + <GW, GH>) / ||A||^2), FP64
// (Sec. 5, relative error; trace form).  When P was formed from a rounded
// copy A~ of A (TF32 / BF16 products), <P, Ht> = <A~, W H> and
//   ||A - WH||^2 = ||A||^2 - 2 <A~, WH> + ||WH||^2 + 2 <A~ - A, WH>;
// the last term is taken as d = n2a[1] = 2 <A~ - A, A> (WH ~ A), which is
// off by 2 <A~ - A, A - WH>, a sum of rounding errors that do not correlate
// with the fit residual.  Without d, the mean of the rounding errors (not
// zero on real value distributions: -8e-6 relative for BF16 on uniform
// low-rank data) would bias the reported residual by ~1e-3 at relres ~1e-2.
// <GW, GH> in FP64 by one block: four interleaved chains per thread keep
// loads in flight (a single chain waited on L2 for every element: 0.58 ms at
// k = 512), combined in a fixed order.
__device__ double gram_dot_block(const float *__restrict__ GW, const float *__restrict__ GH,
                                 int kk) {
  double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
  const int step = blockDim.x;
  int e = threadIdx.x;
  for (; e + 3 * step < kk; e += 4 * step) {
    q0 = fma((double)GW[e], (double)GH[e], q0);
    q1 = fma((double)GW[e + step], (double)GH[e + step], q1);
    q2 = fma((double)GW[e + 2 * step], (double)GH[e + 2 * step], q2);
    q3 = fma((double)GW[e + 3 * step], (double)GH[e + 3 * step], q3);
  }
  for (; e < kk; e += step) q0 = fma((double)GW[e], (double)GH[e], q0);
  return block_sum_d((q0 + q1) + (q2 + q3));
}

__global__ void __launch_bounds__(1024) k_relres_final(const double *__restrict__ partials, int nparts,
                               const float *__restrict__ GW, const float *__restrict__ GH, int k,
                               const double *__restrict__ n2a, double *__restrict__ relres,
                               DevCounters *ctr, double *last) {
  double cross = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) cross += partials[b];
  cross = block_sum_d(cross);
  const double quad = gram_dot_block(GW, GH, k * k);
  if (threadIdx.x == 0) {
    const double a2 = n2a[0];
    double r2 = (a2 + n2a[1]) - 2.0 * cross + quad;
    if (r2 < 0.0) r2 = 0.0;
    const double rr = a2 > 0.0 ? sqrt(r2 / a2) : 0.0;
    if (!isfinite(rr)) ctr->nonfinite += 1;
    if (relres) relres[ctr->iter] = rr;
    ctr->iter += 1;
    if (last) *last = rr;
  }
}
// loss = 0.5 (||A||^2 + d - 2 <P, Ht> + <GW, GH>), FP64 (not clamped); d as
// for the residual.
__global__ void __launch_bounds__(1024) k_loss_final(const double *__restrict__ partials, int nparts,
                             const float *__restrict__ GW, const float *__restrict__ GH, int k,
                             const double *__restrict__ n2a, double *__restrict__ loss) {
  double cross = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) cross += partials[b];
  cross = block_sum_d(cross);
  const double quad = gram_dot_block(GW, GH, k * k);
  if (threadIdx.x == 0) *loss = 0.5 * ((n2a[0] + n2a[1]) - 2.0 * cross + quad);
}
}  // namespace

cudaError_t launch_loss(const float *P, const float *Ht, int64_t len, const float *GW,
                        const float *GH, int k, const double *n2a, double *partials, int nparts,
                        double *loss, cudaStream_t s) {
  k_dot_partial<<<nparts, 256, 0, s>>>(P, Ht, len, partials);
  k_loss_final<<<1, 1024, 0, s>>>(partials, nparts, GW, GH, k, n2a, loss);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_norm2(const float *A, int64_t m, int64_t n, int64_t lda, double *partials,
                         int nparts, double *out, cudaStream_t s) {
  k_norm2_partial<<<nparts, 256, 0, s>>>(A, m, n, lda, partials);
  k_sum_partials<<<1, 256, 0, s>>>(partials, nparts, out);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_norm2_vec(const float *v, int64_t len, double *partials, int nparts,
                             double *out, cudaStream_t s) {
  k_norm2_vec_partial<<<nparts, 256, 0, s>>>(v, len, partials);
  k_sum_partials<<<1, 256, 0, s>>>(partials, nparts, out);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_relres(const float *P, const float *Ht, int64_t len, const float *GW,
                          const float *GH, int k, const double *n2a, double *partials,
                          int nparts, double *relres_dev, DevCounters *ctr, double *last,
                          cudaStream_t s) {
  k_dot_partial<<<nparts, 256, 0, s>>>(P, Ht, len, partials);
  k_relres_final<<<1, 1024, 0, s>>>(partials, nparts, GW, GH, k, n2a, relres_dev, ctr, last);
  g_launches += 2;
  return cudaGetLastError();
}

}  // namespace aunmf
