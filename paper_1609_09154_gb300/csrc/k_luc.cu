// k_luc.cu -- local update computations (LUC) for MU and HALS.
//
// Both factors are held as row-major "rows x k" matrices (W, and H^T for H),
// so one kernel serves both updates.  For k <= 64 two threads share one row
// (k_luc_tpr).  Above, one warp owns one row; lane l holds the entries
// j = l, l + 32, ... (KT = ceil(k / 32) per lane, rounded up to 12 or 16
// above 256; k <= 512), and the k x k
// Gram matrix is staged in shared memory when it fits.
#include <math.h>

#include "internal.cuh"

namespace aunmf {
namespace {

constexpr int kLucThreads = 256;
constexpr int kLucWarps = kLucThreads / kWarp;
constexpr int kSmemGramMaxK = 108;  // 108*108*4 B < 48 KB default dynamic limit
constexpr int kTprMaxK = 64;        // two-threads-per-row forms up to this k

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool SMEM>
__device__ __forceinline__ const float *stage_gram(const float *G, int k, float *sG) {
  if constexpr (!SMEM) {
    return G;
  } else {
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) sG[e] = G[e];
    __syncthreads();
    return sG;
  }
}

// MU (Sec. 4.1, Eq. muupdate) on each row x of X with p the row of P:
//   x_j <- x_j p_j / ((x G)_j + eps), all j at once (old x on the right).
template <int KT, bool SMEM>
__global__ void __launch_bounds__(kLucThreads)
    k_mu(float *__restrict__ X, const float *__restrict__ P, const float *__restrict__ Gg,
         int64_t rows, int k, float eps) {
  extern __shared__ float sG[];
  const float *G = stage_gram<SMEM>(Gg, k, sG);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * kLucWarps + (threadIdx.x >> 5);
  const int64_t wstride = (int64_t)gridDim.x * kLucWarps;
  for (int64_t r = w0; r < rows; r += wstride) {
    float x[KT], den[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      x[t] = j < k ? X[r * k + j] : 0.f;
      den[t] = 0.f;
    }
#pragma unroll
    for (int tl = 0; tl < KT; ++tl) {
      for (int ll = 0; ll < 32; ++ll) {
        const int l = 32 * tl + ll;
        if (l >= k) break;
        const float xl = __shfl_sync(0xffffffffu, x[tl], ll);
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          const int j = lane + 32 * t;
          if (j < k) den[t] = fmaf(xl, G[l * k + j], den[t]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      if (j < k) X[r * k + j] = x[t] * P[r * k + j] / (den[t] + eps);
    }
  }
}

// HALS column sweep (Sec. 4.2, Eq. halsupdate, exact coordinate steps):
//   for i = 0..k-1:  x_i <- max(0, x_i + (p_i - (x G)_i) / G_ii)
// with the current x (earlier entries already updated); G_ii <= 0 skips i.
template <int KT, bool SMEM>
__global__ void __launch_bounds__(kLucThreads)
    k_hals(float *__restrict__ X, const float *__restrict__ P, const float *__restrict__ Gg,
           int64_t rows, int k, int unit) {
  extern __shared__ float sG[];
  const float *G = stage_gram<SMEM>(Gg, k, sG);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * kLucWarps + (threadIdx.x >> 5);
  const int64_t wstride = (int64_t)gridDim.x * kLucWarps;
  for (int64_t r = w0; r < rows; r += wstride) {
    float x[KT], p[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      x[t] = j < k ? X[r * k + j] : 0.f;
      p[t] = j < k ? P[r * k + j] : 0.f;
    }
#pragma unroll
    for (int ti = 0; ti < KT; ++ti) {
      for (int ii = 0; ii < 32; ++ii) {
        const int i = 32 * ti + ii;
        if (i >= k) break;
        const float* Gi = G + i * k;  // G is symmetric: row i = column i
        float part = 0.f;
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          const int j = lane + 32 * t;
          if (j < k) part = fmaf(x[t], Gi[j], part);
        }
        const float dot = warp_sum(part);
        const float gii = Gi[i];
        if (lane == ii && (unit || gii > 0.f)) {
          // unit: Eq. halsupdate as printed, no division by G_ii
          const float v = x[ti] + (unit ? p[ti] - dot : (p[ti] - dot) / gii);
          x[ti] = v > 0.f ? v : 0.f;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      if (j < k) X[r * k + j] = x[t];
    }
  }
}

// The same sweep for wide ranks (k > 108 with k % 4 == 0, the Gram read
// through L1): lane l holds the entries j = 128 t + 4 l + u (t < KT4, u < 4)
// of R rows, so a coordinate's row of G arrives as KT4 16-byte loads shared
// by the R rows, instead of 32 KT4 / 8 scalar loads per row (the scalar form
// spent ~95 instructions per row and coordinate at k = 512, most of them
// load issue and 64-bit address arithmetic, at 41 % issue).
template <int KT4, int R>
__device__ __forceinline__ void hals4_rows(float *__restrict__ X, const float *__restrict__ P,
                                           const float *__restrict__ G, int64_t rows, int k,
                                           int unit) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * kLucWarps + (threadIdx.x >> 5);
  const int64_t wstride = (int64_t)gridDim.x * kLucWarps;
  const int k4 = k >> 2;
  const float4 *G4 = reinterpret_cast<const float4 *>(G);
  for (int64_t rb = w0 * R; rb < rows; rb += wstride * R) {
    float4 x[R][KT4], p[R][KT4];
#pragma unroll
    for (int rho = 0; rho < R; ++rho) {
      const int64_t r = rb + rho;
#pragma unroll
      for (int t = 0; t < KT4; ++t) {
        const int j4 = 32 * t + lane;  // float4 group of entries 4 j4 .. 4 j4 + 3
        const bool in = r < rows && j4 < k4;
        x[rho][t] = in ? reinterpret_cast<const float4 *>(X + r * k)[j4] : make_float4(0.f, 0.f, 0.f, 0.f);
        p[rho][t] = in ? reinterpret_cast<const float4 *>(P + r * k)[j4] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int t = 0; t < KT4; ++t) {
      for (int l = 0; l < 32; ++l) {
        const int i0 = 128 * t + 4 * l;
        if (i0 >= k) break;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u;
          const float4 *Gi = G4 + (size_t)i * k4;  // G is symmetric: row i = column i
          float4 g[KT4];
#pragma unroll
          for (int tt = 0; tt < KT4; ++tt) {
            const int j4 = 32 * tt + lane;
            g[tt] = j4 < k4 ? Gi[j4] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
          const float gii = G[(size_t)i * k + i];
#pragma unroll
          for (int rho = 0; rho < R; ++rho) {
            float part = 0.f;
#pragma unroll
            for (int tt = 0; tt < KT4; ++tt) {
              part = fmaf(x[rho][tt].x, g[tt].x, part);
              part = fmaf(x[rho][tt].y, g[tt].y, part);
              part = fmaf(x[rho][tt].z, g[tt].z, part);
              part = fmaf(x[rho][tt].w, g[tt].w, part);
            }
            const float dot = warp_sum(part);
            if (lane == l && (unit || gii > 0.f)) {
              float *xe = &x[rho][t].x + u;
              const float pe = (&p[rho][t].x)[u];
              const float v = *xe + (unit ? pe - dot : (pe - dot) / gii);
              *xe = v > 0.f ? v : 0.f;
            }
          }
        }
      }
    }
#pragma unroll
    for (int rho = 0; rho < R; ++rho) {
      const int64_t r = rb + rho;
#pragma unroll
      for (int t = 0; t < KT4; ++t) {
        const int j4 = 32 * t + lane;
        if (r < rows && j4 < k4) reinterpret_cast<float4 *>(X + r * k)[j4] = x[rho][t];
      }
    }
  }
}

// The sweep with the compiler's own register choice, and with registers
// capped at 128 for two blocks per SM (a launch bound with a minimum of one
// block already changes the choice: 79 against 62 registers at KT4 = 3).
template <int KT4, int R>
__global__ void __launch_bounds__(kLucThreads)
    k_hals4(float *__restrict__ X, const float *__restrict__ P, const float *__restrict__ G,
            int64_t rows, int k, int unit) {
  hals4_rows<KT4, R>(X, P, G, rows, k, unit);
}
template <int KT4, int R>
__global__ void __launch_bounds__(kLucThreads, 2)
    k_hals4_capped(float *__restrict__ X, const float *__restrict__ P, const float *__restrict__ G,
                   int64_t rows, int k, int unit) {
  hals4_rows<KT4, R>(X, P, G, rows, k, unit);
}

// Gradient rows of 0.5 ||A - W H||_F^2: out = g (X G - P) for X rows x k,
// G k x k, P rows x k (X = W, G = H H^T, P = A H^T gives dL/dW; X = H^T,
// G = W^T W, P = (W^T A)^T gives (dL/dH)^T).  g is read from device memory
// (NULL: g = 1).  Same lane layout as k_mu.
template <int KT, bool SMEM>
__global__ void __launch_bounds__(kLucThreads)
    k_xg_minus_p(const float *__restrict__ X, const float *__restrict__ P,
                 const float *__restrict__ Gg, int64_t rows, int k, const float *__restrict__ gscale,
                 float *__restrict__ out) {
  extern __shared__ float sG[];
  const float *G = stage_gram<SMEM>(Gg, k, sG);
  const float g = gscale ? *gscale : 1.f;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * kLucWarps + (threadIdx.x >> 5);
  const int64_t wstride = (int64_t)gridDim.x * kLucWarps;
  for (int64_t r = w0; r < rows; r += wstride) {
    float x[KT], acc[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      x[t] = j < k ? X[r * k + j] : 0.f;
      acc[t] = 0.f;
    }
#pragma unroll
    for (int tl = 0; tl < KT; ++tl) {
      for (int ll = 0; ll < 32; ++ll) {
        const int l = 32 * tl + ll;
        if (l >= k) break;
        const float xl = __shfl_sync(0xffffffffu, x[tl], ll);
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          const int j = lane + 32 * t;
          if (j < k) acc[t] = fmaf(xl, G[l * k + j], acc[t]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      if (j < k) out[r * k + j] = g * (acc[t] - P[r * k + j]);
    }
  }
}

// HALS normalisation (Eq. halsupdate, w^i / ||w^i||, compensated in H):
// s_i = sqrt(GW_ii); X(:, i) /= s_i; Y(:, i) *= s_i; GW_ij /= s_i s_j.
// A warp per row, its lanes on the row's entries (no index division per
// entry: a 64-bit remainder costs ~40 instructions and bound the pass at
// 5.9e9 entries); the column scales are staged once per block.
__global__ void k_hals_scale_rows(float *__restrict__ X, int64_t rows, int k,
                                  const float *__restrict__ GW, bool divide) {
  // the factor per column: 1 / s_i (divide) or s_i, 1 where G_ii <= 0; a
  // product with the reciprocal differs from the quotient by at most an ulp,
  // and a division per entry bound the pass (0.1 ms for 5e7 entries)
  __shared__ float sc[AUNMF_K_MAX];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const float g = GW[i * k + i];
    const float si = g > 0.f ? sqrtf(g) : 1.f;  // >= 3.7e-23: 1 / si is finite
    sc[i] = divide ? 1.f / si : si;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t ws = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if ((k & 1) == 0 && (reinterpret_cast<uintptr_t>(X) & 7) == 0) {
    // even k: rows start on 8-byte boundaries, a lane scales two entries
    for (int64_t r = w0; r < rows; r += ws) {
      float2 *x = reinterpret_cast<float2 *>(X + r * k);
      for (int i = lane; 2 * i < k; i += 32) {
        float2 v = x[i];
        v.x *= sc[2 * i];
        v.y *= sc[2 * i + 1];
        x[i] = v;
      }
    }
    return;
  }
  for (int64_t r = w0; r < rows; r += ws) {
    float *x = X + r * k;
    for (int i = lane; i < k; i += 32) x[i] *= sc[i];
  }
}

__global__ void __launch_bounds__(512) k_hals_scale_gram(float *__restrict__ GW, int k) {
  // one block of 32 x 16 threads: read the diagonal first, then rescale,
  // 16 rows at a time with a warp along each (no index division per entry:
  // with one it took 0.58 ms at k = 512)
  __shared__ float sd[AUNMF_K_MAX];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int i = tid; i < k; i += blockDim.x * blockDim.y) {
    const float g = GW[i * k + i];
    sd[i] = g > 0.f ? sqrtf(g) : 1.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < k; i += blockDim.y) {
    const float si = sd[i];
    float *row = GW + (size_t)i * k;
    for (int j = threadIdx.x; j < k; j += blockDim.x) row[j] = row[j] / (si * sd[j]);
  }
}

// ---------------------------------------------------------------------------
// Two-threads-per-row forms for k <= 64 (the same three updates).  A warp
// takes 16 consecutive rows, copies them into a shared tile (row stride KP +
// 1, odd) with asynchronous 4-byte copies, all in flight at once; lanes 2r
// and 2r + 1 then share row r, each keeping one half of it (KH = KP / 2
// entries) in registers.  For coordinate i each thread forms its half of (x
// G)_i, one shuffle adds the halves, and the thread that holds x_i updates
// it: no shuffle per entry, half the dependent FMA chain per coordinate and
// half the registers of a thread per row, so twice the warps stay resident.
// The k x k matrix is staged transposed and zero-padded to KP, so (x G)_i =
// sum_j x_j G_ji reads row i of the staged copy with 16-byte loads; padded
// coordinates have G_ii = 0 and stay 0.
enum LucOp { kOpMu = 0, kOpHals = 1, kOpGrad = 2, kOpHalsUnit = 3 };
constexpr int kTprThreads = 256;
constexpr int kTprWarps = kTprThreads / kWarp;
constexpr int kTprRows = 16;  // rows per warp

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  // src-size 0 fills the 4 bytes with zeros and reads nothing
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// tile rows 0..kTprRows-1 = src rows 0..nr-1 (row length k, contiguous), zeros
// elsewhere; the warp's copies complete before it returns.
template <int KP>
__device__ __forceinline__ void tile_in(const float *__restrict__ src, int nr, int k, float *tile,
                                        int lane) {
  constexpr int LDT = KP + 1;
#pragma unroll 4
  for (int rr = 0; rr < kTprRows; ++rr)
#pragma unroll
    for (int c = lane; c < KP; c += 32) {
      const bool v = rr < nr && c < k;
      cp_async4(tile + rr * LDT + c, v ? src + (int64_t)rr * k + c : src, v);
    }
  cp_async_wait_all();
  __syncwarp();
}

template <int KP>
__device__ __forceinline__ void tile_out(float *__restrict__ dst, int nr, int k, const float *tile,
                                         int lane) {
  constexpr int LDT = KP + 1;
  __syncwarp();
  for (int rr = 0; rr < nr; ++rr)
    for (int c = lane; c < k; c += 32) dst[(int64_t)rr * k + c] = tile[rr * LDT + c];
  __syncwarp();
}

// This thread's half of (x G)_i: x its KH entries (columns h*KH ...), the
// staged G^T row i from the same column.
template <int KH>
__device__ __forceinline__ float xg_half(const float (&x)[KH], const float *gi) {
  const float4 *g4 = reinterpret_cast<const float4 *>(gi);
  float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
#pragma unroll
  for (int q = 0; q < KH / 4; ++q) {
    const float4 g = g4[q];
    d0 = fmaf(x[4 * q], g.x, d0);
    d1 = fmaf(x[4 * q + 1], g.y, d1);
    d2 = fmaf(x[4 * q + 2], g.z, d2);
    d3 = fmaf(x[4 * q + 3], g.w, d3);
  }
  return (d0 + d1) + (d2 + d3);
}

template <int KP, int OP>
__global__ void __launch_bounds__(kTprThreads)
    k_luc_tpr(float *__restrict__ X, const float *__restrict__ P, const float *__restrict__ G,
              int64_t rows, int k, float eps, const float *__restrict__ gscale,
              float *__restrict__ out) {
  constexpr int LDT = KP + 1;
  constexpr int KH = KP / 2;
  static_assert(KH % 4 == 0, "half rows of whole 16-byte groups");
  extern __shared__ __align__(16) float smt[];
  float *sGt = smt;  // KP x KP: sGt[i][j] = G[j][i], zero outside k x k
  // HALS: 1 / G_ii; 0 where G_ii <= 0 (the coordinate is left as it is), -1
  // where the reciprocal overflows (a subnormal G_ii: divided by it instead)
  float *sInv = smt + KP * KP;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int h = lane & 1, rw = lane >> 1;  // half of row rw of the warp's rows
  float *tile = sInv + KP + wib * kTprRows * LDT;
  for (int e = threadIdx.x; e < KP * KP; e += blockDim.x) {
    const int i = e / KP, j = e % KP;
    sGt[e] = (i < k && j < k) ? G[j * k + i] : 0.f;
  }
  // the HALS step divides by G_ii for every row: one reciprocal per block
  // instead (the product differs from the quotient by at most an ulp)
  for (int i = threadIdx.x; i < KP; i += blockDim.x) {
    const float gii = i < k ? G[i * k + i] : 0.f;
    const float r = gii > 0.f ? 1.f / gii : 0.f;
    sInv[i] = isfinite(r) ? r : -1.f;
  }
  __syncthreads();
  const float g = (OP == kOpGrad && gscale) ? *gscale : 1.f;
  float *dst = OP == kOpGrad ? out : X;
  const int64_t groups = (rows + kTprRows - 1) / kTprRows;
  for (int64_t grp = (int64_t)blockIdx.x * kTprWarps + wib; grp < groups;
       grp += (int64_t)gridDim.x * kTprWarps) {
    const int64_t r0 = grp * kTprRows;
    const int nr = (int)min((int64_t)kTprRows, rows - r0);
    tile_in<KP>(X + r0 * k, nr, k, tile, lane);
    float x[KH];
    float *t = tile + rw * LDT + h * KH;  // this thread's half of its row
#pragma unroll
    for (int j = 0; j < KH; ++j) x[j] = t[j];
    __syncwarp();
    tile_in<KP>(P + r0 * k, nr, k, tile, lane);
    if constexpr (OP == kOpHals || OP == kOpHalsUnit) {
      // x_i <- max(0, x_i + (p_i - (x G)_i) / G_ii), i ascending, with the
      // entries before i already updated; G_ii <= 0 leaves x_i as it is.
      // kOpHalsUnit: Eq. halsupdate as printed, without the division.
#pragma unroll
      for (int i = 0; i < KP; ++i) {
        const int own = i / KH, il = i % KH;  // the half that holds x_i
        const float inv = sInv[i];
        if (OP == kOpHalsUnit ? i < k : inv != 0.f) {
          float d = xg_half<KH>(x, sGt + i * KP + h * KH);
          d += __shfl_xor_sync(0xffffffffu, d, 1);
          if (h == own) {
            const float c = t[il] - d;
            const float v = x[il] + (OP == kOpHalsUnit ? c
                                                        : (inv > 0.f ? c * inv : c / sGt[i * KP + i]));
            x[il] = v > 0.f ? v : 0.f;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < KH; ++j) t[j] = x[j];
    } else {
      // every entry from the old x: MU x_j p_j / ((x G)_j + eps), gradient
      // g ((x G)_j - p_j); the result replaces p_j in the tile
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        if (j >= k) break;
        float d = xg_half<KH>(x, sGt + j * KP + h * KH);
        d += __shfl_xor_sync(0xffffffffu, d, 1);
        const int own = j / KH, jl = j % KH;
        if (h == own) t[jl] = OP == kOpMu ? x[jl] * t[jl] / (d + eps) : g * (d - t[jl]);
      }
    }
    tile_out<KP>(dst + r0 * k, nr, k, tile, lane);
  }
}

template <int KP, int OP>
cudaError_t launch_tpr(float *X, const float *P, const float *G, int64_t rows, int k, float eps,
                       const float *gscale, float *out, cudaStream_t s) {
  const size_t smem =
      sizeof(float) * ((size_t)KP * KP + KP + (size_t)kTprWarps * kTprRows * (KP + 1));
  cudaFuncSetAttribute(k_luc_tpr<KP, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // one wave of resident blocks (a second, partial wave would leave most
  // SMs idle for its whole length), each walking its share of row groups
  static int resident = 0;
  if (!resident) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_luc_tpr<KP, OP>, kTprThreads, smem);
    resident = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 152);
  }
  const int64_t groups = (rows + kTprRows - 1) / kTprRows;
  int64_t nb = (groups + kTprWarps - 1) / kTprWarps;
  if (nb > resident) nb = resident;
  k_luc_tpr<KP, OP><<<(unsigned)nb, kTprThreads, smem, s>>>(X, P, G, rows, k, eps, gscale, out);
  g_launches += 1;
  return cudaGetLastError();
}

template <int OP>
cudaError_t launch_tpr_k(float *X, const float *P, const float *G, int64_t rows, int k, float eps,
                         const float *gscale, float *out, cudaStream_t s) {
  if (k <= 16) return launch_tpr<16, OP>(X, P, G, rows, k, eps, gscale, out, s);
  if (k <= 32) return launch_tpr<32, OP>(X, P, G, rows, k, eps, gscale, out, s);
  if (k <= 48) return launch_tpr<48, OP>(X, P, G, rows, k, eps, gscale, out, s);
  if (k <= 56) return launch_tpr<56, OP>(X, P, G, rows, k, eps, gscale, out, s);
  return launch_tpr<64, OP>(X, P, G, rows, k, eps, gscale, out, s);
}

int luc_blocks(int64_t rows) {
  int64_t nb = (rows + kLucWarps - 1) / kLucWarps;
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  return (int)nb;
}

#define AUNMF_KT_SWITCH(KT_VAL, CALL) \
  switch (KT_VAL) {                   \
    case 1: CALL(1); break;           \
    case 2: CALL(2); break;           \
    case 3: CALL(3); break;           \
    case 4: CALL(4); break;           \
    case 5: CALL(5); break;           \
    case 6: CALL(6); break;           \
    case 7: CALL(7); break;           \
    case 8: CALL(8); break;           \
    case 9:                           \
    case 10:                          \
    case 11:                          \
    case 12: CALL(12); break;         \
    default: CALL(16); break;         \
  }

// ---------------------------------------------------------------- HALS as printed
// The W sweep of Eq. halsupdate as printed: w^i <- [w^i + P^i - W G^i]_+ with
// no division by G_ii, and w^i normalised before column i + 1 is updated (H
// is not rescaled).  Every column waits for a norm over all rows, so the
// sweep is one cooperative launch: threads own rows (grid-strided); after
// column i the blocks' FP64 sums of squares meet behind a bounded grid
// barrier, each block adds them in block order (the same norm everywhere),
// and each thread rescales its rows' column i when it next reads them.
constexpr int kPrintedThreads = 256;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// true once every block of the grid has arrived for the gen-th time (the
// counter starts at 0); false, with *err set, after `limit` SM clocks or once
// another block has given up.  skip (test hook): this block does not arrive.
__device__ bool grid_barrier(unsigned *count, unsigned gen, int *err, long long limit,
                             bool skip) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!skip) {
      __threadfence();
      atomicAdd(count, 1u);
    }
    const unsigned target = gen * gridDim.x;
    const long long t0 = clock64();
    ok = 1;
    while (ld_acquire_u32(count) < target) {
      if (clock64() - t0 > limit || *(volatile int *)err) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double block_sum_d256(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kPrintedThreads / 32; ++w) t += red[w];
  return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kPrintedThreads)
    k_hals_w_printed(float *__restrict__ W, const float *__restrict__ P,
                     const float *__restrict__ Gg, int64_t rows, int k, int gsm,
                     double *__restrict__ part, unsigned *bar, int *err, long long limit,
                     int inject) {
  extern __shared__ float sG[];
  __shared__ double red[kPrintedThreads / 32];
  __shared__ float s_inv;
  const float *G = Gg;
  if (gsm) {
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) sG[e] = Gg[e];
    __syncthreads();
    G = sG;
  }
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  float inv = 1.f;  // 1 / ||w^{i-1}||, or 1 for a zero column
  for (int i = 0; i < k; ++i) {
    double ss = 0.0;
    for (int64_t r = tid; r < rows; r += nt) {
      float *x = W + r * k;
      if (i > 0) x[i - 1] *= inv;
      float d = 0.f;
      for (int l = 0; l < k; ++l) d = fmaf(x[l], G[l * k + i], d);
      const float v = x[i] + P[r * k + i] - d;
      const float y = v > 0.f ? v : 0.f;
      x[i] = y;
      ss = fma((double)y, (double)y, ss);
    }
    const double bsum = block_sum_d256(ss, red);
    double *pi = part + (size_t)(i & 1) * gridDim.x;
    if (threadIdx.x == 0) pi[blockIdx.x] = bsum;
    // inject (test hook): block 0 never arrives at the first barrier
    if (!grid_barrier(bar, (unsigned)(i + 1), err, limit, inject && i == 0 && blockIdx.x == 0))
      return;
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(pi + b);
      s_inv = t > 0.0 ? (float)(1.0 / sqrt(t)) : 1.f;
    }
    __syncthreads();
    inv = s_inv;
  }
  for (int64_t r = tid; r < rows; r += nt) W[r * k + k - 1] *= inv;
}

// ---------------------------------------------------------------- projected gradient
// Per block: sum over rows of X (rows x k) of p^2, p the projected entry of
// g = (X G - P)_rj: g where X_rj > 0, else min(0, g).  A warp per row; lane
// l holds x_j and g_j for j = l, l + 32, ...; x_l is broadcast by shuffle.
template <int KT>
__global__ void __launch_bounds__(kLucThreads)
    k_pgrad_partial(const float *__restrict__ X, const float *__restrict__ P,
                    const float *__restrict__ G, int64_t rows, int k, double *__restrict__ part) {
  __shared__ double red[kLucWarps];
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * kLucWarps + (threadIdx.x >> 5);
  const int64_t ws = (int64_t)gridDim.x * kLucWarps;
  double acc = 0.0;
  for (int64_t r = w0; r < rows; r += ws) {
    float x[KT], g[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      x[t] = j < k ? X[r * k + j] : 0.f;
      g[t] = 0.f;
    }
#pragma unroll
    for (int tl = 0; tl < KT; ++tl)
      for (int ll = 0; ll < 32; ++ll) {
        const int l = 32 * tl + ll;
        if (l >= k) break;
        const float xl = __shfl_sync(0xffffffffu, x[tl], ll);
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          const int j = lane + 32 * t;
          if (j < k) g[t] = fmaf(xl, G[l * k + j], g[t]);
        }
      }
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int j = lane + 32 * t;
      if (j < k) {
        const float gg = g[t] - P[r * k + j];
        const float pr = x[t] > 0.f ? gg : fminf(gg, 0.f);
        acc = fma((double)pr, (double)pr, acc);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kLucWarps; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// out[ctr->iter] = sqrt(sum of the partials), in partial order.
__global__ void k_pgrad_final(const double *__restrict__ part, int n, const DevCounters *ctr,
                              double *__restrict__ out) {
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int b = 0; b < n; ++b) t += part[b];
  out[ctr->iter] = sqrt(t);
}

}  // namespace

int printed_sweep_blocks() { return 2 * 152; }

cudaError_t launch_hals_w_printed(float *W, const float *P, const float *G, int64_t rows, int k,
                                  double *part, unsigned *bar, int *err, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  int gsm = k <= kSmemGramMaxK ? 1 : 0;
  const size_t smem = gsm ? sizeof(float) * k * k : 0;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hals_w_printed, kPrintedThreads, smem);
  int64_t grid = (int64_t)per_sm * sms;
  const int64_t need = (rows + kPrintedThreads - 1) / kPrintedThreads;
  if (grid > need) grid = need;
  if (grid > printed_sweep_blocks()) grid = printed_sweep_blocks();
  if (grid < 1) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  long long limit = fault::wait_cycles();
  int inject = fault::site() == AUNMF_INJECT_GRID_BARRIER ? 1 : 0;
  void *args[] = {&W, &P, &G, &rows, &k, &gsm, &part, &bar, &err, &limit, &inject};
  e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_hals_w_printed), (int)grid,
                                  kPrintedThreads, args, smem, s);
  g_launches += 1;
  return e;
}

int pgrad_blocks() { return 152 * 2; }

cudaError_t launch_pgrad_partial(const float *X, const float *P, const float *G, int64_t rows,
                                 int k, double *part, cudaStream_t s) {
  const int kt = (k + 31) / 32, nb = pgrad_blocks();
  if (rows == 0) return cudaMemsetAsync(part, 0, sizeof(double) * nb, s);
#define AUNMF_CALL_PG(KT) k_pgrad_partial<KT><<<nb, kLucThreads, 0, s>>>(X, P, G, rows, k, part);
  AUNMF_KT_SWITCH(kt, AUNMF_CALL_PG)
#undef AUNMF_CALL_PG
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_pgrad_final(const double *part, int n, const DevCounters *ctr, double *out,
                               cudaStream_t s) {
  k_pgrad_final<<<1, 32, 0, s>>>(part, n, ctr, out);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_mu(float *X, const float *P, const float *G, int64_t rows, int k, float eps,
                      cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  if (k <= kTprMaxK) return launch_tpr_k<kOpMu>(X, P, G, rows, k, eps, nullptr, nullptr, s);
  const int kt = (k + 31) / 32, nb = luc_blocks(rows);
  const bool sm = k <= kSmemGramMaxK;
  const size_t smem = sm ? sizeof(float) * k * k : 0;
#define AUNMF_CALL_MU(KT)                                                          \
  if (sm) k_mu<KT, true><<<nb, kLucThreads, smem, s>>>(X, P, G, rows, k, eps);     \
  else k_mu<KT, false><<<nb, kLucThreads, 0, s>>>(X, P, G, rows, k, eps);
  AUNMF_KT_SWITCH(kt, AUNMF_CALL_MU)
#undef AUNMF_CALL_MU
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_hals(float *X, const float *P, const float *G, int64_t rows, int k,
                        cudaStream_t s, bool unit) {
  if (rows == 0) return cudaSuccess;
  if (k <= kTprMaxK)
    return unit ? launch_tpr_k<kOpHalsUnit>(X, P, G, rows, k, 0.f, nullptr, nullptr, s)
                : launch_tpr_k<kOpHals>(X, P, G, rows, k, 0.f, nullptr, nullptr, s);
  const int kt = (k + 31) / 32, nb = luc_blocks(rows);
  const bool sm = k <= kSmemGramMaxK;
  const size_t smem = sm ? sizeof(float) * k * k : 0;
  const int u = unit ? 1 : 0;
  if (!sm && (k & 3) == 0 && ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(P) |
                               reinterpret_cast<uintptr_t>(G)) & 15) == 0) {
    // rows per warp and the register cap, measured (update phase per
    // iteration at 96000 x 64000): k <= 256 two rows; 257..384 one row (two
    // rows: 7.27 against 6.34 ms at k = 384); above, two rows capped at 128
    // registers for two blocks per SM (10.3 ms at k = 512; one row 12.4 ms;
    // two rows uncapped took 136 registers, one block per SM: 20.3 ms)
    const int kt4 = (k + 127) / 128, R = kt4 == 3 ? 1 : 2;
    int64_t nbw = (rows + kLucWarps * R - 1) / (kLucWarps * R);
    if (nbw > 152 * 8) nbw = 152 * 8;
    switch (kt4) {
      case 1: k_hals4<1, 2><<<(unsigned)nbw, kLucThreads, 0, s>>>(X, P, G, rows, k, u); break;
      case 2: k_hals4<2, 2><<<(unsigned)nbw, kLucThreads, 0, s>>>(X, P, G, rows, k, u); break;
      case 3: k_hals4<3, 1><<<(unsigned)nbw, kLucThreads, 0, s>>>(X, P, G, rows, k, u); break;
      default: k_hals4_capped<4, 2><<<(unsigned)nbw, kLucThreads, 0, s>>>(X, P, G, rows, k, u); break;
    }
    g_launches += 1;
    return cudaGetLastError();
  }
#define AUNMF_CALL_HALS(KT)                                                       \
  if (sm) k_hals<KT, true><<<nb, kLucThreads, smem, s>>>(X, P, G, rows, k, u);    \
  else k_hals<KT, false><<<nb, kLucThreads, 0, s>>>(X, P, G, rows, k, u);
  AUNMF_KT_SWITCH(kt, AUNMF_CALL_HALS)
#undef AUNMF_CALL_HALS
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_xg_minus_p(const float *X, const float *P, const float *G, int64_t rows, int k,
                              const float *gscale, float *out, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  if (k <= kTprMaxK)
    return launch_tpr_k<kOpGrad>(const_cast<float *>(X), P, G, rows, k, 0.f, gscale, out, s);
  const int kt = (k + 31) / 32, nb = luc_blocks(rows);
  const bool sm = k <= kSmemGramMaxK;
  const size_t smem = sm ? sizeof(float) * k * k : 0;
#define AUNMF_CALL_XG(KT)                                                                  \
  if (sm) k_xg_minus_p<KT, true><<<nb, kLucThreads, smem, s>>>(X, P, G, rows, k, gscale, out); \
  else k_xg_minus_p<KT, false><<<nb, kLucThreads, 0, s>>>(X, P, G, rows, k, gscale, out);
  AUNMF_KT_SWITCH(kt, AUNMF_CALL_XG)
#undef AUNMF_CALL_XG
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_hals_normalise(float *X, int64_t rows_x, float *Y, int64_t rows_y, float *GW,
                                  int k, cudaStream_t s) {
  auto nb = [](int64_t total) {
    int64_t b = (total + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
  };
  auto scale = [&](float *Z, int64_t rows, bool divide) {
    k_hals_scale_rows<<<nb(rows * 32), 256, 0, s>>>(Z, rows, k, GW, divide);
  };
  if (rows_x > 0) scale(X, rows_x, true);
  if (Y && rows_y > 0) scale(Y, rows_y, false);
  k_hals_scale_gram<<<1, dim3(32, 16), 0, s>>>(GW, k);
  g_launches += 1 + (rows_x > 0) + (Y && rows_y > 0);
  return cudaGetLastError();
}

}  // namespace aunmf
