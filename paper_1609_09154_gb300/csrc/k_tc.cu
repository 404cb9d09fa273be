// k_tc.cu -- the two products with A on the 5th-generation tensor cores
// (Alg. 1 lines 3-4: A H^T and W^T A), for sm_103a.
//
// Both products are computed as  C (M x k) = X (M x K) * Y (k x K)^T  with X
// and Y stored K-contiguous ("K-major"):
//   A H^T : X = A   (m x n),  Y = H   (k x n)   ->  C = P_W   (m x k)
//   W^T A : X = A^T (n x m),  Y = W^T (k x m)   ->  C = P_H^T (n x k)
// The library keeps a transposed copy of A for the second product (set up
// once per run), so each product streams one copy of A exactly once.
//
// Kernel: persistent, one CTA per SM, 10 warps.
//   warp 0     TMA producer: 256 x 128 B of X and BN x 128 B of Y per stage,
//              128-byte swizzle, into an N-stage shared-memory ring
//   warp 1     owns the TMEM allocation; one thread issues tcgen05.mma
//              (two M = 128 MMAs per K step share the Y tile) and commits
//              stage releases / accumulator-ready to mbarriers
//   warps 2-9  epilogue: tcgen05.ld of the FP32 accumulators (one row per
//              thread), drained into an FP32 accumulator in shared memory,
//              then stored to the split's partial C
// The tensor core adds each MMA's result into its FP32 accumulator with a
// truncating rounding, so a long accumulation chain drifts toward zero: the
// relative bias grows linearly with the number of MMAs in the chain
// (-1e-6 after ~50, -1e-4 after ~5000 on nonnegative data).  Each work unit
// therefore restarts the TMEM accumulator every `chunk_kb` K blocks and the
// epilogue adds the chunk into its own accumulator with round-to-nearest
// FP32 additions, whose errors carry no bias.  The residual's trace form
// (Sec. 5, relative error) takes the difference of numbers near ||A||^2 and
// needs that: a bias of e in W^T A moves the reported relres by ~e / relres.
// Chunk accumulators are double-buffered in TMEM (2 x 2 x BN columns) when
// BN <= 128 so that draining one chunk overlaps the next chunk's MMAs; eight
// epilogue warps (two per TMEM lane quarter, one per 128-row half) keep a
// drain shorter than a chunk.
// Without the hi/lo split (k > 64) each output has one TMEM column; the
// first 64 sums of a row stay in registers and the rest go to shared memory
// or, when they do not fit beside three pipeline stages (BN > 128), to a
// per-CTA column-major accumulator in global memory that stays in L2.  MMA N
// is at most 256: a wider product (k <= 512) runs as two column blocks in
// one launch.
// Work unit = (256-row tile, K split); splits are summed afterwards in a
// fixed order, so results do not depend on scheduling.
//
// Every mbarrier wait is bounded (clock64); on expiry the kernel raises a
// device error flag and skips the rest of its work, then waits (bounded
// again) for the copies and MMAs it has in flight and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdio.h>

#include <algorithm>

#include "internal.cuh"
#include "ptx.cuh"
#include "tc.cuh"

namespace aunmf {
namespace tc {
namespace {

constexpr int kTileM = 256;          // rows of X per work unit (2 x M=128 MMAs)
constexpr int kMaxBN = 256;          // MMA N limit; wider products are split by columns
constexpr int kStageBytesK = 128;    // K extent of one stage in bytes (one 128B swizzle row)
constexpr int kThreads = 320;
#ifndef AUNMF_TC_CHUNK_KB
#define AUNMF_TC_CHUNK_KB 2
#endif
// K blocks (4 MMAs each) per TMEM accumulation chain: with the accumulator in
// shared memory, and when it is added into P in global memory.  Measured
// bias of <W^T A, H> (relative, nonnegative data): 4 K blocks -6e-7 (TF32)
// and -2.5e-7 (BF16), 2 K blocks -2.5e-7 and -1e-7, 1 K block -1.1e-7 and
// -4e-8.  A shared-memory drain of 256 x BN sums per chunk competes with TMA
// and the MMAs for shared-memory bandwidth, so it takes chunks of 2 K
// blocks; sums in registers drain after every K block at ~1.5% below the
// 4-block speed (96000 x 64000, k = 50).
constexpr int kChunkKB = AUNMF_TC_CHUNK_KB;
#ifndef AUNMF_TC_CHUNK_KB_REG
#define AUNMF_TC_CHUNK_KB_REG 1
#endif
constexpr int kChunkKBReg = AUNMF_TC_CHUNK_KB_REG;  // sums in registers
constexpr int kChunkKBGlobal = 4 * AUNMF_TC_CHUNK_KB;
// Above BN = 128 TMEM holds a single chunk buffer and the MMAs wait while it
// drains: 16 K blocks per chain there (relative bias of the products ~-2e-6
// TF32, ~-1e-6 BF16, extrapolated from the 4-block figures), and 32 when the
// sums live in the L2-resident scratch (~-5e-6 / ~-2e-6), whose round trips
// make each drain the longest.
constexpr int kChunkKBLong = 8 * AUNMF_TC_CHUNK_KB;
constexpr int kChunkKBScratch = 16 * AUNMF_TC_CHUNK_KB;

// ------------------------------------------------------------------ PTX
using namespace aunmf::ptx;

// Scratch sums: kept in L2 (evict last) against the stream of X tiles.
__device__ __forceinline__ float ld_keep(const float *p, uint64_t pol) {
  float v;
  asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_keep(float *p, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
template <bool BF16>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
  if constexpr (BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
      : "memory");
}
// 16 columns of the thread's TMEM lane into r[0..15] without waiting; the
// values may be read only after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// Waits for the thread's outstanding tcgen05.ld; the empty volatile asm per
// register orders every later use of r[0..n) after the wait.
template <int N>
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[N]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < N; ++i) asm volatile("" : "+r"(r[i]));
}

// Shared-memory matrix descriptor for a K-major tile in the canonical
// 128-byte-swizzled layout written by TMA (rows of 128 B, 8-row groups of
// 1024 B): start address >> 4, leading offset 16 B (unused for this layout),
// stride offset 1024 B between 8-row groups, descriptor version 1, swizzle
// mode 2 (128 B).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor (kind::tf32 / kind::f16): FP32 accumulator, A and
// B of the same type (TF32 = 2 or BF16 = 1), both K-major, N >> 3 at bit
// 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc(bool bf16, int M, int N) {
  return (1u << 4) | ((bf16 ? 1u : 2u) << 7) | ((bf16 ? 1u : 2u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// One product C (M x k) = X (M x K) * F (k x K)^T of a launch.  A launch
// runs one problem (passed by value) or a group of problems (a device array,
// e.g. all instances of a batch); work units are numbered across the group.
struct GemmProblem {
  CUtensorMap mapX;    // X: M rows x K, box 128 B x 256 rows
  CUtensorMap mapY;    // Y: F (k rows) or its hi/lo split (2k rows), box 128 B x BN rows
  int64_t M, K;
  int64_t unit0;       // first work unit of this problem in the launch
  int64_t total_kb;    // K blocks of 128 bytes
  int64_t per_split;   // K blocks per split
  float *P;            // partials: S x M x ldc, row-major (S == 1: C itself)
  int k;               // columns of C
  int ldc;             // row stride of C and of each partial (floats)
  int BN;              // MMA N (rows of Y rounded up to 16), <= BNmax
  int S;               // K splits
  int pair;            // 1: Y rows (2i, 2i+1) hold hi/lo of F's row i; C_i = acc_2i + acc_2i+1
};

// Launch-wide shape: the shared-memory ring and TMEM are sized for BNmax.
struct GemmLaunch {
  int64_t units;       // total work units
  int nprob;           // problems in `group` (0: the by-value problem only)
  int BNmax;
  int nstages;
  int nbuf;            // TMEM accumulator buffers (1 or 2)
  uint32_t tmem_cols;  // power of two >= nbuf * 2 * BNmax
  int regacc;          // 1: sums in registers (all problems pair, BN <= 128)
  int chunk_kb;        // K blocks per TMEM accumulation chain
  int acc_ld;          // row stride (floats, odd, >= BN/2 for pair problems and BN
                       // otherwise) of the shared-memory accumulator, 256 rows;
                       // 0: chunks are added into `scratch` (or P without one)
  int interleave;      // 1: two problems (`one`, `two`) with equal unit counts; unit u
                       // is unit u / 2 of problem (u + w) % 2, w the wave of unit u & ~1
  float *scratch;      // without a shared accumulator: per-CTA column-major
  int scr_cols;        // accumulators, scr_cols x 256 floats per CTA (L2-resident)
  int *err;
  long long wait_cycles;  // limit of every bounded wait (SM clocks)
  int inject;          // test hook: the first accumulator chunk's ready signal is withheld
};

// The problem that work unit u belongs to, and the unit's index v within it.
__device__ __forceinline__ const GemmProblem *find_problem(const GemmProblem &one,
                                                          const GemmProblem &two,
                                                          const GemmProblem *group,
                                                          const GemmLaunch &L, int64_t u,
                                                          int64_t *v) {
  if (L.interleave) {
    // the pair of units of one tile swaps blocks from one wave to the next,
    // so that a CTA does not get the same (maybe narrower) block every wave
    const int64_t g = u >> 1;
    *v = g;
    return (((u & 1) + (2 * g) / gridDim.x) & 1) ? &two : &one;
  }
  const GemmProblem *p = &one;
  if (group) {
    int lo = 0, hi = L.nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (group[mid].unit0 <= u) lo = mid; else hi = mid - 1;
    }
    p = group + lo;
  }
  *v = u - p->unit0;
  return p;
}

// REGACC: every problem of the launch is a pair problem with BN <= 128
// (k <= 64); each epilogue thread keeps its row's <= 64 sums in registers.
// Otherwise (one TMEM column per output) the first 64 sums of a row stay in
// registers and the rest live in shared memory (or in P).
// SCRATCH: the sums past the first 64 columns live in L.scratch.
template <bool BF16, bool REGACC, bool SCRATCH>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ GemmProblem one, const __grid_constant__ GemmProblem two,
              const GemmProblem *__restrict__ group, const GemmLaunch L) {
  constexpr int ESZ = BF16 ? 2 : 4;
  constexpr int BKE = kStageBytesK / ESZ;  // K elements per stage
  constexpr int KPM = BF16 ? 16 : 8;       // K elements per MMA (32 bytes)
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const uint32_t xbytes = kTileM * kStageBytesK;
  const uint32_t sbytes = xbytes + (uint32_t)L.BNmax * kStageBytesK;
  float *acc_s = L.acc_ld ? reinterpret_cast<float *>(smem + (size_t)L.nstages * sbytes) : nullptr;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)L.nstages * sbytes +
                                                (size_t)kTileM * L.acc_ld * sizeof(float));
  uint64_t *full = bars;
  uint64_t *empty = bars + L.nstages;
  uint64_t *tfull = bars + 2 * L.nstages;
  uint64_t *tempty = tfull + 2;
  uint64_t *drain = tempty + 2;  // completion of every MMA issued, before TMEM is freed
  uint32_t *tslot = reinterpret_cast<uint32_t *>(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < L.nstages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 256);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!group) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&one.mapX) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&one.mapY) : "memory");
    }
    if (L.interleave) asm volatile("prefetch.tensormap [%0];" ::"l"(&two.mapY) : "memory");
  }
  if (warp == 1) tmem_alloc(tslot, L.tmem_cols);
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      // X streams through once (evict first), unless two column blocks share it
      const uint64_t pol_x = L.interleave ? policy_evict_normal() : policy_evict_first();
      const uint64_t pol_y = policy_evict_last();
      int st = 0;
      uint32_t ph = 0;
      bool ok = true;
      int64_t nissued = 0;
      for (int64_t u = blockIdx.x; u < L.units && ok; u += gridDim.x) {
        int64_t v;
        const GemmProblem *p = find_problem(one, two, group, L, u, &v);
        const int64_t tile = v / p->S, sp = v % p->S;
        const int64_t kb0 = sp * p->per_split, kb1 = min(p->total_kb, kb0 + p->per_split);
        const int row0 = (int)(tile * kTileM);
        const uint32_t tx = xbytes + (uint32_t)p->BN * kStageBytesK;
        for (int64_t kb = kb0; kb < kb1; ++kb) {
          if (!mbar_wait(&empty[st], ph ^ 1u, L.err, L.wait_cycles)) { ok = false; break; }
          uint8_t *xs = smem + (size_t)st * sbytes;
          mbar_expect_tx(&full[st], tx);
          // (checked build: a bad coordinate skips the copies; the stage then
          // never fills and the bounded waits end the launch)
          if (AUNMF_BOUND(kb >= 0 && kb * BKE <= 0x7fffffffLL &&
                              ((kb * BKE * ESZ) & 15) == 0 && row0 >= 0,
                          AUNMF_CHECK_TMA_COORD)) {
            tma_load_2d(xs, &p->mapX, &full[st], (int)(kb * BKE), row0, pol_x);
            tma_load_2d(xs + xbytes, &p->mapY, &full[st], (int)(kb * BKE), 0, pol_y);
          }
          ++nissued;
          if (++st == L.nstages) { st = 0; ph ^= 1u; }
        }
      }
      // Every copy issued must land before the CTA exits (one still in
      // flight would write shared memory the CTA no longer owns).  The c-th
      // load into stage s completes phase c of full[s]; on the normal path
      // the MMA warp has waited for all of them, so these return at once.
      const int64_t rounds = nissued / L.nstages, rem = nissued % L.nstages;
      for (int s = 0; s < L.nstages; ++s) {
        const int64_t cnt = rounds + (s < rem ? 1 : 0);
        if (cnt > 0) mbar_wait_drain(&full[s], (uint32_t)((cnt - 1) & 1), L.wait_cycles);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int st = 0, buf = 0;
      uint32_t ph = 0, tph = 0;
      bool ok = true;
      bool withheld = false;
      for (int64_t u = blockIdx.x; u < L.units && ok; u += gridDim.x) {
        int64_t v;
        const GemmProblem *p = find_problem(one, two, group, L, u, &v);
        const int64_t sp = v % p->S;
        const int64_t kb0 = sp * p->per_split, kb1 = min(p->total_kb, kb0 + p->per_split);
        const uint32_t id = idesc(BF16, 128, p->BN);
        for (int64_t cb0 = kb0; cb0 < kb1 && ok; cb0 += L.chunk_kb) {
          const int64_t cb1 = min(kb1, cb0 + (int64_t)L.chunk_kb);
          if (!mbar_wait(&tempty[buf], tph ^ 1u, L.err, L.wait_cycles)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d0 = tbase + (uint32_t)(buf * 2 * L.BNmax);
          const uint32_t d1 = d0 + (uint32_t)L.BNmax;
          for (int64_t kb = cb0; kb < cb1; ++kb) {
            if (!mbar_wait(&full[st], ph, L.err, L.wait_cycles)) { ok = false; break; }
            tc_fence_after();
            const uint32_t xs = su32(smem + (size_t)st * sbytes);
            const uint32_t ys = xs + xbytes;
#pragma unroll
            for (int kk = 0; kk < BKE / KPM; ++kk) {
              const uint32_t off = (uint32_t)(kk * KPM * ESZ);
              const uint64_t bd = sdesc(ys + off);
              const uint32_t acc = (kb > cb0 || kk > 0) ? 1u : 0u;
              mma<BF16>(d0, sdesc(xs + off), bd, id, acc);
              mma<BF16>(d1, sdesc(xs + 128 * kStageBytesK + off), bd, id, acc);
            }
            mma_commit(&empty[st]);
            if (++st == L.nstages) { st = 0; ph ^= 1u; }
          }
          if (!ok) break;
          if (L.inject && !withheld)
            withheld = true;  // test hook: the epilogue's wait for this chunk runs out
          else
            mma_commit(&tfull[buf]);
          if (++buf == L.nbuf) { buf = 0; tph ^= 1u; }
        }
      }
    }
  } else {
    // ---------------- epilogue: warps 2..9; warp w drains TMEM lane quarter
    // q = w % 4 of accumulator half (w - 2) / 4.  Row rl = half * 128 +
    // q * 32 + lane of the unit belongs to one thread for every chunk.
    // TMEM is read in groups of 32 columns (one wait per group) up to BN
    // rounded up to 32; shared accumulator rows are padded to match, so the
    // columns past BN (never copied out) need no guard.
    const int q = warp & 3, half = (warp - 2) >> 2;
    const int rl = half * 128 + q * 32 + lane;
    float *arow = acc_s ? acc_s + (size_t)rl * L.acc_ld : nullptr;
    int buf = 0;
    uint32_t tph = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; u < L.units && ok; u += gridDim.x) {
      int64_t v;
      const GemmProblem *p = find_problem(one, two, group, L, u, &v);
      const int64_t tile = v / p->S, sp = v % p->S;
      const int64_t kb0 = sp * p->per_split, kb1 = min(p->total_kb, kb0 + p->per_split);
      const int64_t M = p->M;
      const int k = p->k, BN = p->BN;
      const int64_t ldc = p->ldc;
      const int64_t row = tile * kTileM + rl;
      float *Pp = p->P + sp * M * ldc;
      const bool live = row < M;
      if constexpr (REGACC) {
        // pair problem, BN <= 128: C_i = acc_2i + acc_2i+1 for i < BN / 2
        float acc[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) acc[j] = 0.f;
        for (int64_t cb0 = kb0; cb0 < kb1; cb0 += L.chunk_kb) {
          if (!mbar_wait(&tfull[buf], tph, L.err, L.wait_cycles)) { ok = false; break; }
          tc_fence_after();
          const uint32_t taddr =
              tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 2 * L.BNmax + half * L.BNmax);
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            if (32 * g >= BN) break;
            uint32_t r[32];
            tmem_ld16_async(taddr + (uint32_t)(32 * g), r);
            tmem_ld16_async(taddr + (uint32_t)(32 * g + 16), r + 16);
            tmem_wait_ld(r);
#pragma unroll
            for (int j = 0; j < 16; ++j)
              acc[16 * g + j] += __uint_as_float(r[2 * j]) + __uint_as_float(r[2 * j + 1]);
          }
          tc_fence_before();
          mbar_arrive(&tempty[buf]);
          if (++buf == L.nbuf) { buf = 0; tph ^= 1u; }
        }
        if (!ok) break;
        if (live) {
          float *dg = Pp + row * ldc;
#pragma unroll
          for (int o = 0; o < 64; ++o)
            if (o < k) dg[o] = acc[o];
        }
        continue;
      }
      // one TMEM column per output (no split): columns 0..63 summed in
      // registers, the rest in the shared accumulator (row stride acc_ld,
      // column c at c - 64), else in the CTA's column-major scratch (column c
      // at (c - 64) * 256: the 32 rows of a warp are 128 contiguous bytes),
      // else in P itself
      const int W32 = (BN + 31) & ~31;
      float *scol =
          SCRATCH ? L.scratch + (size_t)blockIdx.x * L.scr_cols * kTileM + rl : nullptr;
      const uint64_t pol_s = SCRATCH ? policy_evict_last() : 0;
      float racc[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) racc[j] = 0.f;
      bool first = true;
      for (int64_t cb0 = kb0; cb0 < kb1; cb0 += L.chunk_kb) {
        // scratch sums of the first group, loaded while the chunk's MMAs run
        float nx[SCRATCH ? 32 : 1];
        if constexpr (SCRATCH) {
          if (!first) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) nx[jj] = ld_keep(scol + (size_t)jj * kTileM, pol_s);
          }
        }
        if (!mbar_wait(&tfull[buf], tph, L.err, L.wait_cycles)) { ok = false; break; }
        tc_fence_after();
        const uint32_t taddr =
            tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 2 * L.BNmax + half * L.BNmax);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          if (32 * g >= BN) break;
          uint32_t r[32];
          tmem_ld16_async(taddr + (uint32_t)(32 * g), r);
          tmem_ld16_async(taddr + (uint32_t)(32 * g + 16), r + 16);
          tmem_wait_ld(r);
#pragma unroll
          for (int j = 0; j < 32; ++j) racc[32 * g + j] += __uint_as_float(r[j]);
        }
        for (int g0 = 64; g0 < W32; g0 += 32) {
          uint32_t r[32];
          tmem_ld16_async(taddr + (uint32_t)g0, r);
          tmem_ld16_async(taddr + (uint32_t)(g0 + 16), r + 16);
          tmem_wait_ld(r);
          if (arow) {
            // padded rows: whole 32-column groups, a group's loads before its
            // stores (a guard per element serialises load -> add -> store)
            float *d = arow + (g0 - 64);
            float x[32];
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) x[jj] = __uint_as_float(r[jj]);
            if (!first) {
#pragma unroll
              for (int jj = 0; jj < 32; ++jj) x[jj] += d[jj];
            }
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) d[jj] = x[jj];
          } else if constexpr (SCRATCH) {
            // this group's sums are in nx; the next group's are loaded before
            // this group is stored (one L2 round trip per group, overlapped)
            float *d = scol + (size_t)(g0 - 64) * kTileM;
            if (!first) {
#pragma unroll
              for (int jj = 0; jj < 32; ++jj)
                r[jj] = __float_as_uint(__uint_as_float(r[jj]) + nx[jj]);
              if (g0 + 32 < W32) {
#pragma unroll
                for (int jj = 0; jj < 32; ++jj)
                  nx[jj] = ld_keep(d + (size_t)(32 + jj) * kTileM, pol_s);
              }
            }
#pragma unroll
            for (int jj = 0; jj < 32; ++jj)
              st_keep(d + (size_t)jj * kTileM, __uint_as_float(r[jj]), pol_s);
          } else if (live) {
            float *dst = Pp + row * ldc;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj)
              if (g0 + jj < k) {
                const float x = __uint_as_float(r[jj]);
                dst[g0 + jj] = first ? x : dst[g0 + jj] + x;
              }
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[buf]);
        if (++buf == L.nbuf) { buf = 0; tph ^= 1u; }
        first = false;
      }
      if (!ok) break;
      if (live) {
        float *dg = Pp + row * ldc;
#pragma unroll
        for (int o = 0; o < 64; ++o)
          if (o < k) dg[o] = racc[o];
        if (first)
          for (int o = 64; o < k; ++o) dg[o] = 0.f;
        else if (arow)
          for (int o = 64; o < k; ++o) dg[o] = arow[o - 64];
        else if (SCRATCH)
          for (int o = 64; o < k; ++o) dg[o] = scol[(size_t)(o - 64) * kTileM];
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    // every MMA this CTA issued has finished before TMEM is freed: on the
    // normal path the epilogue has already seen the last one complete; after
    // a wait ran out, some may still be running
    if (lane == 0) {
      mma_commit(drain);
      mbar_wait_drain(drain, 0u, L.wait_cycles);
    }
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tbase, L.tmem_cols);
  }
}

// P[e] = sum_s parts[s][e], s ascending.
__global__ void k_sum_splits(const float *__restrict__ parts, int S, int64_t len,
                             float *__restrict__ P) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = parts[e];
    for (int p = 1; p < S; ++p) s += parts[(int64_t)p * len + e];
    P[e] = s;
  }
}

// out (cols x ldo) = in (rows x cols, ld ldi)^T, converting to T (float or bf16).
// FP32 -> TF32 with round-to-nearest (the tensor core would otherwise drop the
// low 13 mantissa bits, a bias toward zero that does not average out on
// nonnegative data); the result is an FP32 bit pattern with those bits zero.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
template <class T>
__device__ __forceinline__ T cvt(float x);
template <>
__device__ __forceinline__ float cvt<float>(float x) { return round_tf32(x); }
template <>
__device__ __forceinline__ uint16_t cvt<uint16_t>(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

template <class T>
__global__ void k_transpose_to(const float *__restrict__ in, int64_t rows, int64_t cols,
                               int64_t ldi, T *__restrict__ out, int64_t ldo) {
  __shared__ float t[32][33];
  const int64_t tr = (rows + 31) / 32, tcn = (cols + 31) / 32;
  for (int64_t tile = blockIdx.x; tile < tr * tcn; tile += gridDim.x) {
    const int64_t r0 = (tile / tcn) * 32, c0 = (tile % tcn) * 32;
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      const int64_t r = r0 + y, c = c0 + threadIdx.x;
      if (r < rows && c < cols) t[y][threadIdx.x] = in[r * ldi + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      const int64_t c = c0 + y, r = r0 + threadIdx.x;
      if (r < rows && c < cols) out[c * ldo + r] = cvt<T>(t[threadIdx.x][y]);
    }
  }
}

// Two-term split of a factor, transposed: for in (rows x k, ld ldi),
//   out row 2c   = hi_c = round(in(:, c)),
//   out row 2c+1 = lo_c = round(in(:, c) - hi_c)      (ld ldo),
// so hi + lo carries the factor to ~2x the bits of one rounded value.
template <class T>
__device__ __forceinline__ float widen(T x);
template <>
__device__ __forceinline__ float widen<float>(float x) { return x; }
template <>
__device__ __forceinline__ float widen<uint16_t>(uint16_t x) {
  return __bfloat162float(__ushort_as_bfloat16(x));
}

template <class T>
__global__ void k_split_transpose(const float *__restrict__ in, int64_t rows, int k, int64_t ldi,
                                  T *__restrict__ out, int64_t ldo) {
  __shared__ float t[32][33];
  const int64_t tr = (rows + 31) / 32, tcn = (k + 31) / 32;
  for (int64_t tile = blockIdx.x; tile < tr * tcn; tile += gridDim.x) {
    const int64_t r0 = (tile / tcn) * 32, c0 = (tile % tcn) * 32;
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      const int64_t r = r0 + y, c = c0 + threadIdx.x;
      if (r < rows && c < k) t[y][threadIdx.x] = in[r * ldi + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      const int64_t c = c0 + y, r = r0 + threadIdx.x;
      if (r < rows && c < k) {
        const float x = t[threadIdx.x][y];
        const T hi = cvt<T>(x);
        out[(2 * c) * ldo + r] = hi;
        out[(2 * c + 1) * ldo + r] = cvt<T>(x - widen<T>(hi));
      }
    }
  }
}

// One pass over A (m x n, lda) for the tensor-core runs: writes the rounded
// copy X (m x n, ld ldx), the rounded transposed copy Xt (n x m, ld ldxt) and
// per-block partial sums of a_ij^2 and of a_ij (round(a_ij) - a_ij) (FP64;
// each thread first adds the 16 terms it holds in FP32).  64 x 64 tiles: thread (ty, c4) loads the four
// 16-byte pieces A[r0 + ty + 16 i][c0 + 4 c4 .. +3], i < 4, before storing
// anything (VEC: rows of A are 16-byte aligned), then the tile is written
// row-contiguously to X and, through shared memory, to Xt.
template <class T>
__device__ __forceinline__ void store4(T *dst, float a, float b, float c, float d);
template <>
__device__ __forceinline__ void store4<float>(float *dst, float a, float b, float c, float d) {
  *reinterpret_cast<float4 *>(dst) =
      make_float4(cvt<float>(a), cvt<float>(b), cvt<float>(c), cvt<float>(d));
}
template <>
__device__ __forceinline__ void store4<uint16_t>(uint16_t *dst, float a, float b, float c,
                                                 float d) {
  uint2 u;
  u.x = (uint32_t)cvt<uint16_t>(a) | ((uint32_t)cvt<uint16_t>(b) << 16);
  u.y = (uint32_t)cvt<uint16_t>(c) | ((uint32_t)cvt<uint16_t>(d) << 16);
  *reinterpret_cast<uint2 *>(dst) = u;
}

template <class T, bool VEC>
__global__ void __launch_bounds__(256)
    k_prepare(const float *__restrict__ A, int64_t m, int64_t n, int64_t lda, T *__restrict__ X,
              int64_t ldx, T *__restrict__ Xt, int64_t ldxt, double *__restrict__ part) {
  __shared__ float t[64][65];
  const int c4 = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16
  const int64_t tr = (m + 63) / 64, tcn = (n + 63) / 64;
  double acc = 0.0, acc_d = 0.0;
  for (int64_t tile = blockIdx.x; tile < tr * tcn; tile += gridDim.x) {
    const int64_t r0 = (tile / tcn) * 64, c0 = (tile % tcn) * 64;
    const int64_t c = c0 + 4 * c4;
    float v[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = r0 + ty + 16 * i;
      const float *src = A + r * lda + c;
      if (r < m && VEC && c + 3 < n) {
        const float4 q = __ldcs(reinterpret_cast<const float4 *>(src));
        v[i][0] = q.x; v[i][1] = q.y; v[i][2] = q.z; v[i][3] = q.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[i][u] = (r < m && c + u < n) ? src[u] : 0.f;
      }
    }
    float sq = 0.f, sd = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        sq = fmaf(v[i][u], v[i][u], sq);
        sd = fmaf(v[i][u], widen<T>(cvt<T>(v[i][u])) - v[i][u], sd);  // difference exact
      }
    acc += (double)sq;
    acc_d += (double)sd;
    __syncthreads();  // previous tile's transposed reads are done
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int y = ty + 16 * i;
      const int64_t r = r0 + y;
#pragma unroll
      for (int u = 0; u < 4; ++u) t[y][4 * c4 + u] = v[i][u];
      if (r < m) {
        T *dst = X + r * ldx + c;
        if (c + 3 < n) {
          store4<T>(dst, v[i][0], v[i][1], v[i][2], v[i][3]);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (c + u < n) dst[u] = cvt<T>(v[i][u]);
        }
      }
    }
    __syncthreads();
    // transposed: thread -> output row cc = c0 + threadIdx.x / 4, 16 entries
    const int oc = threadIdx.x >> 2, seg = (threadIdx.x & 3) * 16;
    const int64_t cc = c0 + oc;
    if (cc < n) {
      T *dst = Xt + cc * ldxt + r0 + seg;
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        const int64_t r = r0 + seg + q;
        if (r + 3 < m) {
          store4<T>(dst + q, t[seg + q][oc], t[seg + q + 1][oc], t[seg + q + 2][oc],
                    t[seg + q + 3][oc]);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (r + u < m) dst[q + u] = cvt<T>(t[seg + q + u][oc]);
        }
      }
    }
  }
  // block sums in a fixed order
  __shared__ double ws[2][8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    acc_d += __shfl_xor_sync(0xffffffffu, acc_d, o);
  }
  if ((threadIdx.x & 31) == 0) {
    ws[0][threadIdx.x >> 5] = acc;
    ws[1][threadIdx.x >> 5] = acc_d;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, d = 0.0;
    for (int w = 0; w < 8; ++w) {
      s += ws[0][w];
      d += ws[1][w];
    }
    part[2 * blockIdx.x] = s;
    part[2 * blockIdx.x + 1] = d;
  }
}

// out[0] = sum of the even partials (||A||^2), out[1] = 2 x the odd ones.
__global__ void k_sum_partials_d(const double *__restrict__ part, int np, double *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0, d = 0.0;
    for (int i = 0; i < np; ++i) {
      s += part[2 * i];
      d += part[2 * i + 1];
    }
    out[0] = s;
    out[1] = 2.0 * d;
  }
}

// out (rows x cols, ld ldo) = in rounded to T (TF32-valued FP32 or BF16).
template <class T>
__global__ void k_round_copy(const float *__restrict__ in, int64_t rows, int64_t cols, int64_t ldi,
                             T *__restrict__ out, int64_t ldo) {
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const float *src = in + r * ldi;
    T *dst = out + r * ldo;
    for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) dst[c] = cvt<T>(src[c]);
  }
}

// ------------------------------------------------------------------ host
// 2-D tensor map over a row-major rows x cols matrix (leading dimension ld,
// elements) with a box of box_cols (128 bytes) x box_rows, 128 B swizzle.
bool make_map(CUtensorMap *map, const void *base, bool bf16, int64_t rows, int64_t cols,
              int64_t ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const int esz = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(kStageBytesK / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

int pad_to(int64_t x, int q) { return (int)((x + q - 1) / q * q); }

}  // namespace

int bn_for(int k) { return pad_to(k, 16); }

// Split count: smallest S in 1..4 whose unit count fills the SMs evenly.
int splits_for(int64_t M, int64_t K, bool bf16) {
  const int64_t tiles = (M + kTileM - 1) / kTileM;
  const int64_t kb = (K + kStageBytesK / (bf16 ? 2 : 4) - 1) / (kStageBytesK / (bf16 ? 2 : 4));
  const int sms = num_sms();
  int best = 1;
  double best_eff = 0;
  for (int S = 1; S <= 4; ++S) {
    const int64_t per = (kb + S - 1) / S;
    if ((S - 1) * per >= kb) continue;  // the last split would be empty
    const int64_t u = tiles * S;
    const double waves = (double)u / sms;
    const double eff = waves / (double)((u + sms - 1) / sms);
    if (eff > best_eff + 0.02) { best_eff = eff; best = S; }
  }
  return best;
}

int check(int64_t m, int64_t n, int64_t lda, int k, int prec, const float *A) {
  if (prec != AUNMF_TF32 && prec != AUNMF_BF16) return AUNMF_E_INVAL;
  if (k < 1 || k > AUNMF_K_MAX) return AUNMF_E_INVAL;
  if (m > 0x7fffffffLL || n > 0x7fffffffLL) return AUNMF_E_UNSUPPORTED;
  if (!encode_fn()) return AUNMF_E_UNSUPPORTED;
  (void)lda;
  (void)A;
  return AUNMF_OK;
}

size_t factor_elems(int64_t rows, int k) { return (size_t)2 * k * pad_to(rows, 8); }
int64_t copy_ld(int64_t cols) { return pad_to(cols, 8); }
size_t parts_elems(int64_t M, int k) { return (size_t)4 * M * k; }

cudaError_t launch_transpose_to(const float *in, int64_t rows, int64_t cols, int64_t ldi, void *out,
                                int64_t ldo, bool bf16, cudaStream_t s) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  int64_t tiles = ((rows + 31) / 32) * ((cols + 31) / 32);
  if (tiles > (int64_t)num_sms() * 64) tiles = (int64_t)num_sms() * 64;
  if (bf16)
    k_transpose_to<uint16_t><<<(unsigned)tiles, dim3(32, 8), 0, s>>>(in, rows, cols, ldi,
                                                                     (uint16_t *)out, ldo);
  else
    k_transpose_to<float><<<(unsigned)tiles, dim3(32, 8), 0, s>>>(in, rows, cols, ldi,
                                                                 (float *)out, ldo);
  g_launches += 1;
  return cudaGetLastError();
}

int prepare_blocks() { return num_sms() * 8; }

cudaError_t launch_prepare(const float *A, int64_t m, int64_t n, int64_t lda, void *X, int64_t ldx,
                           void *Xt, int64_t ldxt, bool bf16, double *part, double *norm2,
                           cudaStream_t s) {
  const int nb = prepare_blocks();
  const bool vec = (reinterpret_cast<uintptr_t>(A) % 16 == 0) && (lda % 4 == 0);
  if (bf16) {
    if (vec)
      k_prepare<uint16_t, true><<<nb, 256, 0, s>>>(A, m, n, lda, (uint16_t *)X, ldx,
                                                   (uint16_t *)Xt, ldxt, part);
    else
      k_prepare<uint16_t, false><<<nb, 256, 0, s>>>(A, m, n, lda, (uint16_t *)X, ldx,
                                                    (uint16_t *)Xt, ldxt, part);
  } else {
    if (vec)
      k_prepare<float, true><<<nb, 256, 0, s>>>(A, m, n, lda, (float *)X, ldx, (float *)Xt, ldxt,
                                                part);
    else
      k_prepare<float, false><<<nb, 256, 0, s>>>(A, m, n, lda, (float *)X, ldx, (float *)Xt, ldxt,
                                                 part);
  }
  k_sum_partials_d<<<1, 32, 0, s>>>(part, nb, norm2);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_split_transpose(const float *in, int64_t rows, int k, int64_t ldi, void *out,
                                   int64_t ldo, bool bf16, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  int64_t tiles = ((rows + 31) / 32) * ((k + 31) / 32);
  if (tiles > (int64_t)num_sms() * 64) tiles = (int64_t)num_sms() * 64;
  if (bf16)
    k_split_transpose<uint16_t><<<(unsigned)tiles, dim3(32, 8), 0, s>>>(in, rows, k, ldi,
                                                                        (uint16_t *)out, ldo);
  else
    k_split_transpose<float><<<(unsigned)tiles, dim3(32, 8), 0, s>>>(in, rows, k, ldi,
                                                                    (float *)out, ldo);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_round_copy(const float *A, int64_t m, int64_t n, int64_t lda, void *out,
                              int64_t ldo, bool bf16, cudaStream_t s) {
  int64_t nb = m < (int64_t)num_sms() * 16 ? m : (int64_t)num_sms() * 16;
  if (nb < 1) return cudaSuccess;
  if (bf16)
    k_round_copy<uint16_t><<<(unsigned)nb, 256, 0, s>>>(A, m, n, lda, (uint16_t *)out, ldo);
  else
    k_round_copy<float><<<(unsigned)nb, 256, 0, s>>>(A, m, n, lda, (float *)out, ldo);
  g_launches += 1;
  return cudaGetLastError();
}

bool fill_problem(GemmProblem *p, const void *X, int64_t M, int64_t K, int64_t ldx, const void *Y,
                  int k, int64_t ldy, bool split, bool bf16, float *parts, int S) {
  const int ny = split ? 2 * k : k;
  const int BN = bn_for(ny);
  if (BN > 256 || S < 1) return false;
  if (!make_map(&p->mapX, X, bf16, M, K, ldx, kTileM)) return false;
  if (!make_map(&p->mapY, Y, bf16, ny, K, ldy, BN)) return false;
  const int64_t bke = kStageBytesK / (bf16 ? 2 : 4);
  p->M = M;
  p->K = K;
  p->unit0 = 0;
  p->total_kb = (K + bke - 1) / bke;
  p->per_split = (p->total_kb + S - 1) / S;
  p->P = parts;
  p->k = k;
  p->ldc = k;
  p->BN = BN;
  p->S = S;
  p->pair = split ? 1 : 0;
  return true;
}

int64_t problem_units(const GemmProblem &p) { return ((p.M + kTileM - 1) / kTileM) * p.S; }

// Accumulator row width that a problem needs in shared memory: none for a
// pair problem (its <= 64 sums stay in registers); otherwise its MMA columns
// past the first 64 (kept in registers), rounded up to the 32-column drain
// group.
int acc_width(const GemmProblem &p) {
  if (p.pair && p.BN <= 128) return 0;
  const int w = ((p.BN + 31) & ~31) - 64;
  return w > 0 ? w : 0;
}
bool all_pair(const GemmProblem &p) { return p.pair && p.BN <= 128; }

// Shape of a launch whose problems have at most BNmax MMA columns and whose
// shared accumulator rows need at most accw floats.  The FP32 accumulator
// (256 x (accw | 1) floats, odd stride so that the 32 rows a warp touches
// fall in 32 banks) goes to shared memory when three pipeline stages still
// fit beside it; otherwise chunks are added into P in global memory
// (L2-resident), with longer chunks.  TMEM holds nbuf chunk accumulators of
// 2 x BNmax columns; the drain reads up to BN rounded up to 64 columns past
// the start of the last half, which must stay inside the allocation.
bool launch_shape(GemmLaunch *L, int BNmax, int accw, bool pairs, int64_t units, int nprob,
                  int *err) {
  L->units = units;
  L->nprob = nprob;
  L->BNmax = BNmax;
  const int wmax = (BNmax + 63) & ~63;
  L->nbuf = (3 * BNmax + wmax <= 512) ? 2 : 1;
  const int need = (2 * L->nbuf - 1) * BNmax + wmax;
  if (need > 512) return false;
  uint32_t cols = 32;
  while (cols < (uint32_t)need) cols <<= 1;
  L->tmem_cols = cols;
  const size_t sbytes = (size_t)(kTileM + BNmax) * kStageBytesK;
  const size_t budget = 225 * 1024 - 1024 - 256;
  const int ld = accw | 1;
  const size_t acc = (size_t)kTileM * ld * sizeof(float);
  L->regacc = pairs ? 1 : 0;
  if (accw == 0) {
    L->acc_ld = 0;
    L->nstages = (int)(budget / sbytes);
    L->chunk_kb = kChunkKBReg;
  } else if (acc + 3 * sbytes <= budget) {
    // the shared accumulator only with at least three pipeline stages beside
    // it: with two, each stage's TMA latency stalls the MMAs (k = 320, two
    // blocks of 160: 8.34 -> 6.11 ms per TF32 product on the L2 scratch path)
    L->acc_ld = ld;
    L->nstages = (int)((budget - acc) / sbytes);
    L->chunk_kb = kChunkKB;
  } else {
    L->acc_ld = 0;
    L->nstages = (int)(budget / sbytes);
    L->chunk_kb = kChunkKBGlobal;
  }
  if (L->nstages > 8) L->nstages = 8;
  // a single TMEM buffer stalls the MMAs for every drain: long chains
  if (L->nbuf == 1 && L->chunk_kb < kChunkKBLong) L->chunk_kb = kChunkKBLong;
  L->interleave = 0;
  L->scratch = nullptr;
  L->scr_cols = 0;
  L->err = err;
  L->wait_cycles = fault::wait_cycles();
  L->inject = fault::site() == AUNMF_INJECT_TC_WAIT ? 1 : 0;
  return L->nstages >= 2;
}

cudaError_t launch_kernel(const GemmProblem &one, const GemmProblem &two, const GemmProblem *group,
                          const GemmLaunch &L, bool bf16, cudaStream_t s) {
  const size_t sbytes = (size_t)(kTileM + L.BNmax) * kStageBytesK;
  const size_t smem = 1024 + (size_t)L.nstages * sbytes +
                      (size_t)kTileM * L.acc_ld * sizeof(float) + 256;
  const int grid = (int)(L.units < num_sms() ? L.units : num_sms());
  if (grid < 1) return cudaSuccess;
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, kThreads, smem, s>>>(one, two, group, L);
  };
  if (bf16) {
    if (L.regacc) go(k_gemm_tc<true, true, false>);
    else if (L.scratch) go(k_gemm_tc<true, false, true>);
    else go(k_gemm_tc<true, false, false>);
  } else {
    if (L.regacc) go(k_gemm_tc<false, true, false>);
    else if (L.scratch) go(k_gemm_tc<false, false, true>);
    else go(k_gemm_tc<false, false, false>);
  }
  g_launches += 1;
  return cudaGetLastError();
}

size_t scratch_elems() { return (size_t)num_sms() * kTileM * (kMaxBN - 64); }

// Above kMaxBN columns (unsplit factor, k <= 2 kMaxBN) the product runs as two
// problems over column blocks of C, [0, k0) and [k0, k), in one launch.
// Their units alternate, so the two CTAs that need the same tile of
// X ask for it at about the same time and the second read comes from L2.
cudaError_t launch_gemm(const void *X, int64_t M, int64_t K, int64_t ldx, const void *Y, int k,
                        int64_t ldy, bool split, bool bf16, float *parts, int S, float *scratch,
                        int *err, cudaStream_t s) {
  // two blocks of (about) equal width, which stream X at the same speed and
  // so stay close enough for the second read of each X tile to hit L2
  GemmProblem p[2];
  const int k0 = (!split && k > kMaxBN) ? pad_to((k + 1) / 2, 16) : k;
  if (k0 > kMaxBN || k - k0 > kMaxBN) return cudaErrorInvalidValue;
  if (!fill_problem(&p[0], X, M, K, ldx, Y, k0, ldy, split, bf16, parts, S))
    return cudaErrorInvalidValue;
  p[0].ldc = k;
  const int np = k0 < k ? 2 : 1;
  if (np == 2) {
    const char *Y1 = static_cast<const char *>(Y) + (size_t)k0 * ldy * (bf16 ? 2 : 4);
    if (!fill_problem(&p[1], X, M, K, ldx, Y1, k - k0, ldy, false, bf16, parts + k0, S))
      return cudaErrorInvalidValue;
    p[1].ldc = k;
  }
  const int BNmax = std::max(p[0].BN, p[np - 1].BN);
  const int accw = std::max(acc_width(p[0]), acc_width(p[np - 1]));
  GemmLaunch L;
  if (!launch_shape(&L, BNmax, accw, all_pair(p[0]), problem_units(p[0]) * np, 0, err))
    return cudaErrorInvalidValue;
  L.interleave = np == 2 ? 1 : 0;
  if (L.acc_ld == 0 && accw > 0 && scratch) {
    L.scratch = scratch;
    L.scr_cols = accw;
    L.chunk_kb = kChunkKBScratch;
  }
  return launch_kernel(p[0], p[np - 1], nullptr, L, bf16, s);
}

size_t problem_bytes() { return sizeof(GemmProblem); }

bool fill_group_problem(void *host_dst, const void *X, int64_t M, int64_t K, int64_t ldx,
                        const void *Y, int k, int64_t ldy, bool split, bool bf16, float *C,
                        int64_t unit0, int64_t *units, int *BN) {
  GemmProblem *p = reinterpret_cast<GemmProblem *>(host_dst);
  if (!fill_problem(p, X, M, K, ldx, Y, k, ldy, split, bf16, C, 1)) return false;
  p->unit0 = unit0;
  *units = problem_units(*p);
  *BN = p->BN;
  return true;
}

namespace {
bool group_shape(GemmLaunch *L, const void *host_first, int nprob, int64_t units, int BNmax,
                 int *err) {
  const GemmProblem *hp = reinterpret_cast<const GemmProblem *>(host_first);
  int accw = 0;
  bool pairs = true;
  for (int i = 0; i < nprob; ++i) {
    const int w = acc_width(hp[i]);
    accw = w > accw ? w : accw;
    pairs = pairs && all_pair(hp[i]);
  }
  return launch_shape(L, BNmax, accw, pairs, units, nprob, err);
}
}  // namespace

int group_max_stages(const void *host_first, int nprob, int64_t units, int BNmax) {
  GemmLaunch L;
  return group_shape(&L, host_first, nprob, units, BNmax, nullptr) ? L.nstages : 0;
}

cudaError_t launch_gemm_group(const void *dev_problems, const void *host_first, int nprob,
                              int64_t units, int BNmax, bool bf16, int *err, cudaStream_t s,
                              int nstages) {
  GemmLaunch L;
  if (!group_shape(&L, host_first, nprob, units, BNmax, err)) return cudaErrorInvalidValue;
  if (nstages >= 2 && nstages < L.nstages) L.nstages = nstages;
  const GemmProblem &h0 = *reinterpret_cast<const GemmProblem *>(host_first);
  return launch_kernel(h0, h0, reinterpret_cast<const GemmProblem *>(dev_problems), L, bf16, s);
}

cudaError_t launch_sum_splits(const float *parts, int S, int64_t len, float *P, cudaStream_t s) {
  int64_t nb = (len + 255) / 256;
  if (nb > (int64_t)num_sms() * 16) nb = (int64_t)num_sms() * 16;
  if (nb < 1) nb = 1;
  k_sum_splits<<<(unsigned)nb, 256, 0, s>>>(parts, S, len, P);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace aunmf
