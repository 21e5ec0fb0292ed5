// Tensor-core (tcgen05 / TMEM / TMA) mu-mode products for the split-precision
// dtypes.  See tc.cuh for the data flow.
//
// One pass computes D[m, i] = sum_k X[k, m] L[i, k] for the unfolding X (n x M2,
// column-major, the contracted mode contiguous) of the current tensor: M = 128
// rows of X^T per tile, N = one N tile of L's rows (all n_pad of them when
// n_pad <= 256, else ceil(n_pad / 256) equal tiles), K = n in 128-byte chunks.
// Both operands are K-major in shared memory with the 128-byte swizzle, which
// is what TMA writes for a box whose inner extent is 128 bytes.
//
// Split products (FP32 accumulation in TMEM):
//   TF32    D = hi(X) hi(L)                         one plane per operand
//   TF32X3  D = hi hi + hi lo + lo hi, hi/lo tf32   two planes per operand
//   BF16X3  D = hi hi + hi lo + lo hi, hi/lo bf16   two planes per operand
//
// CTA roles (192 threads): warp 0 issues TMA loads, warp 1 owns TMEM and
// issues the MMAs (one elected lane), warps 2..5 drain TMEM (warp w reads TMEM
// lanes 32 (w % 4) .. +31) and store.  Two TMEM accumulators alternate so the
// epilogue of one tile overlaps the MMAs of the next.  Every mbarrier wait is
// bounded (about one second); a wait that gives up records a code in a device
// status word and the CTA unwinds, still freeing its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>

#include "devmem.hpp"
#include "tc.cuh"
#include "pdl.cuh"
#include "tcgen05.cuh"

namespace phiks {

namespace {

thread_local std::string g_tc_err;

using namespace ptx;
constexpr int kTcEpiWarps = 16;  // four per TMEM lane quarter, each a quarter of the columns
constexpr int NTHREADS = 64 + 32 * kTcEpiWarps;

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Split of one FP32 value into the dtype's planes, in FP32 arithmetic
// (x - hi is exact in FP32 for both hi formats).
template <int KIND, int NP>
__device__ __forceinline__ void split_store_f(void* p0, void* p1, int64_t idx, float x) {
  if (KIND == 0) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    ((__nv_bfloat16*)p0)[idx] = hi;
    if (NP == 2) ((__nv_bfloat16*)p1)[idx] = __float2bfloat16_rn(x - __bfloat162float(hi));
  } else {
    const float hi = tf32_rna(x);
    ((float*)p0)[idx] = hi;
    if (NP == 2) ((float*)p1)[idx] = tf32_rna(x - hi);
  }
}

// Split of one FP64 value (inputs and the small exponentials): hi from the
// double, lo from the exact double residual.
template <int KIND, int NP>
__device__ __forceinline__ void split_store(void* p0, void* p1, int64_t idx, double x) {
  if (KIND == 0) {
    const __nv_bfloat16 hi = __double2bfloat16(x);
    ((__nv_bfloat16*)p0)[idx] = hi;
    if (NP == 2) ((__nv_bfloat16*)p1)[idx] = __double2bfloat16(x - (double)__bfloat162float(hi));
  } else {
    const float hi = tf32_rna((float)x);
    ((float*)p0)[idx] = hi;
    if (NP == 2) ((float*)p1)[idx] = tf32_rna((float)(x - (double)hi));
  }
}

// ---------------------------------------------------------------------------
struct GemmParams {
  int n;          // contraction length and output columns
  int n_pad;      // n rounded up to 16
  int ntile;      // MMA N: rows of L per tile (multiple of 16, <= 256)
  int n_ntiles;   // N tiles per row block
  int64_t M2;     // N / n: fibres of one tensor
  int64_t rows;   // fibres of the batch (tensor b owns rows b M2 .. b M2 + M2 - 1)
  int64_t N;      // elements of one tensor
  int nk;         // 128-byte K chunks
  int num_tiles;  // ceil(rows / 128) * n_ntiles
  int stages;
  int tmem_cols;
  int last;       // 0: write planes for the next pass; 1: write FP32 results to out0
  int mixed;      // tensors with their own matrices: every tile within one tensor
  int64_t tpt;    // mixed: row tiles per tensor, ceil(M2 / 128) (the last one partial)
  int shared_a;   // mixed, first pass: every tensor's input is tensor 0's planes
  void* out0;
  void* out1;
  int* status;
  uint32_t b_bytes;  // resident form: shared memory of B (every K chunk and plane)
};

// TMA maps of the B planes (hi, lo) of tensor b's matrix (entry 0 unless mixed).
struct TcMapsB {
  CUtensorMap b[kTcMaxBatch][2];
};

// First fibre (row of the batch) of row tile rt, and its tensor: mixed
// batches tile every tensor on its own (rows of a partial last tile past the
// tensor are computed from whatever the copy brings and not stored).
__device__ __forceinline__ int64_t tc_tile_row0(const GemmParams& P, int64_t rt, int* b) {
  if (P.mixed) {
    const int64_t bb = rt / P.tpt;
    *b = (int)bb;
    return bb * P.M2 + (rt - bb * P.tpt) * BM;
  }
  *b = 0;
  return rt * BM;
}

template <int KIND, int NP>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA0, const __grid_constant__ CUtensorMap mapA1,
                   const __grid_constant__ TcMapsB mapsB, const __grid_constant__ GemmParams P) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = P.stages;
  const uint32_t a_plane = BM * 128;                 // bytes of one A plane per stage
  const uint32_t b_plane = (uint32_t)P.ntile * 128;  // bytes of one B plane per stage
  const uint32_t stage_bytes = NP * (a_plane + b_plane);
  uint64_t* full = (uint64_t*)(smem + (size_t)S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint64_t* mdone = tempty + 2;  // the MMA warp's issued MMAs finished (failure path)
  uint32_t* tmem_slot = (uint32_t*)(mdone + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kTcEpiWarps * 32);
    }
    mbar_init(mdone, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(P.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  pdl_wait();  // operand planes come from the kernels before

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < P.num_tiles && ok; t += gridDim.x) {
        int mi = 0;
        int m0 = (int)tc_tile_row0(P, t / P.n_ntiles, &mi);
        if (P.shared_a) m0 -= (int)(mi * P.M2);  // the one split input
        const int r0 = (t % P.n_ntiles) * P.ntile;
        const CUtensorMap* mapB0 = &mapsB.b[mi][0];
        const CUtensorMap* mapB1 = &mapsB.b[mi][1];
        for (int kc = 0; kc < P.nk && ok; ++kc) {
          if (!mbar_wait(&empty[s], ph ^ 1, P.status, 1)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + (size_t)s * stage_bytes;
          mbar_arrive_expect_tx(&full[s], stage_bytes);
          const int x = kc * (128 / (KIND == 0 ? 2 : 4));
          tma_load_2d(st, &mapA0, &full[s], x, m0);
          if (NP == 2) tma_load_2d(st + a_plane, &mapA1, &full[s], x, m0);
          tma_load_2d(st + NP * a_plane, mapB0, &full[s], x, r0);
          if (NP == 2) tma_load_2d(st + NP * a_plane + b_plane, mapB1, &full[s], x, r0);
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      // let the copies already issued land before the CTA may leave (also
      // after another role gave up)
      for (int k = 0; k < S; ++k) {
        if (--s < 0) {
          s = S - 1;
          ph ^= 1;
        }
        (void)mbar_drain(&full[s], ph);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_make(KIND == 0 ? 1 : 2, P.ntile);
      int s = 0;
      uint32_t ph = 0;
      int buf = 0;
      uint32_t aph = 0;
      bool ok = true, any = false;
      for (int t = blockIdx.x; t < P.num_tiles && ok; t += gridDim.x) {
        if (!mbar_wait(&tempty[buf], aph ^ 1, P.status, 2)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dtm = tmem_base + (uint32_t)(buf * P.ntile);
        for (int kc = 0; kc < P.nk; ++kc) {
          if (!mbar_wait(&full[s], ph, P.status, 3)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
          // descriptors of the stage's planes at K step 0; a K step moves the
          // start address field only (16-byte units, no carry out of it)
          const uint64_t da0 = sdesc_sw128(st), da1 = sdesc_sw128(st + a_plane);
          const uint64_t db0 = sdesc_sw128(st + NP * a_plane), db1 = sdesc_sw128(st + NP * a_plane + b_plane);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // 4 x 32-byte K steps per 128-byte chunk
            const uint64_t off = (uint64_t)((kk * 32) >> 4);
            const uint32_t acc = (kc | kk) != 0;
            umma<KIND>(dtm, da0 + off, db0 + off, idesc, acc);
            if (NP == 2) {
              umma<KIND>(dtm, da0 + off, db1 + off, idesc, 1);
              umma<KIND>(dtm, da1 + off, db0 + off, idesc, 1);
            }
          }
          any = true;
          umma_commit(&empty[s]);
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
        if (!ok) break;
        umma_commit(&tfull[buf]);
        if (++buf == 2) {
          buf = 0;
          aph ^= 1;
        }
      }
      if (!ok && any) {  // given up: the MMAs already issued finish before TMEM is freed
        umma_commit(mdone);
        (void)mbar_drain(mdone, 0);
      }
    }
  } else {
    // ---------------- epilogue: warps 2 .. 2 + kTcEpiWarps - 1; the four
    // warps of a lane quarter take interleaved 16-column chunks
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int grp = (warp - 2) >> 2;
    constexpr int GROUPS = kTcEpiWarps / 4;
    const int row = q * 32 + lane;
    int buf = 0;
    uint32_t aph = 0;
    for (int t = blockIdx.x; t < P.num_tiles; t += gridDim.x) {
      if (!mbar_wait(&tfull[buf], aph, P.status, 4)) break;
      tc_fence_after();
      int tb = 0;
      const int64_t colb = tc_tile_row0(P, t / P.n_ntiles, &tb) + row;  // fibre of the batch
      const int r0 = (t % P.n_ntiles) * P.ntile;
      const bool valid = P.mixed ? (colb - (int64_t)tb * P.M2 < P.M2) : (colb < P.rows);
      const int64_t bt = valid ? (P.mixed ? tb : colb / P.M2) : 0;
      const int64_t col = colb - bt * P.M2 + bt * P.N;  // tensor b's elements start at b N
      const int cend = P.n - r0 < P.ntile ? P.n - r0 : P.ntile;
      const uint32_t tl = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * P.ntile);
      if (P.ntile <= 32 * GROUPS) {
        // at most two 16-column chunks per warp: both in registers, then the
        // TMEM set is released before the stores (a later tile's MMAs run
        // under them)
        uint32_t u[2][16];
        const int c0 = 16 * grp, c1 = c0 + 16 * GROUPS;
        if (c0 < cend) tmem_ld16_nowait(tl + (uint32_t)c0, u[0]);
        if (c1 < cend) tmem_ld16_nowait(tl + (uint32_t)c1, u[1]);
        tmem_wait_ld();
        tc_fence_before();
        mbar_arrive(&tempty[buf]);
        if (valid) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int cb = h ? c1 : c0;
            if (cb >= cend) break;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int i = r0 + cb + j;
              if (i >= P.n) break;
              const int64_t idx = col + P.M2 * (int64_t)i;
              const float x = __uint_as_float(u[h][j]);
              if (!P.last) split_store_f<KIND, NP>(P.out0, P.out1, idx, x);
              else ((float*)P.out0)[idx] = x;
            }
          }
        }
      } else {
        for (int c0 = 16 * grp; c0 < cend; c0 += 16 * GROUPS) {
          float v[16];
          tmem_ld16(tl + (uint32_t)c0, v);
          if (!valid) continue;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int i = r0 + c0 + j;
            if (i >= P.n) break;
            const int64_t idx = col + P.M2 * (int64_t)i;
            if (!P.last) split_store_f<KIND, NP>(P.out0, P.out1, idx, v[j]);
            else ((float*)P.out0)[idx] = v[j];
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[buf]);
      }
      if (++buf == 2) {
        buf = 0;
        aph ^= 1;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(P.tmem_cols)
                 : "memory");
  }
}

// Resident form (one N tile per row block: a tensor's tiles all use the
// whole of its matrix): a CTA takes a contiguous range of tiles and keeps its
// tensor's B planes, every K chunk, in shared memory (loaded once per tensor,
// after the MMAs on the previous tensor's finished); only the A planes stream
// through the S stages.  Roles, TMEM sets and the epilogue as in
// tc_gemm_kernel.
template <int KIND, int NP>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_res_kernel(const __grid_constant__ CUtensorMap mapA0, const __grid_constant__ CUtensorMap mapA1,
                       const __grid_constant__ TcMapsB mapsB, const __grid_constant__ GemmParams P) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = P.stages;
  const uint32_t a_plane = BM * 128;                 // bytes of one A plane per stage
  const uint32_t b_plane = (uint32_t)P.ntile * 128;  // bytes of one B plane per K chunk
  const uint32_t stage_bytes = NP * a_plane;
  uint8_t* const sB = smem;                // [kc][plane]
  uint8_t* const sA = smem + P.b_bytes;    // S stages of NP A planes
  uint64_t* full = (uint64_t*)(sA + (size_t)S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint64_t* mdone = tempty + 2;  // the MMA warp's issued MMAs finished (failure path)
  uint64_t* fullB = mdone + 1;   // the current tensor's B planes landed
  uint64_t* emptyB = fullB + 1;  // the MMAs on the previous tensor's B planes finished
  uint32_t* tmem_slot = (uint32_t*)(emptyB + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kTcEpiWarps * 32);
    }
    mbar_init(mdone, 1);
    mbar_init(fullB, 1);
    mbar_init(emptyB, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(P.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  pdl_wait();  // operand planes come from the kernels before

  // this CTA's tiles: a contiguous range of the row tiles
  const int G = (int)gridDim.x, cta = (int)blockIdx.x;
  const int tbase = P.num_tiles / G, trem = P.num_tiles % G;
  const int t_begin = cta * tbase + min(cta, trem);
  const int t_end = t_begin + tbase + (cta < trem ? 1 : 0);

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0, eph = 0;
      int nB = 0, prev_tb = -1;
      bool ok = true;
      for (int t = t_begin; t < t_end && ok; ++t) {
        int mi = 0;
        int m0 = (int)tc_tile_row0(P, t, &mi);
        if (mi != prev_tb) {  // this tensor's B planes, every K chunk
          if (prev_tb >= 0) {
            if (!mbar_wait(emptyB, eph, P.status, 1)) break;
            eph ^= 1;
          }
          mbar_arrive_expect_tx(fullB, (uint32_t)P.nk * NP * b_plane);
          for (int kc = 0; kc < P.nk; ++kc) {
            const int x = kc * (128 / (KIND == 0 ? 2 : 4));
            tma_load_2d(sB + (size_t)(kc * NP) * b_plane, &mapsB.b[mi][0], fullB, x, 0);
            if (NP == 2) tma_load_2d(sB + (size_t)(kc * NP + 1) * b_plane, &mapsB.b[mi][1], fullB, x, 0);
          }
          ++nB;
          prev_tb = mi;
        }
        if (P.shared_a) m0 -= (int)(mi * P.M2);  // the one split input
        for (int kc = 0; kc < P.nk && ok; ++kc) {
          if (!mbar_wait(&empty[s], ph ^ 1, P.status, 1)) {
            ok = false;
            break;
          }
          uint8_t* st = sA + (size_t)s * stage_bytes;
          mbar_arrive_expect_tx(&full[s], stage_bytes);
          const int x = kc * (128 / (KIND == 0 ? 2 : 4));
          tma_load_2d(st, &mapA0, &full[s], x, m0);
          if (NP == 2) tma_load_2d(st + a_plane, &mapA1, &full[s], x, m0);
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      // let the copies already issued land before the CTA may leave (also
      // after another role gave up)
      for (int k = 0; k < S; ++k) {
        if (--s < 0) {
          s = S - 1;
          ph ^= 1;
        }
        (void)mbar_drain(&full[s], ph);
      }
      if (nB) (void)mbar_drain(fullB, (uint32_t)(nB - 1) & 1u);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_make(KIND == 0 ? 1 : 2, P.ntile);
      int s = 0;
      uint32_t ph = 0, bpar = 0;
      int buf = 0, prev_tb = -1;
      uint32_t aph = 0;
      bool ok = true, any = false;
      const uint32_t sb = smem_u32(sB);
      for (int t = t_begin; t < t_end && ok; ++t) {
        int mi = 0;
        (void)tc_tile_row0(P, t, &mi);
        if (!mbar_wait(&tempty[buf], aph ^ 1, P.status, 2)) {
          ok = false;
          break;
        }
        if (mi != prev_tb) {
          if (!mbar_wait(fullB, bpar, P.status, 3)) {
            ok = false;
            break;
          }
          bpar ^= 1;
          prev_tb = mi;
        }
        tc_fence_after();
        const uint32_t dtm = tmem_base + (uint32_t)(buf * P.ntile);
        for (int kc = 0; kc < P.nk; ++kc) {
          if (!mbar_wait(&full[s], ph, P.status, 3)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(sA + (size_t)s * stage_bytes);
          const uint64_t da0 = sdesc_sw128(st), da1 = sdesc_sw128(st + a_plane);
          const uint64_t db0 = sdesc_sw128(sb + (uint32_t)(kc * NP) * b_plane);
          const uint64_t db1 = sdesc_sw128(sb + (uint32_t)(kc * NP + (NP == 2 ? 1 : 0)) * b_plane);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // 4 x 32-byte K steps per 128-byte chunk
            const uint64_t off = (uint64_t)((kk * 32) >> 4);
            const uint32_t acc = (kc | kk) != 0;
            umma<KIND>(dtm, da0 + off, db0 + off, idesc, acc);
            if (NP == 2) {
              umma<KIND>(dtm, da0 + off, db1 + off, idesc, 1);
              umma<KIND>(dtm, da1 + off, db0 + off, idesc, 1);
            }
          }
          any = true;
          umma_commit(&empty[s]);
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
        if (!ok) break;
        umma_commit(&tfull[buf]);
        // the last tile on these B planes: they may be replaced
        if (t + 1 < t_end) {
          int mn = 0;
          (void)tc_tile_row0(P, t + 1, &mn);
          if (mn != mi) umma_commit(emptyB);
        }
        if (++buf == 2) {
          buf = 0;
          aph ^= 1;
        }
      }
      if (!ok && any) {  // given up: the MMAs already issued finish before TMEM is freed
        umma_commit(mdone);
        (void)mbar_drain(mdone, 0);
      }
    }
  } else {
    // ---------------- epilogue (as in tc_gemm_kernel)
    const int q = warp & 3;
    const int grp = (warp - 2) >> 2;
    constexpr int GROUPS = kTcEpiWarps / 4;
    const int row = q * 32 + lane;
    int buf = 0;
    uint32_t aph = 0;
    for (int t = t_begin; t < t_end; ++t) {
      if (!mbar_wait(&tfull[buf], aph, P.status, 4)) break;
      tc_fence_after();
      int tb = 0;
      const int64_t colb = tc_tile_row0(P, t, &tb) + row;  // fibre of the batch
      const bool valid = P.mixed ? (colb - (int64_t)tb * P.M2 < P.M2) : (colb < P.rows);
      const int64_t bt = valid ? (P.mixed ? tb : colb / P.M2) : 0;
      const int64_t col = colb - bt * P.M2 + bt * P.N;  // tensor b's elements start at b N
      const int cend = P.n < P.ntile ? P.n : P.ntile;
      const uint32_t tl = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * P.ntile);
      if (P.ntile <= 32 * GROUPS) {
        uint32_t u[2][16];
        const int c0 = 16 * grp, c1 = c0 + 16 * GROUPS;
        if (c0 < cend) tmem_ld16_nowait(tl + (uint32_t)c0, u[0]);
        if (c1 < cend) tmem_ld16_nowait(tl + (uint32_t)c1, u[1]);
        tmem_wait_ld();
        tc_fence_before();
        mbar_arrive(&tempty[buf]);
        if (valid) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int cb = h ? c1 : c0;
            if (cb >= cend) break;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int i = cb + j;
              if (i >= P.n) break;
              const int64_t idx = col + P.M2 * (int64_t)i;
              const float x = __uint_as_float(u[h][j]);
              if (!P.last) split_store_f<KIND, NP>(P.out0, P.out1, idx, x);
              else ((float*)P.out0)[idx] = x;
            }
          }
        }
      } else {
        for (int c0 = 16 * grp; c0 < cend; c0 += 16 * GROUPS) {
          float v[16];
          tmem_ld16(tl + (uint32_t)c0, v);
          if (!valid) continue;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int i = c0 + j;
            if (i >= P.n) break;
            const int64_t idx = col + P.M2 * (int64_t)i;
            if (!P.last) split_store_f<KIND, NP>(P.out0, P.out1, idx, v[j]);
            else ((float*)P.out0)[idx] = v[j];
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[buf]);
      }
      if (++buf == 2) {
        buf = 0;
        aph ^= 1;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(P.tmem_cols)
                 : "memory");
  }
}

// x = sum_m coef_m src_m (float or double sources) split into planes.  The
// combination is formed in FP64 only when it has more than one term or a
// coefficient other than one; the split itself runs in FP32 (the planes carry
// at most 22 significant bits, FP32 holds 24).
// Grid rows of a split launch: rows below ntensor are the batch's tensors
// (split into planes, and their FP64 values also stored where store[y] is not
// null); the rest evaluate their combination into store[y] only (float when
// bit y of store_f32 is set).
struct TcSplitJobs {
  Combo c[kTcMaxBatch + kTcMaxSide];
  void* store[kTcMaxBatch + kTcMaxSide];
  unsigned store_f32;
  int ntensor;
  // each coefficient as chi + clo (floats), for combinations of float sources
  float chi[kTcMaxBatch + kTcMaxSide][kMaxSrc], clo[kTcMaxBatch + kTcMaxSide][kMaxSrc];
};

// Knuth's two-sum: s + e = a + b exactly.
__device__ __forceinline__ void tc_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <int KIND, int NP>
__global__ void tc_split_kernel(const __grid_constant__ TcSplitJobs jb, int64_t N, void* p0, void* p1) {
  pdl_wait();
  const int y = blockIdx.y;
  const Combo& in = jb.c[y];
  void* const xout = jb.store[y];
  const bool out32 = (jb.store_f32 >> y) & 1;
  const bool split = y < jb.ntensor;
  const int64_t off = (int64_t)y * N;  // tensor b's elements in the planes
  const bool plain = in.nsrc == 1 && in.coef[0] == 1.0 && !xout;
  const bool f32 = in.f32mask & 1;
  // all sources float (quadrature inputs and sums of FP32 Tucker results):
  // compensated FP32 as in the combination kernels (error-free products,
  // two-sum, about 44 bits), off GB300's slow FP64 pipe; a source in FP64
  // (the squaring's accumulators, eq. (simul) / eq. (comb)) keeps the
  // combination in FP64
  const bool allf32 = in.nsrc > 0 && (unsigned)in.f32mask == (1u << in.nsrc) - 1;
  const float* const chi = jb.chi[y];
  const float* const clo = jb.clo[y];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    float xf;
    if (plain) {
      xf = f32 ? ((const float*)in.src[0])[idx] : (float)in.src[0][idx];
    } else if (allf32) {
      float hi = 0.f, lo = 0.f;
#pragma unroll 4
      for (int m = 0; m < in.nsrc; ++m) {
        const float v = __ldg((const float*)in.src[m] + idx);
        const float p = chi[m] * v;
        const float e = fmaf(chi[m], v, -p) + clo[m] * v;
        float s, t;
        tc_two_sum(hi, p, s, t);
        hi = s;
        lo += t + e;
      }
      xf = hi + lo;
      if (xout) {
        if (out32) ((float*)xout)[idx] = xf;
        else ((double*)xout)[idx] = (double)hi + (double)lo;
      }
    } else {
      double x = 0.0;
#pragma unroll 4
      for (int m = 0; m < in.nsrc; ++m) {
        const double v =
            ((in.f32mask >> m) & 1) ? (double)__ldg((const float*)in.src[m] + idx) : __ldg(in.src[m] + idx);
        x = fma(in.coef[m], v, x);
      }
      if (xout) {
        if (out32) ((float*)xout)[idx] = (float)x;
        else ((double*)xout)[idx] = x;
      }
      xf = (float)x;
    }
    if (split) split_store_f<KIND, NP>(p0, p1, off + idx, xf);
  }
}

// Fills the float splits of every row's coefficients.
void tc_split_coefs(TcSplitJobs& jb, int rows) {
  for (int y = 0; y < rows; ++y)
    for (int m = 0; m < jb.c[y].nsrc && m < kMaxSrc; ++m) {
      jb.chi[y][m] = (float)jb.c[y].coef[m];
      jb.clo[y][m] = (float)(jb.c[y].coef[m] - (double)jb.chi[y][m]);
    }
}

// B planes of an FP64 column-major n x n matrix: plane[i * n_pad + k] from L[i, k].
template <int KIND, int NP>
__global__ void tc_prep_b_kernel(const double* L, int n, int n_pad, void* p0, void* p1) {
  pdl_wait();
  const int64_t tot = (int64_t)n_pad * n_pad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n_pad), k = (int)(e % n_pad);
    const double x = (i < n && k < n) ? L[i + (int64_t)n * k] : 0.0;
    split_store<KIND, NP>(p0, p1, e, x);
  }
}

// The same for up to kPrepBatch matrices, one per grid row.
constexpr int kPrepBatch = 32;
struct TcPrepBatch {
  const double* L[kPrepBatch];
  int n[kPrepBatch];
  void* p0[kPrepBatch];
  void* p1[kPrepBatch];
};

template <int KIND, int NP>
__global__ void tc_prep_b_batch_kernel(const __grid_constant__ TcPrepBatch pb) {
  pdl_wait();
  const int y = blockIdx.y;
  const double* L = pb.L[y];
  const int n = pb.n[y];
  const int n_pad = (n + 15) / 16 * 16;
  const int64_t tot = (int64_t)n_pad * n_pad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n_pad), k = (int)(e % n_pad);
    const double x = (i < n && k < n) ? L[i + (int64_t)n * k] : 0.0;
    split_store<KIND, NP>(pb.p0[y], pb.p1[y], e, x);
  }
}

int planes_of(int dtype) { return dtype == PHIKS_TF32 ? 1 : 2; }
int elt_of(int dtype) { return dtype == PHIKS_BF16X3 ? 2 : 4; }
int pad16(int n) { return (n + 15) / 16 * 16; }

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                              CUtensorMapFloatOOBfill);

EncodeFn g_encode = nullptr;

bool get_encode() {
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  g_encode = (EncodeFn)fn;
  return true;
}

// 2D map over a row-major (rows x inner) array, box {128 bytes of inner, box_rows}.
bool make_map(CUtensorMap* m, int dtype, const void* base, uint64_t inner, uint64_t rows,
              uint32_t box_rows) {
  const int elt = elt_of(dtype);
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * (uint64_t)elt};
  cuuint32_t box[2] = {(cuuint32_t)(128 / elt), box_rows};
  cuuint32_t es[2] = {1, 1};
  CUtensorMapDataType t =
      dtype == PHIKS_BF16X3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = g_encode(m, t, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

struct TcState {
  int dtype = 0;
  int d = 0;
  int64_t n[PHIKS_MAX_D] = {0};
  int64_t N = 0;
  int* status = nullptr;  // device
  uint8_t* ws = nullptr;
  int batch = 0;     // tensors the bound workspace holds
  int last_res = 1;  // plane set holding the last call's results
  int smem_optin = 0;
  int sms = 0;          // streaming multiprocessors of the device
  int ntiles_mult = 0;  // tuned: N tiles per pass, times the minimum (0: by size)
  // encoded tensor maps by (address, inner extent, rows, box rows): encoding
  // costs microseconds of host time, a lookup does not
  std::map<std::tuple<const void*, uint64_t, uint64_t, uint32_t>, CUtensorMap> maps;
};

namespace {

bool cached_map(TcState* s, CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows,
                uint32_t box_rows) {
  auto key = std::make_tuple(base, inner, rows, box_rows);
  auto it = s->maps.find(key);
  if (it != s->maps.end()) {
    *m = it->second;
    return true;
  }
  if (!make_map(m, s->dtype, base, inner, rows, box_rows)) return false;
  if (s->maps.size() > 4096) s->maps.clear();
  s->maps.emplace(key, *m);
  return true;
}

}  // namespace

size_t tc_workspace_bytes(int64_t N, int batch) {
  // two plane sets of up to 2 planes x 4 bytes for `batch` tensors, each
  // rounded to 1 KiB
  const size_t plane = ((size_t)batch * N * 4 + 1023) / 1024 * 1024;
  return 4 * plane + 1024;
}

namespace {
// Whether two input combinations are the same tensors with the same weights.
bool same_combo(const Combo& a, const Combo& b) {
  if (a.nsrc != b.nsrc || a.f32mask != b.f32mask) return false;
  for (int m = 0; m < a.nsrc; ++m)
    if (a.src[m] != b.src[m] || a.coef[m] != b.coef[m]) return false;
  return true;
}
}  // namespace

bool tc_mixed_ok(const TcState* s) {
  (void)s;  // every shape: mixed batches tile each tensor on its own
  return true;
}

phiks_status tc_create(TcState** out, int dtype, int d, const int64_t* n, int64_t N) {
  *out = nullptr;
  for (int mu = 0; mu < d; ++mu) {
    if (n[mu] > kTcMaxN) {
      g_tc_err = "tensor-core path supports n_mu <= 1024";
      return PHIKS_ERR_UNSUPPORTED;
    }
    const int elt = elt_of(dtype);
    if ((n[mu] * elt) % 16 != 0) {
      g_tc_err = "tensor-core path needs n_mu * element size to be a multiple of 16 bytes";
      return PHIKS_ERR_UNSUPPORTED;
    }
  }
  if (!get_encode()) {
    g_tc_err = "cuTensorMapEncodeTiled is not available";
    return PHIKS_ERR_UNSUPPORTED;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess || prop.major < 10) {
    g_tc_err = "tensor-core path needs an sm_100-class device";
    return PHIKS_ERR_UNSUPPORTED;
  }
  TcState* s = new TcState;
  s->dtype = dtype;
  s->d = d;
  for (int mu = 0; mu < d; ++mu) s->n[mu] = n[mu];
  s->N = N;
  s->smem_optin = (int)prop.sharedMemPerBlockOptin;
  s->sms = prop.multiProcessorCount;
  if (dev_malloc((void**)&s->status, sizeof(int)) != cudaSuccess ||
      cudaMemset(s->status, 0, sizeof(int)) != cudaSuccess) {
    dev_free(s->status);
    delete s;
    g_tc_err = "status word allocation failed";
    return PHIKS_ERR_OOM;
  }
  *out = s;
  return PHIKS_OK;
}

void tc_destroy(TcState* s) {
  if (!s) return;
  dev_free(s->status);
  delete s;
}

const char* tc_last_error() { return g_tc_err.c_str(); }

void tc_bind_workspace(TcState* s, void* ws, int batch) {
  s->ws = (uint8_t*)ws;
  s->batch = batch;
}

size_t tc_bplanes_bytes(int dtype, int n) {
  const size_t p = (size_t)pad16(n) * pad16(n) * elt_of(dtype);
  return planes_of(dtype) * ((p + 1023) / 1024 * 1024);
}

cudaError_t tc_prepare_b(int dtype, const double* L, int n, void* dst, cudaStream_t st) {
  const int np = pad16(n);
  const size_t p = ((size_t)np * np * elt_of(dtype) + 1023) / 1024 * 1024;
  uint8_t* p0 = (uint8_t*)dst;
  uint8_t* p1 = p0 + p;
  const int64_t tot = (int64_t)np * np;
  const int grid = (int)std::min<int64_t>((tot + 255) / 256, 1024);
  count_launch();
  void* none = nullptr;
  switch (dtype) {
    case PHIKS_BF16X3: return launch_pdl(tc_prep_b_kernel<0, 2>, dim3(grid), dim3(256), 0, st, L, n, np, p0, p1);
    case PHIKS_TF32X3: return launch_pdl(tc_prep_b_kernel<1, 2>, dim3(grid), dim3(256), 0, st, L, n, np, p0, p1);
    default: return launch_pdl(tc_prep_b_kernel<1, 1>, dim3(grid), dim3(256), 0, st, L, n, np, p0, none);
  }
}

cudaError_t tc_prepare_b_many(int dtype, int count, const double* const* L, const int* n, void* const* dst,
                              cudaStream_t st) {
  for (int k0 = 0; k0 < count; k0 += kPrepBatch) {
    TcPrepBatch pb;
    std::memset(&pb, 0, sizeof pb);
    const int cnt = std::min(kPrepBatch, count - k0);
    int64_t tot = 0;
    for (int k = 0; k < cnt; ++k) {
      const int np = pad16(n[k0 + k]);
      const size_t p = ((size_t)np * np * elt_of(dtype) + 1023) / 1024 * 1024;
      pb.L[k] = L[k0 + k];
      pb.n[k] = n[k0 + k];
      pb.p0[k] = dst[k0 + k];
      pb.p1[k] = (uint8_t*)dst[k0 + k] + p;
      tot = std::max<int64_t>(tot, (int64_t)np * np);
    }
    const int gx = (int)std::min<int64_t>((tot + 255) / 256, 1024);
    count_launch();
    cudaError_t e;
    switch (dtype) {
      case PHIKS_BF16X3: e = launch_pdl(tc_prep_b_batch_kernel<0, 2>, dim3(gx, cnt), dim3(256), 0, st, pb); break;
      case PHIKS_TF32X3: e = launch_pdl(tc_prep_b_batch_kernel<1, 2>, dim3(gx, cnt), dim3(256), 0, st, pb); break;
      default: e = launch_pdl(tc_prep_b_batch_kernel<1, 1>, dim3(gx, cnt), dim3(256), 0, st, pb); break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {

template <int KIND, int NP>
cudaError_t run_gemm(TcState* s, const CUtensorMap* mA, const TcMapsB& mB, GemmParams& P,
                     cudaStream_t st) {
  {  // resident form: one N tile, B (every K chunk) and at least two A stages fit
    const size_t extra = 1024 + 64 * 8 + 64;
    const uint32_t b_bytes = (uint32_t)P.nk * NP * (uint32_t)P.ntile * 128;
    const uint32_t a_stage = NP * BM * 128;
    if (P.n_ntiles == 1 && (size_t)b_bytes + 2 * a_stage + extra <= (size_t)s->smem_optin) {
      int stages = (int)(((size_t)s->smem_optin - extra - b_bytes) / a_stage);
      if (stages > 4) stages = 4;
      P.stages = stages;
      P.b_bytes = b_bytes;
      const size_t smem = (size_t)b_bytes + (size_t)stages * a_stage + extra;
      auto kern = tc_gemm_res_kernel<KIND, NP>;
      static int smem_set_r[64] = {0};
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
      if (smem_set_r[dev] < (int)smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_optin);
        if (e != cudaSuccess) return e;
        smem_set_r[dev] = s->smem_optin;
      }
      // the fewest CTAs that keep the makespan (ceil(tiles / SMs) each)
      const int sms = s->sms > 0 ? s->sms : 152;
      const int per = (P.num_tiles + sms - 1) / sms;
      const int grid = (P.num_tiles + per - 1) / per;
      count_launch();
      return launch_pdl(kern, dim3(grid), dim3(NTHREADS), smem, st, mA[0], mA[1], mB, P);
    }
  }
  const uint32_t stage_bytes = NP * (BM * 128 + (uint32_t)P.ntile * 128);
  const size_t extra = 1024 + 64 * 8 + 64;
  int stages = (int)((size_t)(s->smem_optin - extra) / stage_bytes);
  if (stages > 4) stages = 4;
  if (stages < 2) return cudaErrorInvalidConfiguration;
  P.stages = stages;
  const size_t smem = (size_t)stages * stage_bytes + extra;
  auto kern = tc_gemm_kernel<KIND, NP>;
  // raise the kernel's dynamic shared-memory limit once per process (the
  // attribute applies to every later launch on this device)
  static int smem_set[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem_set[dev] < (int)smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         s->smem_optin);
    if (e != cudaSuccess) return e;
    smem_set[dev] = s->smem_optin;
  }
  // With 512 TMEM columns the shared memory (>= 4 x 34 KiB) already keeps a
  // second CTA off the SM, so co-resident CTAs never oversubscribe TMEM.
  int grid = P.num_tiles < 152 ? P.num_tiles : 152;
  count_launch();
  return launch_pdl(kern, dim3(grid), dim3(NTHREADS), smem, st, mA[0], mA[1], mB, P);
}

}  // namespace

cudaError_t tc_tucker(TcState* s, int B, const Combo* in, const TcMats* mats, const Epi* epi,
                      cudaStream_t st, const float** res, const TcPrologue* pro, const cudaEvent_t* ev) {
  if (B < 1 || B > s->batch || s->batch > kTcMaxBatch) return cudaErrorInvalidValue;
  if (pro && (pro->nside < 0 || pro->nside > kTcMaxSide)) return cudaErrorInvalidValue;
  bool mixed = false;
  for (int b = 1; b < B; ++b)
    for (int mu = 0; mu < s->d; ++mu) mixed = mixed || mats[b].B[mu] != mats[0].B[mu];
  if (mixed && !tc_mixed_ok(s)) return cudaErrorInvalidValue;
  const int nmat = mixed ? B : 1;
  const int dtype = s->dtype;
  const int NP = planes_of(dtype), elt = elt_of(dtype);
  const int64_t N = s->N;
  const size_t plane = ((size_t)s->batch * N * 4 + 1023) / 1024 * 1024;
  uint8_t* set[2][2] = {{s->ws, s->ws + plane}, {s->ws + 2 * plane, s->ws + 3 * plane}};
  // split the (combined) inputs into planes: natural layout, mode 1
  // contiguous, tensor b at element b N of every plane; into the set that
  // does not hold the last call's results, which the inputs may read
  int cur = 1 - s->last_res;
  // tensors with their own matrices and one and the same input (the
  // quadrature nodes of a same-vector call): that input is split once and
  // every tensor's tiles of the first pass read it
  bool shared = mixed && B > 1;
  for (int b = 1; b < B && shared; ++b)
    shared = same_combo(in[b], in[0]) && !(pro && pro->store[b]);
  {
    const int nsplit = shared ? 1 : B;
    TcSplitJobs jb;
    std::memset(&jb, 0, sizeof jb);
    for (int b = 0; b < nsplit; ++b) {
      jb.c[b] = in[b];
      jb.store[b] = pro ? pro->store[b] : nullptr;
    }
    jb.ntensor = nsplit;
    int rows = nsplit;
    if (pro)
      for (int k = 0; k < pro->nside; ++k, ++rows) {
        jb.c[rows] = pro->side[k];
        jb.store[rows] = pro->side_out[k];
        if ((pro->side_f32 >> k) & 1) jb.store_f32 |= 1u << rows;
      }
    tc_split_coefs(jb, rows);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 152 * 8 / rows));
    count_launch();
    void *q0 = set[cur][0], *q1 = set[cur][1], *none = nullptr;
    const dim3 g(grid, rows);
    cudaError_t e;
    if (dtype == PHIKS_BF16X3) e = launch_pdl(tc_split_kernel<0, 2>, g, dim3(256), 0, st, jb, N, q0, q1);
    else if (dtype == PHIKS_TF32X3) e = launch_pdl(tc_split_kernel<1, 2>, g, dim3(256), 0, st, jb, N, q0, q1);
    else e = launch_pdl(tc_split_kernel<1, 1>, g, dim3(256), 0, st, jb, N, q0, none);
    if (e != cudaSuccess) return e;
  }
  for (int mu = 0; mu < s->d; ++mu) {
    const int n = (int)s->n[mu], np = pad16(n);
    const int64_t M2 = N / n;
    const int64_t rows = (int64_t)B * M2;
    // N tiles of at most 256 rows of L.  Tuned: the minimum count times the
    // multiplier (tiles of at least 16 rows).  By size: when the row tiles
    // alone would leave SMs idle (few fibres, large n_mu), more and narrower
    // N tiles (at least 64 rows each) until the pass has about one tile per SM.
    const int64_t row_tiles = mixed ? (int64_t)B * ((M2 + BM - 1) / BM) : (rows + BM - 1) / BM;
    int mult = std::max(s->ntiles_mult, 1);
    if (s->ntiles_mult == 0)
      while (row_tiles * ((np + 255) / 256) * mult < 152 && (np + 255) / 256 * mult * 2 <= np / 64) mult *= 2;
    const int nnt = std::min((np + 255) / 256 * mult, std::max(np / 16, 1));
    const int ntile = pad16((np + nnt - 1) / nnt);
    CUtensorMap mA[2];
    TcMapsB mB;
    std::memset(mA, 0, sizeof mA);
    std::memset(&mB, 0, sizeof mB);
    const size_t bplane = ((size_t)np * np * elt + 1023) / 1024 * 1024;
    for (int p = 0; p < NP; ++p) {
      if (!cached_map(s, &mA[p], set[cur][p], (uint64_t)n, (uint64_t)rows, BM)) {
        g_tc_err = "tensor map for the A operand failed";
        return cudaErrorInvalidValue;
      }
      for (int b = 0; b < nmat; ++b)
        if (!cached_map(s, &mB.b[b][p], (const uint8_t*)mats[b].B[mu] + p * bplane, (uint64_t)np,
                        (uint64_t)np, (uint32_t)ntile)) {
          g_tc_err = "tensor map for the B operand failed";
          return cudaErrorInvalidValue;
        }
    }
    if (NP == 1) {
      mA[1] = mA[0];
      for (int b = 0; b < nmat; ++b) mB.b[b][1] = mB.b[b][0];
    }
    GemmParams P;
    std::memset(&P, 0, sizeof P);
    P.n = n;
    P.n_pad = np;
    P.ntile = ntile;
    P.n_ntiles = nnt;
    P.M2 = M2;
    P.rows = rows;
    P.N = N;
    P.nk = (n * elt + 127) / 128;
    P.tpt = (M2 + BM - 1) / BM;
    P.num_tiles = (int)((mixed ? B * P.tpt : (rows + BM - 1) / BM) * nnt);
    int cols = 32;
    while (cols < 2 * ntile) cols <<= 1;
    P.tmem_cols = cols;
    P.last = (mu == s->d - 1);
    P.mixed = mixed ? 1 : 0;
    P.shared_a = (mu == 0 && shared) ? 1 : 0;
    P.out0 = set[1 - cur][0];
    P.out1 = set[1 - cur][1];
    P.status = s->status;
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[2 * mu], st)) != cudaSuccess) return e;
    if (dtype == PHIKS_BF16X3) e = run_gemm<0, 2>(s, mA, mB, P, st);
    else if (dtype == PHIKS_TF32X3) e = run_gemm<1, 2>(s, mA, mB, P, st);
    else e = run_gemm<1, 1>(s, mA, mB, P, st);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[2 * mu + 1], st)) != cudaSuccess) return e;
    cur = 1 - cur;
  }
  s->last_res = cur;
  if (res) *res = (const float*)set[cur][0];
  if (!epi) return cudaSuccess;
  // FP64 epilogues over all N elements of each tensor with the whole GPU: the
  // result plane is one more (float) source whose coefficient in output t is
  // epi.b[t]
  Epi f[kTcMaxBatch];
  for (int b = 0; b < B; ++b) {
    f[b] = epi[b];
    const int m = f[b].nsrc;
    if (m >= kMaxSrc) return cudaErrorInvalidValue;
    f[b].src[m] = (const double*)((const float*)set[cur][0] + (int64_t)b * N);
    f[b].src_f32mask |= 1 << m;
    for (int t = 0; t < f[b].nout; ++t) f[b].a[t][m] = epi[b].b[t];
    f[b].nsrc = m + 1;
  }
  for (int b0 = 0; b0 < B; b0 += kMaxEpiBatch) {
    cudaError_t e = launch_combine_batch(f + b0, std::min(kMaxEpiBatch, B - b0), N, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int* tc_status_word(TcState* s) { return s->status; }

void tc_set_ntiles(TcState* s, int mult) { s->ntiles_mult = (mult == 1 || mult == 2 || mult == 4) ? mult : 0; }

int tc_read_status(TcState* s, cudaStream_t st) {
  int h = 0;
  if (cudaMemcpyAsync(&h, s->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  if (h) cudaMemsetAsync(s->status, 0, sizeof(int), st);
  return h;
}

}  // namespace phiks
