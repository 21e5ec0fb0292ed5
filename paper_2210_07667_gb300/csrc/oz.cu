// FP64 mu-mode products emulated by exact bf16 digit products on tcgen05
// (see oz.cuh for the arithmetic).
//
// A Tucker operator runs d passes; pass mu contracts the contiguous mode of
// the current layout and writes its FP64 result with that mode moved to the
// slowest position (so the next mode is contiguous and the natural layout is
// back after d passes):
//   1. split:  every fibre of X (n consecutive doubles) -> its exponent and
//              seven bf16 digit planes (n / 8 threads per fibre);
//   2. tcgen05: per tile of 128 fibres x NT rows of L, the 28 digit products
//              accumulate into seven FP32 TMEM accumulators G_0..G_6 (exact);
//              the epilogue assembles sum_k 2^(8(6-k)) G_k in 64-bit integers
//              and rounds it to FP64.
// The last pass writes natural-layout FP64 results that a full-GPU combine
// pass turns into the Tucker operator's epilogue outputs.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <string>
#include <tuple>

#include "devmem.hpp"
#include "oz.cuh"
#include "pdl.cuh"
#include "tcgen05.cuh"

namespace phiks {

namespace {

using namespace ptx;
thread_local std::string g_oz_err;

// Fixed-point value of a double relative to the fibre exponent E (biased):
// x = Q 2^(E - 1077) up to rounding, |Q| < 2^55 (Q = 0 for zeros and
// subnormals, and for elements more than 2^60 below the fibre maximum).
__device__ __forceinline__ long long oz_fixed(double x, int E) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7FF);
  long long Q = 0;
  if (e > 0 && E > 0) {
    const unsigned long long mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = E - e - 2;  // Q = mant * 2^(e - E + 2)
    if (sh <= 0) {
      Q = (long long)(mant << (-sh));
    } else if (sh < 60) {
      Q = (long long)((mant + (1ull << (sh - 1))) >> sh);
    }
    if (bits >> 63) Q = -Q;
  }
  return Q;
}

// The 7 balanced base-256 digits c_0 (most significant) .. c_6 of Q, as
// floats: Q = sum_s c_s 2^(8 (6 - s)), c_1..c_6 in [-128, 127], |c_0| <= 128.
// Adding 128 to each of the six low digit positions turns the balanced digits
// into plain bytes (c_s + 128); the top digit is what remains above them.
__device__ __forceinline__ void oz_digits(long long Q, float* c) {
  const long long Qp = Q + 0x0000808080808080ll;
  const uint32_t lo = (uint32_t)Qp, hi = (uint32_t)((unsigned long long)Qp >> 32);
  // byte b of a word as the float 2^23 + b, minus 2^23 + 128
  auto byte_f = [](uint32_t w, uint32_t b) {
    return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7440u | b)) - 8388736.0f;
  };
  c[6] = byte_f(lo, 0);
  c[5] = byte_f(lo, 1);
  c[4] = byte_f(lo, 2);
  c[3] = byte_f(lo, 3);
  c[2] = byte_f(hi, 0);
  c[1] = byte_f(hi, 1);
  c[0] = (float)((int)hi >> 16);
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ int biased_exp(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
}

constexpr int kSplitThreads = 64;  // threads per block (128 made a call 1% slower, 256 3%)

// Grid rows of a split launch: rows below ntensor are the batch's tensors
// X_b = (combination c[b]), split into digit planes; the rest evaluate their
// combination only.  store[y] (or null): where row y's FP64 values are also
// written.
struct SplitJobs {
  Combo c[kOzMaxBatch + kOzMaxSide];
  double* store[kOzMaxBatch + kOzMaxSide];
  int ntensor;
};

// Each thread splits 8 consecutive elements of one fibre of X_b = (combination
// jb.c[b], b = blockIdx.y) and writes one 16-byte chunk of every digit plane;
// a block holds `fpb` whole fibres (n / 8 threads each), whose exponents meet
// in shared memory.  Plane s of tensor b starts at planes + s * PS + b * N;
// the fibre exponents of tensor b at scale + b * M2.
__global__ void __launch_bounds__(kSplitThreads) oz_split_kernel(const __grid_constant__ SplitJobs jb, int n,
                                                                 int64_t M2, int fpb,
                                                                 __nv_bfloat16* planes, int64_t N,
                                                                 int64_t PS, int* scale) {
  __shared__ int emax[kSplitThreads];
  pdl_wait();
  const int y = blockIdx.y;
  const Combo& in = jb.c[y];
  double* const xout = jb.store[y];
  planes += (int64_t)y * N;
  scale += (int64_t)y * M2;
  const int cpf = n >> 3;
  const int t = threadIdx.x;
  const int fl = t / cpf;
  const int64_t m = (int64_t)blockIdx.x * fpb + fl;
  const bool active = fl < fpb && m < M2;
  const int64_t base = m * n + (int64_t)(t - fl * cpf) * 8;
  if (t < fpb) emax[t] = 0;
  double x[8];
  int E = 0;
  if (active) {
    if (in.nsrc == 1 && in.coef[0] == 1.0) {
      const double* p = in.src[0] + base;
      if (((uintptr_t)p & 15) == 0) {
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          const double2 v = __ldg(reinterpret_cast<const double2*>(p + j));
          x[j] = v.x;
          x[j + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = p[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = 0.0;
      for (int k = 0; k < in.nsrc; ++k) {
        const double* p = in.src[k] + base;
        const double a = in.coef[k];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(a, p[j], x[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) E = max(E, biased_exp(x[j]));
    if (xout) {
      double* q = xout + base;
      if (((uintptr_t)q & 15) == 0) {
#pragma unroll
        for (int j = 0; j < 8; j += 2) *reinterpret_cast<double2*>(q + j) = make_double2(x[j], x[j + 1]);
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) q[j] = x[j];
      }
    }
  }
  if (y >= jb.ntensor) return;  // a combination only (uniform over the block)
  if ((cpf & (cpf - 1)) == 0) {  // (uniform) a fibre's threads are cpf <= 32 consecutive lanes
    for (int o = 1; o < cpf; o <<= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
  } else {
    __syncthreads();
    if (active) atomicMax(&emax[fl], E);
    __syncthreads();
    E = emax[fl];
  }
  if (!active) return;
  uint32_t w[kOzSlices][4];
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    float c0[kOzSlices], c1[kOzSlices];
    oz_digits(oz_fixed(x[j], E), c0);
    oz_digits(oz_fixed(x[j + 1], E), c1);
#pragma unroll
    for (int s = 0; s < kOzSlices; ++s) w[s][j >> 1] = pack_bf16x2(c0[s], c1[s]);
  }
#pragma unroll
  for (int s = 0; s < kOzSlices; ++s)
    *reinterpret_cast<uint4*>(planes + s * PS + base) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
  if (t == fl * cpf) scale[m] = E - 1029;
}

// Fibre exponent of an all-zero fibre in the split of exact sums (below any
// element's; the GEMM pass then assembles S = 0 for it).
constexpr int kOzZeroExp = -(1 << 28);

// Q = S 2^(e - (E - 1077)) rounded half away from zero (the fixed point of
// oz_fixed for the value S 2^e and the fibre exponent E, with E at least the
// biased exponent the value would have as a double: |Q| < 2^55).
__device__ __forceinline__ long long oz_fixed_sum(long long S, int e, int E) {
  if (S == 0) return 0;
  const unsigned long long u = S < 0 ? 0ull - (unsigned long long)S : (unsigned long long)S;
  const int sh = E - 1077 - e;
  unsigned long long q;
  if (sh <= 0) q = u << (-sh);
  else if (sh < 64) q = (u >> sh) + ((u >> (sh - 1)) & 1ull);
  else q = 0;
  return S < 0 ? -(long long)q : (long long)q;
}

// The previous pass's exact sums: element idx of tensor b is S[b N + idx],
// value S 2^(xs[m] + ls[i] - 40) with m = idx mod M2p, i = idx / M2p (the
// previous pass's fibre and output row of its matrix).
struct SplitSums {
  const long long* S;
  const int* xs;               // the previous pass's fibre exponents (row b M2p + m, or m when shared)
  const int* ls[kOzMaxBatch];  // row exponents of tensor b's matrix of the previous mode (entry 0 unless mixed)
  int64_t M2p;
  uint32_t fpr;  // fibres of this pass per row i of the previous pass: M2p / n
  int shared;
  int mixed;
};

// The split of oz_split_kernel for a pass whose input is the previous pass's
// exact sums (no combination): the same threads, exponents and digit planes,
// the fibre exponent the largest value's biased exponent as a double, each
// value rounded once to the fibre's fixed point.
__global__ void __launch_bounds__(kSplitThreads) oz_split_sums_kernel(const __grid_constant__ SplitSums in, int n,
                                                                      int64_t M2, int fpb, __nv_bfloat16* planes,
                                                                      int64_t N, int64_t PS, int* scale) {
  __shared__ int emax[kSplitThreads];
  pdl_wait();
  const int y = blockIdx.y;
  planes += (int64_t)y * N;
  scale += (int64_t)y * M2;
  const int cpf = n >> 3;
  const int t = threadIdx.x;
  const int fl = t / cpf;
  const int64_t m = (int64_t)blockIdx.x * fpb + fl;
  const bool active = fl < fpb && m < M2;
  const int64_t base = m * n + (int64_t)(t - fl * cpf) * 8;
  if (t < fpb) emax[t] = kOzZeroExp;
  long long S[8];
  int e[8];
  int E = kOzZeroExp;
  if (active) {
    const long long* p = in.S + (int64_t)y * N + base;
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const longlong2 v = __ldg(reinterpret_cast<const longlong2*>(p + j));
      S[j] = v.x;
      S[j + 1] = v.y;
    }
    // row i of the previous pass: M2p / n whole fibres each (m < 2^32 here)
    const uint32_t i = (uint32_t)m / in.fpr;
    const int64_t m0 = base - (int64_t)i * in.M2p;
    const int ls = __ldg(in.ls[in.mixed ? y : 0] + i);
    const int4* xs = reinterpret_cast<const int4*>(in.xs + (in.shared ? 0 : (int64_t)y * in.M2p) + m0);
    const int4 xa = __ldg(xs), xb = __ldg(xs + 1);
    const int xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      e[j] = xv[j] + ls - 40;
      if (S[j] != 0) {
        const unsigned long long u = S[j] < 0 ? 0ull - (unsigned long long)S[j] : (unsigned long long)S[j];
        E = max(E, (64 - __clzll((long long)u)) + e[j] + 1022);
      }
    }
  }
  if ((cpf & (cpf - 1)) == 0) {  // (uniform) a fibre's threads are cpf <= 32 consecutive lanes
    for (int o = 1; o < cpf; o <<= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
  } else {
    __syncthreads();
    if (active) atomicMax(&emax[fl], E);
    __syncthreads();
    E = emax[fl];
  }
  if (!active) return;
  uint32_t w[kOzSlices][4];
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    float c0[kOzSlices], c1[kOzSlices];
    oz_digits(oz_fixed_sum(S[j], e[j], E), c0);
    oz_digits(oz_fixed_sum(S[j + 1], e[j + 1], E), c1);
#pragma unroll
    for (int s = 0; s < kOzSlices; ++s) w[s][j >> 1] = pack_bf16x2(c0[s], c1[s]);
  }
#pragma unroll
  for (int s = 0; s < kOzSlices; ++s)
    *reinterpret_cast<uint4*>(planes + s * PS + base) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
  if (t == fl * cpf) scale[m] = E - 1029;
}

// B digits: row i of L (column-major n x n), row-major planes n_pad x n_pad;
// one warp per row, one grid row (blockIdx.y) per matrix of the batch.
constexpr int kPrepBatch = 32;
struct PrepBatch {
  const double* L[kPrepBatch];
  int n[kPrepBatch];
  __nv_bfloat16* planes[kPrepBatch];
};

__global__ void oz_prep_b_kernel(PrepBatch pb) {
  pdl_wait();
  const double* L = pb.L[blockIdx.y];
  const int n = pb.n[blockIdx.y];
  const int n_pad = (n + 63) / 64 * 64;
  __nv_bfloat16* planes = pb.planes[blockIdx.y];
  int* scale = (int*)((uint8_t*)planes + (((size_t)kOzSlices * n_pad * n_pad * 2 + 1023) / 1024 * 1024));
  const int lane = threadIdx.x & 31;
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (i >= n_pad) return;
  const int64_t P = (int64_t)n_pad * n_pad;
  int E = 0;
  for (int k = lane; k < n; k += 32)
    if (i < n) E = max(E, biased_exp(L[i + (int64_t)n * k]));
  E = warp_max(E);
  for (int k = lane; k < n_pad; k += 32) {
    float c[kOzSlices];
    const double x = (i < n && k < n) ? L[i + (int64_t)n * k] : 0.0;
    oz_digits(oz_fixed(x, E), c);
#pragma unroll
    for (int s = 0; s < kOzSlices; ++s) planes[s * P + (int64_t)i * n_pad + k] = __float2bfloat16_rn(c[s]);
  }
  if (lane == 0) scale[i] = E - 1029;
}

// T 2^e rounded to a double, T = sum_k G_k 2^(8 (6 - k)) for the exact
// integer accumulators G_0..G_6 (FP32 bit patterns, |G_k| < 2^24): with
// |T| < 2^70 for n <= 128, S = floor(T / 2^8) fits 63 bits; its conversion
// to double rounds to nearest (an error below (1/2 + 2^-8) ulp of T 2^e in
// all), and 2^(e + 8) enters the exponent field.
//
// The first NM accumulators are bounded by |G_k| <= (k + 1) n 2^14 <= 2^22
// (k + 1 digit products per term, each at most 2^14 in magnitude, n terms):
// for them G_k + 1.5 2^23 is exact and lies in [2^23, 2^24], so its bit
// pattern minus that of 1.5 2^23 is G_k (one FP32 add on the FMA pipe in
// place of a float-to-integer conversion).
template <int NM>
__device__ __forceinline__ long long oz_digit_sum(const uint32_t* G) {
  int g[kOzSlices];
#pragma unroll
  for (int k = 0; k < kOzSlices; ++k)
    g[k] = k < NM ? __float_as_int(__uint_as_float(G[k]) + 12582912.0f) - 0x4B400000
                  : __float2int_rn(__uint_as_float(G[k]));
  long long S;
  if constexpr (NM >= 4) {
    // n <= 64, |G_k| <= (k + 1) 2^20: with T = A 2^40 + B 2^24 + C 2^8 + G_6,
    // A = 2^8 G_0 + G_1, B = 2^8 G_2 + G_3, C = 2^8 G_4 + G_5, the partial
    // sums and C + floor(G_6 / 2^8) fit 32 bits (below 2^31 in magnitude)
    const int A = g[0] * 256 + g[1], B = g[2] * 256 + g[3], C = g[4] * 256 + g[5] + (g[6] >> 8);
    S = (long long)A * 4294967296ll + (long long)B * 65536ll + (long long)C;
  } else {
    long long hi = (long long)(g[0] * 256 + g[1]);
    hi = hi * 256 + g[2];
    hi = hi * 256 + g[3];
    long long lo = (long long)g[4] * 256 + g[5];
    lo = lo * 256 + g[6];
    S = hi * 65536 + (lo >> 8);
  }
  return S;
}

template <int NM>
__device__ __forceinline__ double oz_assemble(const uint32_t* G, int e) {
  const long long S = oz_digit_sum<NM>(G);
  if (S == 0) return 0.0;
  const long long d = __double_as_longlong(__ll2double_rn(S));
  const int be = (int)((d >> 52) & 0x7FF) + e + 8;  // biased exponent of the result
  if (be <= 0) return __longlong_as_double(d & (1ll << 63));  // below the normal range: signed zero
  if (be >= 2047) return __longlong_as_double((d & (1ll << 63)) | (0x7FFll << 52));
  return __longlong_as_double(d + ((long long)(e + 8) << 52));
}

struct OzParams {
  int n;          // contraction length
  int n_pad;      // rows of L padded to a multiple of NT
  int64_t M2;     // fibres of one tensor
  int64_t rows;   // fibres of the batch (tensor b owns rows b M2 .. b M2 + M2 - 1)
  int64_t N;      // elements of one tensor (the output stride between tensors)
  int nk;         // 64-element K chunks
  int n_ntiles;   // tiles of NT rows of L
  int num_tiles;
  int tmem_cols;
  int nbuf;       // TMEM accumulator sets (1 or 2)
  int resident;   // nk == 1: A kept across a row tile's column tiles, B per tensor
  int int_out;    // store the exact digit sums S (int64, value S 2^(sx + ls - 40)) for
                  // the next pass's split instead of rounded doubles
  uint32_t stage_bytes;  // shared memory of the A and B planes
  double* out;    // FP64 result of tensor b, rotated layout: out[b N + m + M2 i]
  const int* xscale;
  int mixed;      // tensors with their own matrices: every tile within one tensor
  int64_t tpt;    // mixed: row tiles per tensor, ceil(M2 / 128) (the last one partial)
  int shared_a;   // mixed, first pass: every tensor's input is tensor 0's (planes and exponents)
  const int* lscale[kOzMaxBatch];  // row exponents of tensor b's matrix (entry 0 unless mixed)
  int* status;
};

// TMA maps of the B digit planes: of tensor b's matrix (entry 0 unless mixed).
struct OzMaps {
  CUtensorMap b[kOzMaxBatch];
};

// First fibre (row of the batch) of row tile rt, and its tensor.  Mixed
// batches tile every tensor on its own (a tensor's last tile may be partial:
// its rows past the tensor read the next tensor's fibres, or the copy's zero
// fill past the batch, and are not stored), so that a tile never needs two
// matrices; otherwise the rows of all tensors are tiled together.
__device__ __forceinline__ int64_t oz_tile_row0(const OzParams& P, int64_t rt, int* b) {
  if (P.mixed) {
    const int64_t bb = rt / P.tpt;
    *b = (int)bb;
    return bb * P.M2 + (rt - bb * P.tpt) * BM;
  }
  *b = 0;
  return rt * BM;
}

constexpr int kOzEpiWarps = 16;
constexpr int NTH = 64 + 32 * kOzEpiWarps;
constexpr int kOzMaxColTiles = 4;  // column tiles of a resident B (n <= 64, NT >= 16)

// This CTA's tiles: a contiguous range of the tile order (row tile major), so
// that consecutive tiles of a CTA mostly share their row tile.
__device__ __forceinline__ void oz_tile_range(const OzParams& P, int* t0, int* t1) {
  const int G = (int)gridDim.x, c = (int)blockIdx.x;
  const int base = P.num_tiles / G, rem = P.num_tiles % G;
  *t0 = c * base + min(c, rem);
  *t1 = *t0 + base + (c < rem ? 1 : 0);
}

// Per tile: A = 7 digit planes of 128 fibres x 64 K, B = 7 digit planes of
// NT rows x 64 K stored back to back, so that one MMA multiplies A plane t by
// B planes 0..6-t at once (N = (7 - t) NT) and writes block s of its result
// to TMEM column block t + s: block k then accumulates
//     G_k = sum_{s + t = k} B_s A_t^T,  k = 0..6,
// with 7 MMAs per 16-wide K step instead of 28 (the first, t = 0, covers all
// seven blocks and starts them).  A planes land on their own barriers, so
// the MMAs of plane t start once it is in.  Warp 0 issues the copies, one
// thread of warp 1 the MMAs, and the kOzEpiWarps warps from 2 on the
// epilogue (kOzEpiWarps / 4 warps per TMEM lane quarter, each taking an
// equal share of the NT columns); two TMEM accumulator sets let a tile's
// MMAs run during the previous tile's epilogue.
//
// This kernel is the resident form (n <= 64: one K chunk): a CTA's tiles are
// consecutive, the A planes of a row tile (112 KiB) are loaded once for all of
// its column tiles, and each column tile's B planes once per tensor (one slot
// and one barrier per column tile), so that the copies of the next row tile
// overlap the epilogues of the current one.  n > 64 runs
// oz_gemm_stream_kernel below, which streams every tile's K chunks of A and B
// through one stage.

template <int NT>
__global__ void __launch_bounds__(NTH, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ OzMaps mapsB,
                   const __grid_constant__ OzParams P) {
  static_assert(kOzSlices * NT <= 256 && (kOzSlices * NT) % 16 == 0, "MMA N out of range");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr uint32_t A_SLICE = BM * 128;  // bytes of one digit plane of the A tile
  constexpr uint32_t B_SLICE = NT * 128;
  constexpr uint32_t SET = kOzSlices * NT;  // TMEM columns of one accumulator set
  uint64_t* fullA = (uint64_t*)(smem + P.stage_bytes);  // [7]: plane t of A landed
  uint64_t* fullB = fullA + kOzSlices;  // [kOzMaxColTiles]: the B planes of a column tile landed
  uint64_t* empty = fullB + kOzMaxColTiles;
  uint64_t* tfull = empty + 1;
  uint64_t* tempty = tfull + 2;
  uint64_t* mdone = tempty + 2;  // the MMA warp's issued MMAs finished (failure path)
  uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int t = 0; t < kOzSlices; ++t) mbar_init(&fullA[t], 1);
    for (int c = 0; c < kOzMaxColTiles; ++c) mbar_init(&fullB[c], 1);
    mbar_init(empty, 1);
    mbar_init(mdone, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 32 * kOzEpiWarps);
    }
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
  pdl_wait();  // the digit planes and scales come from the kernels before

  int t_begin = 0, t_end = 0;
  oz_tile_range(P, &t_begin, &t_end);
  uint8_t* const smemB = smem + kOzSlices * A_SLICE;
  if (warp == 0) {
    if (lane == 0) {
      uint32_t eph = 0, bmask = 0, bever = 0, bph = 0;  // per column tile: loaded, parity of the next load
      int nA = 0;
      int prev_rt = -1, prev_tb = -1;
      for (int t = t_begin; t < t_end; ++t) {
        const int rt = t / P.n_ntiles, ct = t % P.n_ntiles;
        int tb = 0;
        int m0 = (int)oz_tile_row0(P, rt, &tb);
        if (rt != prev_rt) {
          if (prev_rt >= 0) {  // the MMAs on the previous row tile's planes finished
            if (!mbar_wait(empty, eph, P.status, 11)) break;
            eph ^= 1;
          }
          if (tb != prev_tb) {  // another tensor's matrix: every B slot is stale
            bmask = 0;
            prev_tb = tb;
          }
        }
        if (!((bmask >> ct) & 1u)) {  // B first: the tile's first MMA needs it and A plane 0
          mbar_arrive_expect_tx(&fullB[ct], kOzSlices * B_SLICE);
#pragma unroll 1
          for (int s = 0; s < kOzSlices; ++s)
            tma_load_3d(smemB + (ct * kOzSlices + s) * B_SLICE, &mapsB.b[tb], &fullB[ct], 0, ct * NT, s);
          bmask |= 1u << ct;
          bever |= 1u << ct;
          bph ^= 1u << ct;
        }
        if (rt != prev_rt) {
          if (P.shared_a) m0 -= (int)(tb * P.M2);  // the one split input
#pragma unroll 1
          for (int s = 0; s < kOzSlices; ++s) {
            mbar_arrive_expect_tx(&fullA[s], A_SLICE);
            tma_load_3d(smem + s * A_SLICE, &mapA, &fullA[s], 0, m0, s);
          }
          ++nA;
          prev_rt = rt;
        }
      }
      // the last copies landed (also after another role gave up)
      if (nA)
        for (int s = 0; s < kOzSlices; ++s) (void)mbar_drain(&fullA[s], (uint32_t)(nA - 1) & 1u);
      for (int c = 0; c < kOzMaxColTiles; ++c)
        if ((bever >> c) & 1u) (void)mbar_drain(&fullB[c], ((bph >> c) & 1u) ^ 1u);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t aph = 0, apar = 0, bmask = 0, bpar = 0;
      int buf = 0, prev_rt = -1, prev_tb = -1;
      bool ok = true, any = false;
      for (int t = t_begin; t < t_end && ok; ++t) {
        const int rt = t / P.n_ntiles, ct = t % P.n_ntiles;
        if (!mbar_wait(&tempty[buf], aph ^ 1, P.status, 12)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d0 = tmem_base + (uint32_t)buf * SET;
        const uint32_t a0 = smem_u32(smem);
        {
          int tb = 0;
          (void)oz_tile_row0(P, rt, &tb);
          const bool newA = rt != prev_rt;
          if (newA && tb != prev_tb) {
            bmask = 0;
            prev_tb = tb;
          }
          if (!((bmask >> ct) & 1u)) {
            if (!mbar_wait(&fullB[ct], (bpar >> ct) & 1u, P.status, 13)) {
              ok = false;
              break;
            }
            bpar ^= 1u << ct;
            bmask |= 1u << ct;
          }
          // descriptors of plane 0 / K step 0; the others differ in the start
          // address field only (16-byte units, no carry out of the field)
          const uint64_t da = sdesc_sw128(a0);
          const uint64_t db = sdesc_sw128(smem_u32(smemB) + (uint32_t)(ct * kOzSlices) * B_SLICE);
#pragma unroll
          for (int at = 0; at < kOzSlices; ++at) {  // digit plane at of X times every plane of L
            if (newA && !mbar_wait(&fullA[at], apar, P.status, 13)) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              umma<0>(d0 + (uint32_t)(at * NT), da + (uint64_t)((at * A_SLICE + kk * 32) >> 4),
                      db + (uint64_t)((kk * 32) >> 4), idesc_make(1, (kOzSlices - at) * NT),
                      (kk == 0 && at == 0) ? 0u : 1u);
            any = true;
          }
          if (!ok) break;
          if (newA) {
            apar ^= 1;
            prev_rt = rt;
          }
          // the last tile on these A planes: the stage is free for the next row tile
          if (t + 1 < t_end && (t + 1) / P.n_ntiles != rt) umma_commit(empty);
        }
        umma_commit(&tfull[buf]);
        if (++buf == P.nbuf) {
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
    const int q = warp & 3;  // TMEM lane quarter of this warp
    constexpr int GROUPS = kOzEpiWarps / 4;   // warps per lane quarter
    constexpr int CW = NT / GROUPS;           // columns per warp: one TMEM load per block
    static_assert(CW == 8 || CW == 4, "epilogue column split");
    const int grp = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    int buf = 0;
    uint32_t aph = 0;
    for (int t = t_begin; t < t_end; ++t) {
      // the tile's fibre and row exponents first: their loads run while the
      // MMAs finish (none of them depends on this tile's accumulators)
      int tb = 0;
      const int64_t m0t = oz_tile_row0(P, t / P.n_ntiles, &tb);
      const int64_t rg = m0t + row;  // fibre of the batch
      const int r0 = (t % P.n_ntiles) * NT;
      const bool valid = P.mixed ? (rg - (int64_t)tb * P.M2 < P.M2) : (rg < P.rows);
      const int sx = valid ? P.xscale[P.shared_a ? rg - (int64_t)tb * P.M2 : rg] : 0;
      const int64_t bt = valid ? (P.mixed ? tb : rg / P.M2) : 0;
      double* const outb = P.out + bt * P.N;
      const int64_t m = rg - bt * P.M2;
      const int* const lscale = P.lscale[P.mixed ? tb : 0];
      int ls[CW];  // (lscale has n_pad >= every tile's columns entries)
#pragma unroll
      for (int j = 0; j < CW; ++j) ls[j] = lscale[r0 + grp * CW + j];
      if (!mbar_wait(&tfull[buf], aph, P.status, 14)) break;
      tc_fence_after();
      const int c0 = grp * CW;
      uint32_t G[kOzSlices][CW];
      {
        const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * SET + (uint32_t)c0;
        if constexpr (CW == 8) {
#pragma unroll
          for (int k = 0; k < kOzSlices; ++k) tmem_ld8_nowait(ta + (uint32_t)(k * NT), G[k]);
        } else {
#pragma unroll
          for (int k = 0; k < kOzSlices; ++k) tmem_ld4_nowait(ta + (uint32_t)(k * NT), G[k]);
        }
        tmem_wait_ld();
      }
      // the accumulators are in registers: the set is free for the MMAs of a
      // later tile (which frees this row tile's A planes sooner)
      tc_fence_before();
      mbar_arrive(&tempty[buf]);
      if (valid && P.int_out) {
        // the exact sums: the next pass's split takes them with their scale
        long long* const outi = reinterpret_cast<long long*>(outb);
        long long r[CW];
        if (P.n <= 36) {
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            uint32_t g[kOzSlices];
#pragma unroll
            for (int k = 0; k < kOzSlices; ++k) g[k] = G[k][j];
            r[j] = oz_digit_sum<7>(g);
          }
        } else {  // n <= 64
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            uint32_t g[kOzSlices];
#pragma unroll
            for (int k = 0; k < kOzSlices; ++k) g[k] = G[k][j];
            r[j] = oz_digit_sum<4>(g);
          }
        }
#pragma unroll
        for (int j = 0; j < CW; ++j)
          if (r0 + c0 + j < P.n) outi[m + P.M2 * (int64_t)(r0 + c0 + j)] = r[j];
      } else if (valid) {
        // independent assemblies, then the stores of the columns below n
        double r[CW];
        // accumulators small enough for the exact FP32 conversion: (k + 1) n <= 256
        if (P.n <= 36) {
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            uint32_t g[kOzSlices];
#pragma unroll
            for (int k = 0; k < kOzSlices; ++k) g[k] = G[k][j];
            r[j] = oz_assemble<7>(g, sx + ls[j] - 48);
          }
        } else {  // n <= 64
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            uint32_t g[kOzSlices];
#pragma unroll
            for (int k = 0; k < kOzSlices; ++k) g[k] = G[k][j];
            r[j] = oz_assemble<4>(g, sx + ls[j] - 48);
          }
        }
#pragma unroll
        for (int j = 0; j < CW; ++j)
          if (r0 + c0 + j < P.n) outb[m + P.M2 * (int64_t)(r0 + c0 + j)] = r[j];
      }
      if (++buf == P.nbuf) {
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

// The streaming form for n > 64 (several 64-wide K chunks): every gridDim-th
// tile streams its K chunks of A and B through one shared-memory stage
// (112 KiB of A digits per chunk); otherwise as above (seven A-plane barriers,
// two TMEM accumulator sets, 16 epilogue warps) with every accumulator
// converted by a float-to-integer conversion.
template <int NT>
__global__ void __launch_bounds__(NTH, 1)
    oz_gemm_stream_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ OzMaps mapsB,
                   const __grid_constant__ OzParams P) {
  static_assert(kOzSlices * NT <= 256 && (kOzSlices * NT) % 16 == 0, "MMA N out of range");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr uint32_t A_SLICE = BM * 128;  // bytes of one digit plane of the A tile
  constexpr uint32_t B_SLICE = NT * 128;
  constexpr uint32_t STAGE = kOzSlices * (A_SLICE + B_SLICE);
  constexpr uint32_t SET = kOzSlices * NT;  // TMEM columns of one accumulator set
  uint64_t* fullA = (uint64_t*)(smem + STAGE);  // [7]: plane t of A landed
  uint64_t* fullB = fullA + kOzSlices;          // all planes of B landed
  uint64_t* empty = fullB + 1;
  uint64_t* tfull = empty + 1;
  uint64_t* tempty = tfull + 2;
  uint64_t* mdone = tempty + 2;  // the MMA warp's issued MMAs finished (failure path)
  uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int t = 0; t < kOzSlices; ++t) mbar_init(&fullA[t], 1);
    mbar_init(fullB, 1);
    mbar_init(empty, 1);
    mbar_init(mdone, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 32 * kOzEpiWarps);
    }
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
  pdl_wait();  // the digit planes and scales come from the kernels before

  if (warp == 0) {
    if (lane == 0) {
      uint32_t ph = 0;
      int issued = 0;
      for (int t = blockIdx.x; t < P.num_tiles; t += gridDim.x) {
        int tb = 0;
        int m0 = (int)oz_tile_row0(P, t / P.n_ntiles, &tb);
        if (P.shared_a) m0 -= (int)(tb * P.M2);  // the one split input
        const int r0 = (t % P.n_ntiles) * NT;
        const CUtensorMap* mapB = &mapsB.b[tb];
        bool ok = true;
        for (int kc = 0; kc < P.nk; ++kc) {
          if (!mbar_wait(empty, ph ^ 1, P.status, 11)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(fullB, kOzSlices * B_SLICE);
#pragma unroll 1
          for (int s = 0; s < kOzSlices; ++s)
            tma_load_3d(smem + kOzSlices * A_SLICE + s * B_SLICE, mapB, fullB, kc * 64, r0, s);
#pragma unroll 1
          for (int s = 0; s < kOzSlices; ++s) {
            mbar_arrive_expect_tx(&fullA[s], A_SLICE);
            tma_load_3d(smem + s * A_SLICE, &mapA, &fullA[s], kc * 64, m0, s);
          }
          ph ^= 1;
          ++issued;
        }
        if (!ok) break;
      }
      if (issued) {  // the last copies landed (also after another role gave up)
        (void)mbar_drain(fullB, ph ^ 1);
        for (int s = 0; s < kOzSlices; ++s) (void)mbar_drain(&fullA[s], ph ^ 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t ph = 0, aph = 0;
      int buf = 0;
      bool ok = true, any = false;
      for (int t = blockIdx.x; t < P.num_tiles && ok; t += gridDim.x) {
        if (!mbar_wait(&tempty[buf], aph ^ 1, P.status, 12)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d0 = tmem_base + (uint32_t)buf * SET;
        for (int kc = 0; kc < P.nk && ok; ++kc) {
          const uint32_t a0 = smem_u32(smem), b0 = a0 + kOzSlices * A_SLICE;
          if (!mbar_wait(fullB, ph, P.status, 13)) {
            ok = false;
            break;
          }
#pragma unroll 1
          for (int at = 0; at < kOzSlices; ++at) {  // digit plane at of X times every plane of L
            if (!mbar_wait(&fullA[at], ph, P.status, 13)) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t first = (kc == 0 && kk == 0 && at == 0) ? 0u : 1u;
              umma<0>(d0 + (uint32_t)(at * NT), sdesc_sw128(a0 + at * A_SLICE + kk * 32),
                      sdesc_sw128(b0 + kk * 32), idesc_make(1, (kOzSlices - at) * NT), first);
            }
            any = true;
          }
          if (!ok) break;
          umma_commit(empty);
          ph ^= 1;
        }
        if (!ok) break;
        umma_commit(&tfull[buf]);
        if (++buf == P.nbuf) {
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
    const int q = warp & 3;  // TMEM lane quarter of this warp
    constexpr int GROUPS = kOzEpiWarps / 4;   // warps per lane quarter
    constexpr int CW = NT / GROUPS;           // columns per warp
    constexpr int CH = CW >= 8 ? 8 : 4;       // columns per TMEM load
    static_assert(CW % CH == 0, "epilogue column split");
    const int grp = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    int buf = 0;
    uint32_t aph = 0;
    for (int t = blockIdx.x; t < P.num_tiles; t += gridDim.x) {
      // the tile's fibre and row exponents first: their loads run while the
      // MMAs finish (none of them depends on this tile's accumulators)
      int tb = 0;
      const int64_t m0t = oz_tile_row0(P, t / P.n_ntiles, &tb);
      const int64_t rg = m0t + row;  // fibre of the batch
      const int r0 = (t % P.n_ntiles) * NT;
      const bool valid = P.mixed ? (rg - (int64_t)tb * P.M2 < P.M2) : (rg < P.rows);
      const int sx = valid ? P.xscale[P.shared_a ? rg - (int64_t)tb * P.M2 : rg] : 0;
      const int64_t bt = valid ? (P.mixed ? tb : rg / P.M2) : 0;
      double* const outb = P.out + bt * P.N;
      const int64_t m = rg - bt * P.M2;
      const int* const lscale = P.lscale[P.mixed ? tb : 0];
      int ls[CW];  // (lscale has n_pad >= every tile's columns entries)
#pragma unroll
      for (int j = 0; j < CW; ++j) ls[j] = lscale[r0 + grp * CW + j];
      if (!mbar_wait(&tfull[buf], aph, P.status, 14)) break;
      tc_fence_after();
#pragma unroll
      for (int c0 = grp * CW; c0 < (grp + 1) * CW; c0 += CH) {
        const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * SET + (uint32_t)c0;
        uint32_t G[kOzSlices][CH];
        if constexpr (CH == 8) {
#pragma unroll
          for (int k = 0; k < kOzSlices; ++k) tmem_ld8_nowait(tb + (uint32_t)(k * NT), G[k]);
        } else {
#pragma unroll
          for (int k = 0; k < kOzSlices; ++k) tmem_ld4_nowait(tb + (uint32_t)(k * NT), G[k]);
        }
        tmem_wait_ld();
        if (!valid) continue;
        if (P.int_out) {  // the exact sums for the next pass's split ((k + 1) n <= 256 for k < 2)
          long long* const outi = reinterpret_cast<long long*>(outb);
          long long r[CH];
#pragma unroll
          for (int j = 0; j < CH; ++j) {
            uint32_t g[kOzSlices];
#pragma unroll
            for (int k = 0; k < kOzSlices; ++k) g[k] = G[k][j];
            r[j] = oz_digit_sum<2>(g);
          }
#pragma unroll
          for (int j = 0; j < CH; ++j)
            if (r0 + c0 + j < P.n) outi[m + P.M2 * (int64_t)(r0 + c0 + j)] = r[j];
          continue;
        }
        // independent assemblies, then the stores of the columns below n
        double r[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          uint32_t g[kOzSlices];
#pragma unroll
          for (int k = 0; k < kOzSlices; ++k) g[k] = G[k][j];
          r[j] = oz_assemble<0>(g, sx + ls[c0 - grp * CW + j] - 48);
        }
#pragma unroll
        for (int j = 0; j < CH; ++j)
          if (r0 + c0 + j < P.n) outb[m + P.M2 * (int64_t)(r0 + c0 + j)] = r[j];
      }
      tc_fence_before();
      mbar_arrive(&tempty[buf]);
      if (++buf == P.nbuf) {
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

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                              CUtensorMapFloatOOBfill);
EncodeFn g_enc = nullptr;

bool get_enc() {
  if (g_enc) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  g_enc = (EncodeFn)fn;
  return true;
}

// 3D map over 7 planes of row-major (rows x inner) bf16 arrays, plane_elems
// elements apart; box {64, box_rows, 1} (one plane) with the 128-byte swizzle.
bool make_map3(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows,
               uint64_t plane_elems) {
  cuuint64_t dims[3] = {inner, rows, (cuuint64_t)kOzSlices};
  cuuint64_t strides[2] = {inner * 2, plane_elems * 2};
  cuuint32_t box[3] = {64, box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return g_enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t up1k(size_t x) { return (x + 1023) / 1024 * 1024; }

int ntile_for(int n, int64_t M2) {
  // enough tiles to spread over the SMs, at most 32 rows (one MMA covers the
  // seven B planes: N = 7 NT <= 256)
  const int64_t mt = (M2 + BM - 1) / BM;
  if (n <= 16) return 16;
  if (mt * ((n + 31) / 32) >= 152 || n <= 32) return 32;
  return mt * ((n + 15) / 16) >= 152 ? 32 : 16;
}

}  // namespace

struct OzState {
  int d = 0;
  int64_t n[PHIKS_MAX_D] = {0};
  int64_t N = 0;
  int* status = nullptr;
  uint8_t* ws = nullptr;
  double* tmp[2] = {nullptr, nullptr};
  int batch = 0;  // tensors the bound workspace holds
  int smem_optin = 0;
  int sms = 0;    // streaming multiprocessors of the device
  int ntile = 0;  // rows of L per GEMM tile (0: by size)
  std::map<std::tuple<const void*, uint64_t, uint64_t, uint32_t, uint64_t>, CUtensorMap> maps;
};

// Digit planes and two sets of fibre exponents (a pass's and its
// predecessor's) of `batch` tensors.
size_t oz_workspace_bytes(int d, const int64_t* n, int64_t N, int batch) {
  int64_t m2 = 0;
  for (int mu = 0; mu < d; ++mu) m2 = std::max<int64_t>(m2, N / n[mu]);
  return up1k((size_t)kOzSlices * batch * N * 2) + 2 * up1k((size_t)batch * m2 * 4) + 1024;
}

phiks_status oz_create(OzState** out, int d, const int64_t* n, int64_t N) {
  *out = nullptr;
  for (int mu = 0; mu < d; ++mu)
    if (n[mu] > kOzMaxN || n[mu] % 8 != 0) {
      g_oz_err = "FP64 emulation needs every n_mu to be a multiple of 8 and at most 128";
      return PHIKS_ERR_UNSUPPORTED;
    }
  if (!get_enc()) {
    g_oz_err = "cuTensorMapEncodeTiled is not available";
    return PHIKS_ERR_UNSUPPORTED;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess || prop.major < 10) {
    g_oz_err = "FP64 emulation needs an sm_100-class device";
    return PHIKS_ERR_UNSUPPORTED;
  }
  OzState* s = new OzState;
  s->d = d;
  for (int mu = 0; mu < d; ++mu) s->n[mu] = n[mu];
  s->N = N;
  s->smem_optin = (int)prop.sharedMemPerBlockOptin;
  s->sms = prop.multiProcessorCount;
  if (dev_malloc((void**)&s->status, sizeof(int)) != cudaSuccess ||
      cudaMemset(s->status, 0, sizeof(int)) != cudaSuccess) {
    dev_free(s->status);
    delete s;
    g_oz_err = "status word allocation failed";
    return PHIKS_ERR_OOM;
  }
  *out = s;
  return PHIKS_OK;
}

void oz_destroy(OzState* s) {
  if (!s) return;
  dev_free(s->status);
  delete s;
}

const char* oz_last_error() { return g_oz_err.c_str(); }

void oz_bind_workspace(OzState* s, void* ws, double* tmp0, double* tmp1, int batch) {
  s->ws = (uint8_t*)ws;
  s->batch = batch;
  s->tmp[0] = tmp0;
  s->tmp[1] = tmp1;
}

size_t oz_bplanes_bytes(int n) {
  const size_t np = (size_t)(n + 63) / 64 * 64;
  return up1k((size_t)kOzSlices * np * np * 2) + up1k(np * 4);
}

cudaError_t oz_prepare_b(int count, const double* const* L, const int* n, void* const* dst,
                         cudaStream_t st) {
  for (int k0 = 0; k0 < count; k0 += kPrepBatch) {
    PrepBatch pb;
    std::memset(&pb, 0, sizeof pb);
    const int cnt = std::min(kPrepBatch, count - k0);
    int npmax = 64;
    for (int k = 0; k < cnt; ++k) {
      pb.L[k] = L[k0 + k];
      pb.n[k] = n[k0 + k];
      pb.planes[k] = (__nv_bfloat16*)dst[k0 + k];
      npmax = std::max(npmax, (n[k0 + k] + 63) / 64 * 64);
    }
    count_launch();
    cudaError_t e = launch_pdl(oz_prep_b_kernel, dim3((npmax * 32 + 255) / 256, cnt), dim3(256), 0, st, pb);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {

template <int NT>
cudaError_t run_oz_gemm(OzState* s, const CUtensorMap& mA, const OzMaps& mB, const OzParams& P,
                        cudaStream_t st) {
  const size_t smem = P.stage_bytes + 1024 + 256;  // alignment slack, barriers
  if ((int)smem > s->smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = P.resident ? oz_gemm_kernel<NT> : oz_gemm_stream_kernel<NT>;
  static int set[2][64] = {{0}};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!set[P.resident][dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_optin);
    if (e != cudaSuccess) return e;
    set[P.resident][dev] = 1;
  }
  // resident form: the fewest CTAs that still give every CTA at most
  // ceil(tiles / SMs) tiles: the same makespan, and the SMs left over take
  // the work that runs beside the pass (the next squaring level's small
  // exponentials); the streaming form, bound by its copies, takes every SM
  const int sms = s->sms > 0 ? s->sms : 152;
  const int per = (P.num_tiles + sms - 1) / sms;
  const int grid = P.resident ? (P.num_tiles + per - 1) / per : std::min(P.num_tiles, sms);
  count_launch();
  return launch_pdl(kern, dim3(grid), dim3(NTH), smem, st, mA, mB, P);
}

bool cached(OzState* s, CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint32_t box,
            uint64_t plane_elems) {
  auto key = std::make_tuple(base, inner, rows, box, plane_elems);
  auto it = s->maps.find(key);
  if (it != s->maps.end()) {
    *m = it->second;
    return true;
  }
  if (!make_map3(m, base, inner, rows, box, plane_elems)) return false;
  if (s->maps.size() > 4096) s->maps.clear();
  s->maps.emplace(key, *m);
  return true;
}

}  // namespace

namespace {
// Whether two input combinations are the same tensors with the same weights.
bool same_combo(const Combo& a, const Combo& b) {
  if (a.nsrc != b.nsrc || a.f32mask != b.f32mask) return false;
  for (int m = 0; m < a.nsrc; ++m)
    if (a.src[m] != b.src[m] || a.coef[m] != b.coef[m]) return false;
  return true;
}
}  // namespace

bool oz_mixed_ok(const OzState* s) {
  (void)s;  // every shape: mixed batches tile each tensor on its own
  return true;
}

cudaError_t oz_tucker(OzState* s, int B, const Combo* in, const OzMats* mats, const Epi* epi,
                      cudaStream_t st, const cudaEvent_t* ev, const double** res, const OzPrologue* pro) {
  if (B < 1 || B > s->batch || s->batch > kOzMaxBatch) return cudaErrorInvalidValue;
  if (pro && (pro->nside < 0 || pro->nside > kOzMaxSide)) return cudaErrorInvalidValue;
  bool mixed = false;
  for (int b = 1; b < B; ++b)
    for (int mu = 0; mu < s->d; ++mu) mixed = mixed || mats[b].B[mu] != mats[0].B[mu];
  if (mixed && !oz_mixed_ok(s)) return cudaErrorInvalidValue;
  const int nmat = mixed ? B : 1;
  const int64_t N = s->N;
  const int64_t PS = (int64_t)s->batch * N;  // elements between digit planes
  __nv_bfloat16* planes = (__nv_bfloat16*)s->ws;
  int64_t m2max = 0;
  for (int mu = 0; mu < s->d; ++mu) m2max = std::max<int64_t>(m2max, N / s->n[mu]);
  // fibre exponents of pass mu in xs[mu & 1]: the split of exact sums reads
  // the previous pass's
  int* xs[2];
  xs[0] = (int*)(s->ws + up1k((size_t)kOzSlices * PS * 2));
  xs[1] = (int*)((uint8_t*)xs[0] + up1k((size_t)s->batch * m2max * 4));
  // tensors with their own matrices and one and the same input (the
  // quadrature nodes of a same-vector call): the first pass splits that input
  // once and every tensor's tiles read it
  bool shared = mixed && B > 1;
  for (int b = 1; b < B && shared; ++b)
    shared = same_combo(in[b], in[0]) && !(pro && pro->store[b]);
  const int nsplit = shared ? 1 : B;
  SplitJobs cur;
  std::memset(&cur, 0, sizeof cur);
  for (int b = 0; b < nsplit; ++b) {
    cur.c[b] = in[b];
    cur.store[b] = pro ? pro->store[b] : nullptr;
  }
  cur.ntensor = nsplit;
  int rows0 = nsplit;  // grid rows of the first split
  if (pro)
    for (int k = 0; k < pro->nside; ++k, ++rows0) {
      cur.c[rows0] = pro->side[k];
      cur.store[rows0] = pro->side_out[k];
    }
  double* dst = nullptr;
  bool sums_in = false;  // the previous pass left exact sums (sin) rather than doubles
  SplitSums sin;
  std::memset(&sin, 0, sizeof sin);
  for (int mu = 0; mu < s->d; ++mu) {
    const int n = (int)s->n[mu];
    const int64_t M2 = N / n;
    const int64_t rows = (int64_t)B * M2;
    int* const xscale = xs[mu & 1];
    {  // split: n / 8 threads per fibre, whole fibres per block, one grid row per tensor
      const int fpb = kSplitThreads / (n / 8);
      const int64_t blocks = (M2 + fpb - 1) / fpb;
      count_launch();
      cudaError_t e =
          sums_in ? launch_pdl(oz_split_sums_kernel, dim3((unsigned)blocks, (unsigned)B), dim3(kSplitThreads), 0, st,
                               sin, n, M2, fpb, planes, N, PS, xscale)
                  : launch_pdl(oz_split_kernel, dim3((unsigned)blocks, (unsigned)(mu == 0 ? rows0 : B)),
                               dim3(kSplitThreads), 0, st, cur, n, M2, fpb, planes, N, PS, xscale);
      if (e != cudaSuccess) return e;
    }
    const int np = (n + 63) / 64 * 64;
    const int NT = s->ntile ? s->ntile : ntile_for(n, rows);
    OzParams P;
    std::memset(&P, 0, sizeof P);
    OzMaps mB;
    CUtensorMap mA;
    if (!cached(s, &mA, planes, (uint64_t)n, (uint64_t)rows, BM, (uint64_t)PS)) {
      g_oz_err = "tensor map encoding failed";
      return cudaErrorInvalidValue;
    }
    for (int b = 0; b < nmat; ++b) {
      const uint8_t* bpl = (const uint8_t*)mats[b].B[mu];
      P.lscale[b] = (const int*)(bpl + up1k((size_t)kOzSlices * np * np * 2));
      if (!cached(s, &mB.b[b], bpl, (uint64_t)np, (uint64_t)np, (uint32_t)NT, (uint64_t)np * np)) {
        g_oz_err = "tensor map encoding failed";
        return cudaErrorInvalidValue;
      }
    }
    dst = s->tmp[mu & 1];
    P.n = n;
    P.n_pad = np;
    P.M2 = M2;
    P.rows = rows;
    P.N = N;
    P.nk = (n + 63) / 64;
    P.n_ntiles = (n + NT - 1) / NT;
    P.tpt = (M2 + BM - 1) / BM;
    P.num_tiles = (int)((mixed ? B * P.tpt : (rows + BM - 1) / BM) * P.n_ntiles);
    P.nbuf = (2 * kOzSlices * NT <= 512) ? 2 : 1;
    P.resident = (P.nk == 1 && P.n_ntiles <= kOzMaxColTiles) ? 1 : 0;
    P.stage_bytes = (uint32_t)kOzSlices * (BM * 128 + (P.resident ? P.n_ntiles : 1) * NT * 128);
    // every pass but the last leaves exact sums for the next split
    P.int_out = (mu + 1 < s->d && N / s->n[mu + 1] < (1ll << 32)) ? 1 : 0;
    int cols = 32;
    while (cols < P.nbuf * kOzSlices * NT) cols <<= 1;
    P.tmem_cols = cols;
    P.out = dst;
    P.xscale = xscale;
    P.mixed = mixed ? 1 : 0;
    P.shared_a = (mu == 0 && shared) ? 1 : 0;
    P.status = s->status;
    if (ev) {
      cudaError_t e = cudaEventRecord(ev[2 * mu], st);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = NT == 16 ? run_oz_gemm<16>(s, mA, mB, P, st) : run_oz_gemm<32>(s, mA, mB, P, st);
    if (e != cudaSuccess) return e;
    if (ev) {
      e = cudaEventRecord(ev[2 * mu + 1], st);
      if (e != cudaSuccess) return e;
    }
    sums_in = P.int_out != 0;
    if (sums_in) {
      std::memset(&sin, 0, sizeof sin);
      sin.S = reinterpret_cast<const long long*>(dst);
      sin.xs = xscale;
      for (int b = 0; b < nmat; ++b) sin.ls[b] = P.lscale[b];
      sin.M2p = M2;
      sin.shared = P.shared_a;
      // (the next pass's fibre count per row; its fibres number below 2^32)
      sin.fpr = (uint32_t)(M2 / s->n[mu + 1]);
      sin.mixed = P.mixed;
    }
    std::memset(&cur, 0, sizeof cur);
    for (int b = 0; b < B; ++b) {
      cur.c[b].nsrc = 1;
      cur.c[b].src[0] = dst + (int64_t)b * N;
      cur.c[b].coef[0] = 1.0;
    }
    cur.ntensor = B;
  }
  if (res) *res = dst;
  if (!epi) return cudaSuccess;
  // the Tucker operators' epilogues over their N elements with the whole GPU
  Epi f[kOzMaxBatch];
  for (int b = 0; b < B; ++b) {
    f[b] = epi[b];
    const int m = f[b].nsrc;
    if (m >= kMaxSrc) return cudaErrorInvalidValue;
    f[b].src[m] = dst + (int64_t)b * N;
    for (int t = 0; t < f[b].nout; ++t) f[b].a[t][m] = epi[b].b[t];
    f[b].nsrc = m + 1;
  }
  for (int b0 = 0; b0 < B; b0 += kMaxEpiBatch) {
    cudaError_t e = launch_combine_batch(f + b0, std::min(kMaxEpiBatch, B - b0), N, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int* oz_status_word(OzState* s) { return s->status; }

void oz_set_ntile(OzState* s, int nt) { s->ntile = (nt == 16 || nt == 32) ? nt : 0; }

int oz_read_status(OzState* s, cudaStream_t st) {
  int h = 0;
  if (cudaMemcpyAsync(&h, s->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  if (h) cudaMemsetAsync(s->status, 0, sizeof(int), st);
  return h;
}

}  // namespace phiks
