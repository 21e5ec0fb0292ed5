// Fused small-slab Tucker operator in FP64 (Sec. 2, the Tucker operator; the
// batches of independent operators of eq. integrandsimul / eq. integrandcomb):
// all d mu-mode products of a tensor in one kernel, the intermediates held in
// shared memory instead of global temporaries, and the batch's input
// combinations, stores and extra combinations (the deferred FP64
// combinations of the previous batch) in the same launch.
//
// Work split.  The modes commute, so a CTA takes the slowest mode first,
// restricted to a chunk J of nj of its output rows:
//     U(x, jj) = sum_k V(x, k) L_d(j0 + jj, k),   x < M = N / n_d,
// which needs the whole input but produces a slab of M nj elements whose
// fibres along modes 1 .. d-1 are all inside the slab; those modes are then
// applied in shared memory.  Summed over the n_d / nj chunks of a tensor this
// is exactly the flop count of the unfused operator (2 N sum n_mu); only the
// input is read once per chunk (from L2: the tensors it is chosen for are
// small).  The FP64 pipe (2 DFMA per clock per SM) bounds the arithmetic, so
// the loops only need enough independent loads in flight.
#include <algorithm>
#include <cstring>

#include "kernels.cuh"
#include "pdl.cuh"

namespace phiks {

namespace {

constexpr int kFusedThreads = 256;

struct FusedGeom {
  int d;
  int n[kFusedMaxD];
  int64_t N;
  int M;          // N / n_d
  int nchunks;    // chunks of the last mode
  int stageL;     // L_1 .. L_{d-1} staged in shared memory
  int lofs[kFusedMaxD];  // their offsets there (doubles)
  int lsize;      // doubles taken by the staged L
};

__device__ __forceinline__ double combo_at(const Combo& c, int64_t idx) {
  if (c.nsrc == 1 && c.f32mask == 0 && c.coef[0] == 1.0) return __ldg(c.src[0] + idx);
  double v = 0.0;
  for (int m = 0; m < c.nsrc; ++m) {
    const double x = ((c.f32mask >> m) & 1) ? (double)__ldg((const float*)c.src[m] + idx) : __ldg(c.src[m] + idx);
    v = fma(c.coef[m], x, v);
  }
  return v;
}

// Kept out of line: the epilogue's local arrays stay out of the main loops.
__device__ __noinline__ void fused_epi(const Epi& e, int64_t idx, double res) { epi_apply(e, idx, res); }

template <int NJ, bool EPI>
__global__ void __launch_bounds__(kFusedThreads)
    tucker_fused_f64_kernel(const __grid_constant__ FusedBatch fb, const __grid_constant__ FusedGeom g,
                            const __grid_constant__ Epi epi) {
  extern __shared__ __align__(16) double sm[];
  pdl_wait();
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int b = blockIdx.y;
  const int chunk = blockIdx.x;
  const int d = g.d;
  const int nl = g.n[d - 1];
  const int M = g.M;
  const int j0 = chunk * NJ;
  const int njc = min(NJ, nl - j0);
  double* sLd = sm;                      // NJ x nl: rows j0.. of L_d
  double* sL = sLd + NJ * nl;            // staged L_1 .. L_{d-1}
  double* S0 = sL + g.lsize;            // slab, M x NJ
  double* S1 = S0 + (size_t)M * NJ;

  // the deferred combinations of the previous batch (elementwise over N),
  // spread over every CTA of the grid
  if (fb.nside) {
    const int64_t cta = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    const int64_t ncta = (int64_t)gridDim.x * gridDim.y;
    for (int s = 0; s < fb.nside; ++s)
      for (int64_t i = cta * T + tid; i < g.N; i += ncta * T) fb.side_out[s][i] = combo_at(fb.side[s], i);
  }

  const double* Ld = fb.L[b][d - 1];
  for (int e = tid; e < NJ * nl; e += T) {
    const int jj = e / nl, k = e - jj * nl;
    sLd[e] = jj < njc ? __ldg(Ld + (j0 + jj) + (int64_t)nl * k) : 0.0;
  }
  if (g.stageL)
    for (int mu = 0; mu + 1 < d; ++mu) {
      const int n2 = g.n[mu] * g.n[mu];
      const double* L = fb.L[b][mu];
      for (int e = tid; e < n2; e += T) sL[g.lofs[mu] + e] = __ldg(L + e);
    }
  __syncthreads();

  // slowest mode, this chunk's rows: S0(x, jj) = sum_k V(x + M k) L_d(j0 + jj, k)
  const Combo& pro = fb.pro[b];
  double* const store = fb.store[b];
  for (int x = tid; x < M; x += T) {
    double acc[NJ];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) acc[jj] = 0.0;
#pragma unroll 4
    for (int k = 0; k < nl; ++k) {
      const int64_t idx = x + (int64_t)M * k;
      const double v = combo_at(pro, idx);
      if (store && k % g.nchunks == chunk) store[idx] = v;  // each element stored by one CTA
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) acc[jj] = fma(sLd[jj * nl + k], v, acc[jj]);
    }
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj)
      if (jj < njc) S0[x + M * jj] = acc[jj];
  }
  __syncthreads();

  // modes 1 .. d-1 inside the slab (M njc elements, x + M jj)
  double* cur = S0;
  double* nxt = S1;
  const int tot = M * njc;
  int a = 1;
  for (int mu = 0; mu + 1 < d; ++mu) {
    const int n = g.n[mu];
    const int an = a * n;
    const double* L = g.stageL ? sL + g.lofs[mu] : fb.L[b][mu];
    for (int o = tid; o < tot; o += T) {
      const int x = o % a;
      const int r = o / a;
      const int i = r % n;
      const int y = r / n;
      const double* in = cur + x + an * y;
      double acc = 0.0;
      if (g.stageL) {
#pragma unroll 8
        for (int k = 0; k < n; ++k) acc = fma(L[i + n * k], in[a * k], acc);
      } else {
#pragma unroll 8
        for (int k = 0; k < n; ++k) acc = fma(__ldg(L + i + n * k), in[a * k], acc);
      }
      nxt[o] = acc;
    }
    __syncthreads();
    double* t = cur;
    cur = nxt;
    nxt = t;
    a = an;
  }

  // the slab is elements M j0 .. M j0 + tot - 1 of the result
  const int64_t base = (int64_t)M * j0;
  if (EPI) {
    for (int o = tid; o < tot; o += T) fused_epi(epi, base + o, cur[o]);
  } else {
    double* W = fb.W[b] + base;
    for (int o = tid; o < tot; o += T) W[o] = cur[o];
  }
}

template <int NJ, bool EPI>
cudaError_t launch_nj(const FusedBatch& fb, const FusedGeom& g, const Epi& e, size_t smem, cudaStream_t st) {
  auto kern = tucker_fused_f64_kernel<NJ, EPI>;
  static int set_bytes[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem > 48 * 1024 && set_bytes[dev] < (int)smem) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedMaxSmem);
    if (err != cudaSuccess) return err;
    set_bytes[dev] = kFusedMaxSmem;
  }
  const int threads = std::min(kFusedThreads, std::max(64, (g.M + 31) / 32 * 32));
  count_launch();
  return launch_pdl(kern, dim3(g.nchunks, fb.B), dim3(threads), smem, st, fb, g, e);
}

size_t fused_smem(int d, const int64_t* n, int64_t N, int nj, int* stageL) {
  const int64_t nl = n[d - 1];
  const int64_t M = N / nl;
  size_t Lsum = 0;
  for (int mu = 0; mu + 1 < d; ++mu) Lsum += (size_t)n[mu] * n[mu];
  *stageL = Lsum * 8 <= 64 * 1024 ? 1 : 0;
  return ((size_t)nj * nl + (*stageL ? Lsum : 0) + 2 * (size_t)M * nj) * 8;
}

}  // namespace

bool fused_f64_ok(int d, const int64_t* n, int64_t N) {
  if (d < 2 || d > kFusedMaxD || N > kFusedMaxN) return false;
  int st = 0;
  return fused_smem(d, n, N, 1, &st) <= (size_t)kFusedMaxSmem;
}

int fused_f64_default_nj(int d, const int64_t* n, int64_t N, int B) {
  // about two CTAs per SM over the batch, the largest power of two <= 8
  // rows per chunk that keeps that many chunks and fits shared memory
  const int64_t nl = n[d - 1];
  const int64_t want = (2 * 152 + B - 1) / std::max(B, 1);
  int nj = 8;
  int st = 0;
  while (nj > 1 && ((nl + nj - 1) / nj < want || fused_smem(d, n, N, nj, &st) > (size_t)kFusedMaxSmem / 2))
    nj >>= 1;
  return nj;
}

cudaError_t launch_tucker_fused_f64(const FusedBatch& fb, int d, const int64_t* n, int64_t N, int nj,
                                    const Epi* epi, cudaStream_t st) {
  if (!fused_f64_ok(d, n, N) || fb.B < 1 || fb.B > kMaxModeBatch || fb.nside < 0 || fb.nside > kFusedMaxSide)
    return cudaErrorInvalidValue;
  if (nj != 1 && nj != 2 && nj != 4 && nj != 8) return cudaErrorInvalidValue;
  {  // fewer rows per CTA when the slab would not fit shared memory
    int st = 0;
    while (nj > 1 && fused_smem(d, n, N, nj, &st) > (size_t)kFusedMaxSmem) nj >>= 1;
  }
  FusedGeom g;
  std::memset(&g, 0, sizeof g);
  g.d = d;
  for (int mu = 0; mu < d; ++mu) g.n[mu] = (int)n[mu];
  g.N = N;
  g.M = (int)(N / n[d - 1]);
  g.nchunks = (int)((n[d - 1] + nj - 1) / nj);
  const size_t smem = fused_smem(d, n, N, nj, &g.stageL);
  if (smem > (size_t)kFusedMaxSmem) return cudaErrorInvalidValue;
  int off = 0;
  for (int mu = 0; mu + 1 < d; ++mu) {
    g.lofs[mu] = off;
    off += (int)(n[mu] * n[mu]);
  }
  g.lsize = g.stageL ? off : 0;
  Epi e;
  if (epi) {
    e = *epi;
  } else {
    std::memset(&e, 0, sizeof e);
  }
  epi_finalize(e);
  const bool E = epi && epi->nout > 0;
  switch (nj) {
    case 1: return E ? launch_nj<1, true>(fb, g, e, smem, st) : launch_nj<1, false>(fb, g, e, smem, st);
    case 2: return E ? launch_nj<2, true>(fb, g, e, smem, st) : launch_nj<2, false>(fb, g, e, smem, st);
    case 4: return E ? launch_nj<4, true>(fb, g, e, smem, st) : launch_nj<4, false>(fb, g, e, smem, st);
    default: return E ? launch_nj<8, true>(fb, g, e, smem, st) : launch_nj<8, false>(fb, g, e, smem, st);
  }
}

}  // namespace phiks
