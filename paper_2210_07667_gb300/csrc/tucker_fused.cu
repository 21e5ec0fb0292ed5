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
//
// An input that is a combination of several tensors (the deferred FP64
// combinations of the previous batch) costs one DFMA per source and element;
// formed by every CTA of a tensor it would cost n_d / nj times the whole
// combination.  The chunks of a tensor are therefore launched as thread-block
// clusters: each CTA of a cluster forms 1/C of the elements into its shared
// memory and copies the other slices from its peers' shared memory
// (distributed shared memory), so the combination is formed once per cluster.
#include <cooperative_groups.h>

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
  int stageV;     // the whole input staged in shared memory first (small N)
};

// A combination's value at idx: every source load issued before the first
// multiply-add (the loads of one element are independent).
__device__ __forceinline__ double combo_at(const Combo& c, int64_t idx) {
  if (c.nsrc == 1 && c.f32mask == 0 && c.coef[0] == 1.0) return __ldg(c.src[0] + idx);
  double x[kMaxSrc];
#pragma unroll
  for (int m = 0; m < kMaxSrc; ++m)
    if (m < c.nsrc)
      x[m] = ((c.f32mask >> m) & 1) ? (double)__ldg((const float*)c.src[m] + idx) : __ldg(c.src[m] + idx);
  double v = 0.0;
#pragma unroll
  for (int m = 0; m < kMaxSrc; ++m)
    if (m < c.nsrc) v = fma(c.coef[m], x[m], v);
  return v;
}

// 8-byte asynchronous copy global -> shared (LDGSTS): the thread does not
// wait for it, so every copy of a staging phase is in flight at once.
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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
  double* sV = S1 + (size_t)M * NJ;      // the input, when staged (N doubles)

  // matrices (and a plain small input) copied asynchronously, all in flight
  // together
  const Combo& pro = fb.pro[b];
  double* const store = fb.store[b];
  const bool plain = pro.nsrc == 1 && pro.f32mask == 0 && pro.coef[0] == 1.0;
  const double* Ld = fb.L[b][d - 1];
  for (int e = tid; e < NJ * nl; e += T) {
    const int jj = e / nl, k = e - jj * nl;
    if (jj < njc) cp_async8(sLd + e, Ld + (j0 + jj) + (int64_t)nl * k);
    else sLd[e] = 0.0;
  }
  if (g.stageL)
    for (int mu = 0; mu + 1 < d; ++mu) {
      const int n2 = g.n[mu] * g.n[mu];
      const double* L = fb.L[b][mu];
      for (int e = tid; e < n2; e += T) cp_async8(sL + g.lofs[mu] + e, L + e);
    }
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();       // CTAs of this tensor's cluster (1 without)
  const int crank = (int)cluster.block_rank();
  if (g.stageV) {
    // small tensors: the whole input in shared memory (each CTA needs all of
    // it for its rows of the slowest mode)
    if (plain) {
      for (int e = tid; e < (int)g.N; e += T) cp_async8(sV + e, pro.src[0] + e);
    } else {
      // this CTA's slice of the combination (independent loads), the
      // cluster's other slices from its peers
      const int e0 = (int)(g.N * crank / C), e1 = (int)(g.N * (crank + 1) / C);
      const bool first_cluster = chunk < C;  // stores each element once per tensor
#pragma unroll 4
      for (int e = e0 + tid; e < e1; e += T) {
        const double v = combo_at(pro, e);
        sV[e] = v;
        if (store && first_cluster) store[e] = v;
      }
      if (C > 1) {
        cluster.sync();  // every slice written (and visible in the cluster)
        for (int r = 0; r < C; ++r) {
          if (r == crank) continue;
          const int r0 = (int)(g.N * r / C), r1 = (int)(g.N * (r + 1) / C);
          const double* peer = cluster.map_shared_rank(sV, r);
          for (int e = r0 + tid; e < r1; e += T) sV[e] = peer[e];
        }
        cluster.sync();  // no CTA leaves while a peer may still read its slice
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // slowest mode, this chunk's rows: S0(x, jj) = sum_k V(x + M k) L_d(j0 + jj, k)
  if (g.stageV) {
    if (store && plain)  // element x + M k is stored by the CTA of chunk k mod nchunks
      for (int e = tid; e < (int)g.N; e += T)
        if ((e / M) % g.nchunks == chunk) store[e] = sV[e];
    for (int x = tid; x < M; x += T) {
      double acc[NJ];
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) acc[jj] = 0.0;
#pragma unroll 4
      for (int k = 0; k < nl; ++k) {
        const double v = sV[x + M * k];
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) acc[jj] = fma(sLd[jj * nl + k], v, acc[jj]);
      }
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj)
        if (jj < njc) S0[x + M * jj] = acc[jj];
    }
  } else {
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

  // the deferred combinations of the previous batch (elementwise over N, off
  // the critical path), spread over every CTA of the grid
  if (fb.nside) {
    const int64_t cta = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    const int64_t ncta = (int64_t)gridDim.x * gridDim.y;
    const int64_t items = (int64_t)fb.nside * g.N;  // (combination, element) pairs
    for (int64_t it = cta * T + tid; it < items; it += ncta * T) {
      const int s = (int)(it / g.N);
      const int64_t i = it - (int64_t)s * g.N;
      fb.side_out[s][i] = combo_at(fb.side[s], i);
    }
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
  const int threads = g.stageV ? 128 : std::min(kFusedThreads, std::max(64, (g.M + 31) / 32 * 32));
  // clusters of the chunks of a tensor (a power of two <= 8 dividing the
  // chunk count) when some input is a combination to form in shared memory
  int csize = 1;
  bool combos = false;
  for (int b = 0; b < fb.B; ++b)
    combos = combos || !(fb.pro[b].nsrc == 1 && fb.pro[b].f32mask == 0 && fb.pro[b].coef[0] == 1.0);
  if (g.stageV && combos)
    while (csize < 8 && g.nchunks % (2 * csize) == 0) csize *= 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g.nchunks, fb.B);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  at[1].id = cudaLaunchAttributeClusterDimension;
  at[1].val.clusterDim.x = csize;
  at[1].val.clusterDim.y = 1;
  at[1].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, fb, g, e);
}

// Shared memory of one CTA; *stageL / *stageV say whether the matrices and
// the whole input are staged there (inputs of at most kStageVMax elements).
constexpr int64_t kStageVMax = 8192;
size_t fused_smem(int d, const int64_t* n, int64_t N, int nj, int* stageL, int* stageV = nullptr) {
  const int64_t nl = n[d - 1];
  const int64_t M = N / nl;
  size_t Lsum = 0;
  for (int mu = 0; mu + 1 < d; ++mu) Lsum += (size_t)n[mu] * n[mu];
  *stageL = Lsum * 8 <= 64 * 1024 ? 1 : 0;
  const int sv = N <= kStageVMax ? 1 : 0;
  if (stageV) *stageV = sv;
  return ((size_t)nj * nl + (*stageL ? Lsum : 0) + 2 * (size_t)M * nj + (sv ? (size_t)N : 0)) * 8;
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
  const size_t smem = fused_smem(d, n, N, nj, &g.stageL, &g.stageV);
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
