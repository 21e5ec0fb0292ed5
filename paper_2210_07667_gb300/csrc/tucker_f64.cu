// FP64 mu-mode product (Sec. 2): W = V x_mu L, with a fused input combination
// (prologue, eq. integrandcomb) and a fused multi-output linear epilogue (the
// quadrature accumulation of eq. integrandsimul / eq. integrandcomb and the
// doubling combinations of eq. simul / eq. comb).
//
// On GB300 the FP64 pipe retires about 2 DFMA per clock per SM (1.19 TFLOP/s
// measured over 152 SMs), two orders of magnitude below the shared-memory and
// L2 bandwidth such a kernel needs, so the design goal is only to keep every
// SM's DFMA pipe fed: many resident warps, independent accumulators per
// thread, and as few FP64 instructions outside the contraction as possible.
//
// The tensor is viewed as (a, n, b) with element (x, j, y) at x + a j + a n y;
// a CTA computes a TI x TC tile of outputs (rows i of L, "columns" c = x + a y)
// by staging KC-deep slices of L and of the fibres V(x, :, y) in shared memory.
#include <atomic>
#include <cstring>

#include "kernels.cuh"
#include "pdl.cuh"

namespace phiks {

namespace {
std::atomic<uint64_t> g_launches{0};
}
uint64_t kernel_launch_count() { return g_launches.load(); }
void count_launch(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {

__device__ __forceinline__ double load_combo(const Combo& pro, int64_t idx, bool plain) {
  if (plain) return __ldg(pro.src[0] + idx);
  double v = pro.coef[0] * __ldg(pro.src[0] + idx);
  for (int m = 1; m < pro.nsrc; ++m) v = fma(pro.coef[m], __ldg(pro.src[m] + idx), v);
  return v;
}

// Kept out of line so that the local arrays of the epilogue do not affect the
// register allocation of the contraction loop.
__device__ __noinline__ void epi_apply_call(const Epi& epi, int64_t idx, double res) {
  epi_apply(epi, idx, res);
}

__device__ __forceinline__ void store_epi(const Epi& epi, double* W, int64_t idx, double res) {
  if (epi.nout == 0) {
    W[idx] = res;
    return;
  }
  epi_apply_call(epi, idx, res);
}

// CTA tile: TI rows of L x TC columns c = x + a y; RI x RC outputs per thread
// (rows ti + r * TI/RI, columns tc + c * TC/RC, so a warp reads consecutive
// shared-memory words); KC-deep slices of L and of the fibres, the next slice
// fetched into registers while the current one is consumed.
template <int TI, int TC, int RI, int RC, int KC, bool XFAST, bool EPI>
__device__ __forceinline__ void mode_product_tile(const Combo& pro, const double* __restrict__ L, ModeGeom g,
                                                  double* W, const Epi* epi) {
  constexpr int TROWS = TI / RI, TCOLS = TC / RC, NT = TROWS * TCOLS;
  constexpr int LPT = (TI * KC + NT - 1) / NT;
  constexpr int VPT = (TC * KC + NT - 1) / NT;
  __shared__ double sL[KC][TI + 1];
  __shared__ double sV[KC][TC + 1];
  const int tid = threadIdx.x;
  const int tc = tid % TCOLS;
  const int ti = tid / TCOLS;
  const int i0 = blockIdx.y * TI;
  const int64_t c0 = (int64_t)blockIdx.x * TC;
  const int64_t ncols = g.a * g.b;
  const int n = g.n;
  const int64_t an = g.a * (int64_t)n;
  const bool plain = (pro.nsrc == 1 && pro.coef[0] == 1.0);

  double rl[LPT], rv[VPT];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int e = 0; e < LPT; ++e) {
      const int idx = tid + e * NT;
      const int ii = idx % TI, kk = idx / TI;
      const int i = i0 + ii, k = k0 + kk;
      rl[e] = (idx < TI * KC && i < n && k < n) ? __ldg(L + i + (int64_t)n * k) : 0.0;
    }
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * NT;
      int cc, kk;
      if (XFAST) {
        cc = idx % TC;
        kk = idx / TC;
      } else {
        kk = idx % KC;
        cc = idx / KC;
      }
      const int64_t c = c0 + cc;
      const int k = k0 + kk;
      double val = 0.0;
      if (idx < TC * KC && c < ncols && k < n) {
        const int64_t x = c % g.a, y = c / g.a;
        val = load_combo(pro, x + g.a * k + an * y, plain);
      }
      rv[e] = val;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int e = 0; e < LPT; ++e) {
      const int idx = tid + e * NT;
      if (idx < TI * KC) sL[idx / TI][idx % TI] = rl[e];
    }
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * NT;
      if (idx < TC * KC) {
        if (XFAST) sV[idx / TC][idx % TC] = rv[e];
        else sV[idx % KC][idx / KC] = rv[e];
      }
    }
  };

  double acc[RI][RC];
#pragma unroll
  for (int r = 0; r < RI; ++r)
#pragma unroll
    for (int c = 0; c < RC; ++c) acc[r][c] = 0.0;

  fetch(0);
  for (int k0 = 0; k0 < n; k0 += KC) {
    stash();
    __syncthreads();
    if (k0 + KC < n) fetch(k0 + KC);
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      double lv[RI], vv[RC];
#pragma unroll
      for (int r = 0; r < RI; ++r) lv[r] = sL[kk][ti + r * TROWS];
#pragma unroll
      for (int c = 0; c < RC; ++c) vv[c] = sV[kk][tc + c * TCOLS];
#pragma unroll
      for (int r = 0; r < RI; ++r)
#pragma unroll
        for (int c = 0; c < RC; ++c) acc[r][c] = fma(lv[r], vv[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < RI; ++r) {
    const int i = i0 + ti + r * TROWS;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < RC; ++c) {
      const int64_t col = c0 + tc + c * TCOLS;
      if (col >= ncols) continue;
      const int64_t x = col % g.a, y = col / g.a;
      if (EPI) store_epi(*epi, W, x + g.a * i + an * y, acc[r][c]);
      else W[x + g.a * i + an * y] = acc[r][c];
    }
  }
}

template <int TI, int TC, int RI, int RC, int KC, bool XFAST>
__global__ void __launch_bounds__((TI / RI) * (TC / RC))
    mode_product_f64_kernel(Combo pro, const double* __restrict__ L, ModeGeom g, double* W, Epi epi) {
  pdl_wait();
  mode_product_tile<TI, TC, RI, RC, KC, XFAST, true>(pro, L, g, W, &epi);
}

// Independent mode products of the same geometry, one per grid layer
// (blockIdx.z), results stored plainly.
template <int TI, int TC, int RI, int RC, int KC, bool XFAST>
__global__ void __launch_bounds__((TI / RI) * (TC / RC))
    mode_product_f64_batch_kernel(const __grid_constant__ ModeBatch mb, ModeGeom g) {
  pdl_wait();
  const int z = blockIdx.z;
  mode_product_tile<TI, TC, RI, RC, KC, XFAST, false>(mb.pro[z], mb.L[z], g, mb.W[z], nullptr);
}

// Complex variant (PHIKS_C128): elements of V and W are interleaved complex
// numbers (element e at doubles 2e, 2e+1); L is the 2n x 2n real
// representation [[Re, -Im], [Im, Re]] of the complex n x n L, so Re L(i, k)
// = L[i + 2n k] and Im L(i, k) = L[n + i + 2n k].  The prologue combination
// and the epilogue take real coefficients and act on both parts.
template <int TI, int TC, int RI, int RC, int KC, bool XFAST>
__global__ void __launch_bounds__((TI / RI) * (TC / RC))
    mode_product_c128_kernel(Combo pro, const double* __restrict__ L, ModeGeom g, double* W, Epi epi) {
  pdl_wait();
  constexpr int TROWS = TI / RI, TCOLS = TC / RC, NT = TROWS * TCOLS;
  constexpr int LPT = (TI * KC + NT - 1) / NT;
  constexpr int VPT = (TC * KC + NT - 1) / NT;
  __shared__ double2 sL[KC][TI + 1];
  __shared__ double2 sV[KC][TC + 1];
  const int tid = threadIdx.x;
  const int tc = tid % TCOLS;
  const int ti = tid / TCOLS;
  const int i0 = blockIdx.y * TI;
  const int64_t c0 = (int64_t)blockIdx.x * TC;
  const int64_t ncols = g.a * g.b;
  const int n = g.n;
  const int64_t m = 2 * (int64_t)n;
  const int64_t an = g.a * (int64_t)n;
  const bool plain = (pro.nsrc == 1 && pro.coef[0] == 1.0);

  double2 rl[LPT], rv[VPT];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int e = 0; e < LPT; ++e) {
      const int idx = tid + e * NT;
      const int ii = idx % TI, kk = idx / TI;
      const int i = i0 + ii, k = k0 + kk;
      double2 v = make_double2(0.0, 0.0);
      if (idx < TI * KC && i < n && k < n) {
        v.x = __ldg(L + i + m * k);
        v.y = __ldg(L + n + i + m * k);
      }
      rl[e] = v;
    }
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * NT;
      int cc, kk;
      if (XFAST) {
        cc = idx % TC;
        kk = idx / TC;
      } else {
        kk = idx % KC;
        cc = idx / KC;
      }
      const int64_t c = c0 + cc;
      const int k = k0 + kk;
      double2 val = make_double2(0.0, 0.0);
      if (idx < TC * KC && c < ncols && k < n) {
        const int64_t x = c % g.a, y = c / g.a;
        const int64_t el = x + g.a * k + an * y;
        val.x = load_combo(pro, 2 * el, plain);
        val.y = load_combo(pro, 2 * el + 1, plain);
      }
      rv[e] = val;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int e = 0; e < LPT; ++e) {
      const int idx = tid + e * NT;
      if (idx < TI * KC) sL[idx / TI][idx % TI] = rl[e];
    }
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * NT;
      if (idx < TC * KC) {
        if (XFAST) sV[idx / TC][idx % TC] = rv[e];
        else sV[idx % KC][idx / KC] = rv[e];
      }
    }
  };

  double2 acc[RI][RC];
#pragma unroll
  for (int r = 0; r < RI; ++r)
#pragma unroll
    for (int c = 0; c < RC; ++c) acc[r][c] = make_double2(0.0, 0.0);

  fetch(0);
  for (int k0 = 0; k0 < n; k0 += KC) {
    stash();
    __syncthreads();
    if (k0 + KC < n) fetch(k0 + KC);
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      double2 lv[RI], vv[RC];
#pragma unroll
      for (int r = 0; r < RI; ++r) lv[r] = sL[kk][ti + r * TROWS];
#pragma unroll
      for (int c = 0; c < RC; ++c) vv[c] = sV[kk][tc + c * TCOLS];
#pragma unroll
      for (int r = 0; r < RI; ++r)
#pragma unroll
        for (int c = 0; c < RC; ++c) {
          acc[r][c].x = fma(lv[r].x, vv[c].x, fma(-lv[r].y, vv[c].y, acc[r][c].x));
          acc[r][c].y = fma(lv[r].x, vv[c].y, fma(lv[r].y, vv[c].x, acc[r][c].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < RI; ++r) {
    const int i = i0 + ti + r * TROWS;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < RC; ++c) {
      const int64_t col = c0 + tc + c * TCOLS;
      if (col >= ncols) continue;
      const int64_t x = col % g.a, y = col / g.a;
      const int64_t el = x + g.a * i + an * y;
      store_epi(epi, W, 2 * el, acc[r][c].x);
      store_epi(epi, W, 2 * el + 1, acc[r][c].y);
    }
  }
}

template <int TI, int TC, int RI, int RC, int KC>
cudaError_t launch_tiled_c128(const Combo& pro, const double* L, ModeGeom g, double* W, const Epi& e,
                              cudaStream_t st) {
  constexpr int NT = (TI / RI) * (TC / RC);
  const int64_t ncols = g.a * g.b;
  dim3 grid((unsigned)((ncols + TC - 1) / TC), (unsigned)((g.n + TI - 1) / TI));
  if (g.a >= TC)
    return launch_pdl(mode_product_c128_kernel<TI, TC, RI, RC, KC, true>, grid, dim3(NT), 0, st, pro, L,
                      g, W, e);
  return launch_pdl(mode_product_c128_kernel<TI, TC, RI, RC, KC, false>, grid, dim3(NT), 0, st, pro, L, g,
                    W, e);
}

template <int TI, int TC, int RI, int RC, int KC>
cudaError_t launch_tiled_batch(const ModeBatch& mb, int B, ModeGeom g, cudaStream_t st) {
  constexpr int NT = (TI / RI) * (TC / RC);
  const int64_t ncols = g.a * g.b;
  dim3 grid((unsigned)((ncols + TC - 1) / TC), (unsigned)((g.n + TI - 1) / TI), (unsigned)B);
  if (g.a >= TC)
    return launch_pdl(mode_product_f64_batch_kernel<TI, TC, RI, RC, KC, true>, grid, dim3(NT), 0, st, mb, g);
  return launch_pdl(mode_product_f64_batch_kernel<TI, TC, RI, RC, KC, false>, grid, dim3(NT), 0, st, mb, g);
}

template <int TI, int TC, int RI, int RC, int KC>
cudaError_t launch_tiled(const Combo& pro, const double* L, ModeGeom g, double* W, const Epi& e,
                         cudaStream_t st) {
  constexpr int NT = (TI / RI) * (TC / RC);
  const int64_t ncols = g.a * g.b;
  dim3 grid((unsigned)((ncols + TC - 1) / TC), (unsigned)((g.n + TI - 1) / TI));
  if (g.a >= TC)
    return launch_pdl(mode_product_f64_kernel<TI, TC, RI, RC, KC, true>, grid, dim3(NT), 0, st, pro, L, g,
                      W, e);
  return launch_pdl(mode_product_f64_kernel<TI, TC, RI, RC, KC, false>, grid, dim3(NT), 0, st, pro, L, g,
                    W, e);
}

struct EpiBatch {
  Epi e[kMaxEpiBatch];
};

// One combination per grid row (blockIdx.y), each over N elements.
__global__ void combine_batch_kernel(EpiBatch eb, int64_t N) {
  pdl_wait();
  const Epi& e = eb.e[blockIdx.y];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N;
       idx += (int64_t)gridDim.x * blockDim.x)
    epi_apply(e, idx, 0.0);
}

// The common case of one output: out = sum_k c_k src_k in FP64 arithmetic,
// sources and output each double or float (the split dtypes' results and
// outputs are float), two elements per thread with 16- or 8-byte loads and
// no local arrays (the general epilogue indexes its sources dynamically,
// which puts them in local memory).
struct Lin1 {
  int nterm;
  unsigned srcf32;  // bit k: src[k] is float
  int outf32;
  const void* src[kMaxSrc];
  double c[kMaxSrc];
  float chi[kMaxSrc], clo[kMaxSrc];  // c = chi + clo (rounded to 48 bits), for lincomb1_f32_kernel
  void* out;
};
struct Lin1Batch {
  Lin1 l[kMaxEpiBatch];
};

__global__ void lincomb1_kernel(Lin1Batch lb, int64_t N2) {
  pdl_wait();
  const Lin1& L = lb.l[blockIdx.y];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N2;
       i += (int64_t)gridDim.x * blockDim.x) {
    double ox = 0.0, oy = 0.0;
    // unrolled by four: four independent loads in flight ahead of their FMAs
#pragma unroll 4
    for (int k = 0; k < L.nterm; ++k) {
      double x0, x1;
      if ((L.srcf32 >> k) & 1) {
        const float2 f = __ldg(reinterpret_cast<const float2*>(L.src[k]) + i);
        x0 = f.x;
        x1 = f.y;
      } else {
        const double2 x = __ldg(reinterpret_cast<const double2*>(L.src[k]) + i);
        x0 = x.x;
        x1 = x.y;
      }
      ox = fma(L.c[k], x0, ox);
      oy = fma(L.c[k], x1, oy);
    }
    if (L.outf32) reinterpret_cast<float2*>(L.out)[i] = make_float2((float)ox, (float)oy);
    else reinterpret_cast<double2*>(L.out)[i] = make_double2(ox, oy);
  }
}

// An all-float combination with a float output (the split dtypes' sums of
// their FP32 Tucker results), in compensated FP32 arithmetic instead of on
// GB300's FP64 pipe (two DFMA per clock per SM against 128 FP32 FMAs): each
// product c x is formed without error as chi x = p + e (the FMA gives e
// exactly) plus clo x, and the running sum is kept as an unevaluated pair
// (hi, lo) with error-free additions (Knuth's two-sum).  The pair carries
// about 44 significant bits, far beyond the float the result is rounded to.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__global__ void lincomb1_f32_kernel(Lin1Batch lb, int64_t N2) {
  pdl_wait();
  const Lin1& L = lb.l[blockIdx.y];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N2;
       i += (int64_t)gridDim.x * blockDim.x) {
    float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
#pragma unroll 4
    for (int k = 0; k < L.nterm; ++k) {
      const float2 x = __ldg(reinterpret_cast<const float2*>(L.src[k]) + i);
      const float ch = L.chi[k], cl = L.clo[k];
      float p, e, s, t;
      p = ch * x.x;
      e = fmaf(ch, x.x, -p) + cl * x.x;
      two_sum(hx, p, s, t);
      hx = s;
      lx += t + e;
      p = ch * x.y;
      e = fmaf(ch, x.y, -p) + cl * x.y;
      two_sum(hy, p, s, t);
      hy = s;
      ly += t + e;
    }
    reinterpret_cast<float2*>(L.out)[i] = make_float2(hx + lx, hy + ly);
  }
}

// One combination as a Lin1 when it has a single output, no product term,
// an even N and pointers aligned for the paired loads and stores.
bool as_lin1(const Epi& e, int64_t N, Lin1* l) {
  if (e.nout != 1 || e.bnz || (N & 1)) return false;
  const bool of = (e.out_f32mask & 1) != 0;
  if (((uintptr_t)e.out[0] & (of ? 7 : 15)) != 0) return false;
  l->nterm = e.nterm;
  l->out = e.out[0];
  l->outf32 = of ? 1 : 0;
  l->srcf32 = 0;
  for (int k = 0; k < e.nterm; ++k) {
    const int m = e.term_m[k];
    const bool sf = ((e.src_f32mask >> m) & 1) != 0;
    l->src[k] = e.src[m];
    l->c[k] = e.term_c[k];
    l->chi[k] = (float)e.term_c[k];
    l->clo[k] = (float)(e.term_c[k] - (double)l->chi[k]);
    if (sf) l->srcf32 |= 1u << k;
    if (((uintptr_t)l->src[k] & (sf ? 7 : 15)) != 0) return false;
  }
  return true;
}

// Several outputs over one list of sources (the pending outputs of a batch,
// which read the same node results with other weights): every source is read
// once for all outputs.  out[t] = sum_k c[t][k] src[k], t < nout <= kLinMOut,
// FP64 arithmetic, or compensated FP32 when every source and output is float.
constexpr int kLinMOut = 4;
struct LinM {
  int nout, nterm;
  unsigned srcf32;
  int outf32;
  const void* src[kMaxSrc];
  double c[kLinMOut][kMaxSrc];
  float chi[kLinMOut][kMaxSrc], clo[kLinMOut][kMaxSrc];
  void* out[kLinMOut];
};
struct LinMBatch {
  LinM l[kMaxEpiBatch];
};

__global__ void lincombm_kernel(const __grid_constant__ LinMBatch lb, int64_t N2) {
  pdl_wait();
  const LinM& L = lb.l[blockIdx.y];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N2;
       i += (int64_t)gridDim.x * blockDim.x) {
    double ox[kLinMOut] = {0.0, 0.0, 0.0, 0.0}, oy[kLinMOut] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 2
    for (int k = 0; k < L.nterm; ++k) {
      double x0, x1;
      if ((L.srcf32 >> k) & 1) {
        const float2 f = __ldg(reinterpret_cast<const float2*>(L.src[k]) + i);
        x0 = f.x;
        x1 = f.y;
      } else {
        const double2 x = __ldg(reinterpret_cast<const double2*>(L.src[k]) + i);
        x0 = x.x;
        x1 = x.y;
      }
#pragma unroll
      for (int t = 0; t < kLinMOut; ++t)
        if (t < L.nout && L.c[t][k] != 0.0) {  // (uniform branches: no predicated-off DFMA)
          ox[t] = fma(L.c[t][k], x0, ox[t]);
          oy[t] = fma(L.c[t][k], x1, oy[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < kLinMOut; ++t)
      if (t < L.nout) {
        if (L.outf32) reinterpret_cast<float2*>(L.out[t])[i] = make_float2((float)ox[t], (float)oy[t]);
        else reinterpret_cast<double2*>(L.out[t])[i] = make_double2(ox[t], oy[t]);
      }
  }
}

__global__ void lincombm_f32_kernel(const __grid_constant__ LinMBatch lb, int64_t N2) {
  pdl_wait();
  const LinM& L = lb.l[blockIdx.y];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N2;
       i += (int64_t)gridDim.x * blockDim.x) {
    float hx[kLinMOut] = {0.f, 0.f, 0.f, 0.f}, lx[kLinMOut] = {0.f, 0.f, 0.f, 0.f};
    float hy[kLinMOut] = {0.f, 0.f, 0.f, 0.f}, ly[kLinMOut] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
    for (int k = 0; k < L.nterm; ++k) {
      const float2 x = __ldg(reinterpret_cast<const float2*>(L.src[k]) + i);
#pragma unroll
      for (int t = 0; t < kLinMOut; ++t) {
        if (t >= L.nout) break;
        const float ch = L.chi[t][k], cl = L.clo[t][k];
        float p, e, sm, tt;
        p = ch * x.x;
        e = fmaf(ch, x.x, -p) + cl * x.x;
        two_sum(hx[t], p, sm, tt);
        hx[t] = sm;
        lx[t] += tt + e;
        p = ch * x.y;
        e = fmaf(ch, x.y, -p) + cl * x.y;
        two_sum(hy[t], p, sm, tt);
        hy[t] = sm;
        ly[t] += tt + e;
      }
    }
#pragma unroll
    for (int t = 0; t < kLinMOut; ++t)
      if (t < L.nout) reinterpret_cast<float2*>(L.out[t])[i] = make_float2(hx[t] + lx[t], hy[t] + ly[t]);
  }
}

// A combination with 1..kLinMOut outputs as a LinM: no product term, every
// output of one element type, an even N, aligned pointers.
bool as_linm(const Epi& e, int64_t N, LinM* l) {
  if (e.nout < 1 || e.nout > kLinMOut || e.bnz || (N & 1)) return false;
  const bool of = (e.out_f32mask & 1) != 0;
  if (e.out_f32mask != (of ? (1 << e.nout) - 1 : 0)) return false;
  std::memset(l, 0, sizeof *l);
  l->nout = e.nout;
  l->nterm = e.nsrc;
  l->outf32 = of ? 1 : 0;
  for (int t = 0; t < e.nout; ++t) {
    l->out[t] = e.out[t];
    if (((uintptr_t)e.out[t] & (of ? 7 : 15)) != 0) return false;
  }
  for (int m = 0; m < e.nsrc; ++m) {
    const bool sf = ((e.src_f32mask >> m) & 1) != 0;
    l->src[m] = e.src[m];
    if (sf) l->srcf32 |= 1u << m;
    if (((uintptr_t)e.src[m] & (sf ? 7 : 15)) != 0) return false;
    for (int t = 0; t < e.nout; ++t) {
      l->c[t][m] = e.a[t][m];
      l->chi[t][m] = (float)e.a[t][m];
      l->clo[t][m] = (float)(e.a[t][m] - (double)l->chi[t][m]);
    }
  }
  return true;
}

__global__ void combine_kernel(Epi e, int64_t N) {
  pdl_wait();
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N;
       idx += (int64_t)gridDim.x * blockDim.x)
    epi_apply(e, idx, 0.0);
}

struct PtrArray {
  const void* p[kMaxSrc];
};

__global__ void sumsq_kernel_arr(PtrArray xs, int64_t N, int is_f32, double* out) {
  pdl_wait();
  const int k = blockIdx.y;
  double s = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double v = is_f32 ? (double)((const float*)xs.p[k])[idx] : ((const double*)xs.p[k])[idx];
    s = fma(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out + k, s);
  }
}

int grid_for(int64_t N, int threads) {
  int64_t g = (N + threads - 1) / threads;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t launch_mode_product_f64(const Combo& pro, const double* L, ModeGeom g, double* W,
                                    const Epi* epi, cudaStream_t st, int tile) {
  Epi e;
  if (epi) {
    e = *epi;
  } else {
    e.nout = 0;
    e.nsrc = 0;
  }
  epi_finalize(e);
  count_launch();
  // Large problems: 32 x 64 tiles (256 threads, 8 outputs each).  Otherwise
  // 16 x 16 tiles (64 threads, 4 outputs each), so that even N = 2^18 spreads
  // over ~1000 CTAs and the 152 SMs' FP64 pipes stay evenly loaded.
  const int64_t big_tiles = ((g.a * g.b + 63) / 64) * ((g.n + 31) / 32);
  if (tile == 2 || (tile == 0 && big_tiles >= 8 * 152)) return launch_tiled<32, 64, 2, 4, 16>(pro, L, g, W, e, st);
  return launch_tiled<16, 16, 2, 2, 32>(pro, L, g, W, e, st);
}

cudaError_t launch_mode_product_f64_batch(const ModeBatch& mb, int B, ModeGeom g, cudaStream_t st, int tile) {
  if (B < 1 || B > kMaxModeBatch) return cudaErrorInvalidValue;
  count_launch();
  const int64_t big_tiles = B * ((g.a * g.b + 63) / 64) * ((g.n + 31) / 32);
  if (tile == 2 || (tile == 0 && big_tiles >= 8 * 152)) return launch_tiled_batch<32, 64, 2, 4, 16>(mb, B, g, st);
  return launch_tiled_batch<16, 16, 2, 2, 32>(mb, B, g, st);
}

cudaError_t launch_mode_product_c128(const Combo& pro, const double* L, ModeGeom g, double* W,
                                     const Epi* epi, cudaStream_t st) {
  Epi e;
  if (epi) {
    e = *epi;
  } else {
    e.nout = 0;
    e.nsrc = 0;
  }
  epi_finalize(e);
  count_launch();
  // four DFMA per complex product: the small tiles already give ~1000 CTAs
  // at N = 2^18, the large ones when there are eight per SM
  const int64_t big_tiles = ((g.a * g.b + 63) / 64) * ((g.n + 31) / 32);
  if (big_tiles >= 8 * 152) return launch_tiled_c128<32, 64, 2, 4, 16>(pro, L, g, W, e, st);
  return launch_tiled_c128<16, 16, 2, 2, 32>(pro, L, g, W, e, st);
}

cudaError_t launch_combine_batch(const Epi* e0, int B, int64_t N, cudaStream_t st) {
  if (N <= 0 || B <= 0) return cudaSuccess;
  if (B > kMaxEpiBatch) return cudaErrorInvalidValue;
  EpiBatch eb;
  Lin1Batch lb;
  bool lin = true, linm = true;
  LinMBatch mb;
  for (int b = 0; b < B; ++b) {
    eb.e[b] = e0[b];
    for (int t = 0; t < kMaxOut; ++t) eb.e[b].b[t] = 0.0;  // no product result here
    epi_finalize(eb.e[b]);
    lin = lin && as_lin1(eb.e[b], N, &lb.l[b]);
    linm = linm && as_linm(eb.e[b], N, &mb.l[b]);
  }
  count_launch();
  if (linm && !lin) {
    int gx = grid_for(N / 2, 256) / B;
    if (gx < 1) gx = 1;
    bool f32 = true;
    for (int b = 0; b < B; ++b)
      f32 = f32 && mb.l[b].outf32 && mb.l[b].srcf32 == (1u << mb.l[b].nterm) - 1;
    if (f32) return launch_pdl(lincombm_f32_kernel, dim3(gx, B), dim3(256), 0, st, mb, N / 2);
    return launch_pdl(lincombm_kernel, dim3(gx, B), dim3(256), 0, st, mb, N / 2);
  }
  if (lin) {
    int gx = grid_for(N / 2, 256) / B;
    if (gx < 1) gx = 1;
    bool f32 = true;  // every combination all-float with a float output
    for (int b = 0; b < B; ++b)
      f32 = f32 && lb.l[b].outf32 && lb.l[b].srcf32 == (lb.l[b].nterm >= 32 ? ~0u : (1u << lb.l[b].nterm) - 1);
    if (f32) return launch_pdl(lincomb1_f32_kernel, dim3(gx, B), dim3(256), 0, st, lb, N / 2);
    return launch_pdl(lincomb1_kernel, dim3(gx, B), dim3(256), 0, st, lb, N / 2);
  }
  int gx = grid_for(N, 256) / B;
  if (gx < 1) gx = 1;
  return launch_pdl(combine_batch_kernel, dim3(gx, B), dim3(256), 0, st, eb, N);
}

cudaError_t launch_combine(const Epi& e0, int64_t N, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  Epi e = e0;
  e.nout = e0.nout;
  for (int t = 0; t < kMaxOut; ++t) e.b[t] = 0.0;  // no product result here
  epi_finalize(e);
  Lin1Batch lb;
  if (as_lin1(e, N, &lb.l[0])) {
    count_launch();
    const Lin1& l = lb.l[0];
    if (l.outf32 && l.nterm > 0 && l.srcf32 == (1u << l.nterm) - 1)
      return launch_pdl(lincomb1_f32_kernel, dim3(grid_for(N / 2, 256)), dim3(256), 0, st, lb, N / 2);
    return launch_pdl(lincomb1_kernel, dim3(grid_for(N / 2, 256)), dim3(256), 0, st, lb, N / 2);
  }
  count_launch();
  return launch_pdl(combine_kernel, dim3(grid_for(N, 256)), dim3(256), 0, st, e, N);
}

cudaError_t launch_sumsq(const void* const* x, int count, int64_t N, int is_f32, double* out,
                         cudaStream_t st) {
  if (count <= 0 || N <= 0) return cudaSuccess;
  if (count > kMaxSrc) return cudaErrorInvalidValue;
  PtrArray a;
  for (int k = 0; k < count; ++k) a.p[k] = x[k];
  dim3 grid(grid_for(N, 256) > 304 ? 304 : grid_for(N, 256), count);
  count_launch();
  return launch_pdl(sumsq_kernel_arr, grid, dim3(256), 0, st, a, N, is_f32, out);
}

}  // namespace phiks
