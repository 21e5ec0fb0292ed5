// Small dense FP64 matrices: batched GEMM with an identity term and batched
// scaling, the building blocks of the truncated-Taylor scaling-and-squaring
// exponential of the small matrices (1 - theta_i) tau A_mu / 2^s (Sec. 3.1,
// eq. Tuckerprod) and of the squaring chain exp(A_mu/2^(j-1)) =
// exp(A_mu/2^j)^2 (eq. simul, eq. comb).
#include "kernels.cuh"
#include "pdl.cuh"

namespace phiks {
namespace {

constexpr int GK = 16;

// One CTA per GT x GT tile of one C_k, (GT / GR)^2 threads with GR x GR
// outputs each.  The FP64 pipe bounds this kernel, so small matrices take
// small tiles to spread over every SM.
template <int GT, int GR>
__global__ void __launch_bounds__((GT / GR) * (GT / GR)) gemm_batch_f64_kernel(GemmBatch gb) {
  pdl_wait();
  constexpr int GTHR = GT / GR;
  constexpr int GNT = GTHR * GTHR;
  const int k = blockIdx.z;
  const int n = gb.n[k];
  const int tiles = (n + GT - 1) / GT;
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (bi >= tiles || bj >= tiles) return;
  const double* __restrict__ A = gb.A[k];
  const double* __restrict__ B = gb.B[k];
  double* C = gb.C[k];
  __shared__ double sA[GK][GT + 1];   // sA[kk][ii] = A[i0+ii, k0+kk]
  __shared__ double sB[GK][GT + 1];   // sB[kk][jj] = B[k0+kk, j0+jj]
  const int tid = threadIdx.x;
  const int tj = tid % GTHR, ti = tid / GTHR;
  const int i0 = bi * GT, j0 = bj * GT;
  double acc[GR][GR];
#pragma unroll
  for (int r = 0; r < GR; ++r)
#pragma unroll
    for (int c = 0; c < GR; ++c) acc[r][c] = 0.0;
  const int kend = gb.alpha[k] != 0.0 ? n : 0;  // alpha = 0: addends only
  for (int k0 = 0; k0 < kend; k0 += GK) {
    for (int e = tid; e < GT * GK; e += GNT) {
      int ii = e % GT, kk = e / GT;
      int i = i0 + ii, kc = k0 + kk;
      sA[kk][ii] = (i < n && kc < n) ? A[i + (int64_t)n * kc] : 0.0;
      int kr = k0 + (e % GK), jj = e / GK, j = j0 + jj;
      sB[e % GK][jj] = (kr < n && j < n) ? B[kr + (int64_t)n * j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[GR], b[GR];
#pragma unroll
      for (int r = 0; r < GR; ++r) {
        a[r] = sA[kk][ti + r * GTHR];
        b[r] = sB[kk][tj + r * GTHR];
      }
#pragma unroll
      for (int r = 0; r < GR; ++r)
#pragma unroll
        for (int c = 0; c < GR; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  const double alpha = gb.alpha[k], beta = gb.beta_I[k];
#pragma unroll
  for (int r = 0; r < GR; ++r)
#pragma unroll
    for (int c = 0; c < GR; ++c) {
      int i = i0 + ti + r * GTHR, j = j0 + tj + c * GTHR;
      if (i < n && j < n) {
        const int64_t e = i + (int64_t)n * j;
        double v = alpha * acc[r][c] + (i == j ? beta : 0.0);
        for (int a = 0; a < 3; ++a)
          if (gb.addm[k][a]) v = fma(gb.addc[k][a], gb.addm[k][a][e], v);
        C[e] = v;
      }
    }
}

__global__ void poly_batch_f64_kernel(const __grid_constant__ PolyBatch pb) {
  pdl_wait();
  const int k = blockIdx.y;
  const int n = pb.n[k], m = pb.m[k];
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
       e += (int64_t)gridDim.x * blockDim.x) {
    double x[kPolyMax];  // all loads issued before the sum
#pragma unroll
    for (int i = 0; i < kPolyMax; ++i) x[i] = i < m ? __ldg(pb.P[k][i] + e) : 0.0;
    double v = 0.0;
#pragma unroll
    for (int i = kPolyMax; i >= 1; --i)
      if (i <= m) v = fma(pb.c[k][i], x[i - 1], v);
    if (e % n == e / n) v += pb.c[k][0];
    pb.Y[k][e] = v;
  }
}

}  // namespace

cudaError_t launch_poly_batch_f64(const PolyBatch& pb, int nmax, cudaStream_t st) {
  if (pb.count <= 0) return cudaSuccess;
  if (pb.count > kPolyBatch) return cudaErrorInvalidValue;
  const int64_t nn = (int64_t)nmax * nmax;
  const int gx = (int)std::min<int64_t>((nn + 255) / 256, 64);
  count_launch();
  return launch_pdl(poly_batch_f64_kernel, dim3(gx, pb.count), dim3(256), 0, st, pb);
}

cudaError_t launch_gemm_batch_f64(const GemmBatch& gb, int nmax, cudaStream_t st) {
  if (gb.count <= 0) return cudaSuccess;
  if (gb.count > kMaxBatch) return cudaErrorInvalidValue;
  // the largest tile that still gives every SM a few CTAs
  auto ctas = [&](int gt) { return (int64_t)gb.count * ((nmax + gt - 1) / gt) * ((nmax + gt - 1) / gt); };
  count_launch();
  if (ctas(32) >= 4 * 152) {
    const int t = (nmax + 31) / 32;
    return launch_pdl(gemm_batch_f64_kernel<32, 2>, dim3(t, t, gb.count), dim3(256), 0, st, gb);
  } else if (ctas(16) >= 4 * 152) {
    const int t = (nmax + 15) / 16;
    return launch_pdl(gemm_batch_f64_kernel<16, 1>, dim3(t, t, gb.count), dim3(256), 0, st, gb);
  } else {
    const int t = (nmax + 7) / 8;
    return launch_pdl(gemm_batch_f64_kernel<8, 1>, dim3(t, t, gb.count), dim3(64), 0, st, gb);
  }
}

}  // namespace phiks
