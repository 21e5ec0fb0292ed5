// Device-side building blocks of the phiks hot path and their launchers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace phiks {

// Sets the message phiks_last_error() returns on this thread.
void set_error_message(const char* msg);

// Process-wide count of kernels launched by this library.
uint64_t kernel_launch_count();
// dtype of a plan (phiks_dtype), -1 for NULL
int plan_dtype(const void* plan);
void count_launch(uint64_t k = 1);

constexpr int kMaxSrc = 12;  // tensors one combination may read (all nodes of q <= 12 and one more)
constexpr int kMaxOut = 8;   // tensors one epilogue may write

// Input of a mu-mode product as a linear combination of tensors:
//   x[idx] = sum_m coef[m] * src[m][idx]        (nsrc >= 1)
// (the prologue of eq. integrandcomb; a plain input is nsrc = 1, coef = 1).
struct Combo {
  int nsrc;
  int f32mask;                 // bit m set: src[m] holds float, else double
  const double* src[kMaxSrc];  // typed by f32mask
  double coef[kMaxSrc];
};

// Output stage shared by the Tucker epilogue and the elementwise kernel:
//   out[t][idx] = b[t] * result + sum_m a[t][m] * src[m][idx],  t < nout.
// With nout == 0 the result is stored to the kernel's plain output.  An out[t]
// may equal a src[m]: each element is read before it is written by the same
// thread.
struct Epi {
  int nout;
  int nsrc;
  int out_f32mask;             // bit t set: out[t] is float (FP64 arithmetic, rounded once)
  int src_f32mask;             // bit m set: src[m] is float
  double* out[kMaxOut];        // typed by out_f32mask
  const double* src[kMaxSrc];
  double b[kMaxOut];
  double a[kMaxOut][kMaxSrc];
  // filled by epi_finalize (the launchers call it): the nonzero a[t][m] as a
  // flat list of terms, so that device code issues exactly one FP64 FMA per
  // term (predicated-off FP64 instructions would still occupy the slow FP64
  // pipe), and bit t of bnz set when b[t] != 0
  int nterm;
  unsigned char term_t[kMaxOut * kMaxSrc];
  unsigned char term_m[kMaxOut * kMaxSrc];
  double term_c[kMaxOut * kMaxSrc];
  unsigned char bnz;
};

inline void epi_finalize(Epi& e) {
  e.bnz = 0;
  e.nterm = 0;
  for (int t = 0; t < e.nout && t < kMaxOut; ++t) {
    if (e.b[t] != 0.0) e.bnz |= (unsigned char)(1u << t);
    for (int m = 0; m < e.nsrc && m < kMaxSrc; ++m)
      if (e.a[t][m] != 0.0) {
        e.term_t[e.nterm] = (unsigned char)t;
        e.term_m[e.nterm] = (unsigned char)m;
        e.term_c[e.nterm] = e.a[t][m];
        e.nterm++;
      }
  }
}

// out[t][idx] for every output of `e`, given the product result `res`
// (device helper shared by the epilogues).
#ifdef __CUDACC__
__device__ __forceinline__ void epi_apply(const Epi& e, int64_t idx, double res) {
  double sv[kMaxSrc];
  double o[kMaxOut];
#pragma unroll 1
  for (int m = 0; m < e.nsrc; ++m)
    sv[m] = ((e.src_f32mask >> m) & 1) ? (double)((const float*)e.src[m])[idx] : e.src[m][idx];
#pragma unroll 1
  for (int t = 0; t < e.nout; ++t) o[t] = ((e.bnz >> t) & 1) ? e.b[t] * res : 0.0;
#pragma unroll 1
  for (int k = 0; k < e.nterm; ++k) o[e.term_t[k]] = fma(e.term_c[k], sv[e.term_m[k]], o[e.term_t[k]]);
#pragma unroll 1
  for (int t = 0; t < e.nout; ++t) {
    if ((e.out_f32mask >> t) & 1) ((float*)e.out[t])[idx] = (float)o[t];
    else e.out[t][idx] = o[t];
  }
}
#endif

// Geometry of one mu-mode product on a tensor viewed as (a, n, b):
// element (x, j, y) at x + a*j + a*n*y.
struct ModeGeom {
  int64_t a;   // product of n_nu for nu < mu
  int n;       // n_mu
  int64_t b;   // product of n_nu for nu > mu
};

// W = V x_mu L (FP64).  V given by `pro` (a combination), L column-major
// n x n.  With epi == nullptr or epi->nout == 0 the result goes to W.
// tile: 0 by size, 1 16 x 16 output tiles, 2 32 x 64 output tiles.
cudaError_t launch_mode_product_f64(const Combo& pro, const double* L, ModeGeom g, double* W,
                                    const Epi* epi, cudaStream_t st, int tile = 0);
// B <= kMaxModeBatch independent mode products of the same geometry in one
// launch: W[b] = (combination pro[b]) x_mu L[b], stored plainly.
constexpr int kMaxModeBatch = 16;
struct ModeBatch {
  Combo pro[kMaxModeBatch];
  const double* L[kMaxModeBatch];
  double* W[kMaxModeBatch];
};
cudaError_t launch_mode_product_f64_batch(const ModeBatch& mb, int B, ModeGeom g, cudaStream_t st,
                                          int tile = 0);
// The same for complex V, W (interleaved) and L given as its 2n x 2n real
// representation (PHIKS_C128 plans).
cudaError_t launch_mode_product_c128(const Combo& pro, const double* L, ModeGeom g, double* W,
                                    const Epi* epi, cudaStream_t st);

// out[t][i] = sum_m a[t][m] src[m][i] over N elements (Epi with b ignored),
// FP64 arithmetic; sources and outputs double or float as the masks say.
cudaError_t launch_combine(const Epi& e, int64_t N, cudaStream_t st);
// B <= kMaxEpiBatch independent combinations over N elements each, in one launch.
constexpr int kMaxEpiBatch = 8;
cudaError_t launch_combine_batch(const Epi* e, int B, int64_t N, cudaStream_t st);

// out[k] = ||x_k||_2^2 accumulated (out must be zeroed), k < count; x_k double
// (is_f32 == 0) or float.
cudaError_t launch_sumsq(const void* const* x, int count, int64_t N, int is_f32, double* out,
                         cudaStream_t st);

// Fused small-slab Tucker operators (tucker_fused.cu): B <= kMaxModeBatch
// independent FP64 Tucker operators W[b] = (combination pro[b]) x_1 L[b][0]
// ... x_d L[b][d-1] in one launch, every intermediate in shared memory;
// store[b] (or null) also receives the input combination's values, and nside
// elementwise combinations side[k] -> side_out[k] over N elements run in the
// same launch (they may read what the launch's inputs read, and nothing the
// launch writes).  Needs the slab of one last-mode row, 16 N / n_d bytes, and
// the matrices in shared memory (fused_f64_ok).  nj: last-mode rows per CTA
// (1, 2, 4 or 8; fewer when the slab would not fit); with an epilogue
// (epi->nout > 0) the results go through it instead of W.
constexpr int kFusedMaxD = 8;
constexpr int kFusedMaxSide = 8;
constexpr int64_t kFusedMaxN = int64_t(1) << 20;
constexpr int kFusedMaxSmem = 200 * 1024;
struct FusedBatch {
  int B;
  Combo pro[kMaxModeBatch];
  const double* L[kMaxModeBatch][kFusedMaxD];
  double* W[kMaxModeBatch];
  double* store[kMaxModeBatch];
  int nside;
  Combo side[kFusedMaxSide];
  double* side_out[kFusedMaxSide];
};
bool fused_f64_ok(int d, const int64_t* n, int64_t N);
int fused_f64_default_nj(int d, const int64_t* n, int64_t N, int B);
cudaError_t launch_tucker_fused_f64(const FusedBatch& fb, int d, const int64_t* n, int64_t N, int nj,
                                    const Epi* epi, cudaStream_t st);

// One CTA of a tcgen05 kernel whose mbarrier wait has nothing to arrive at:
// the wait gives up after limit_ns and records its failure in *status (the
// status word of a tensor-core plan); waitcheck.cu.
cudaError_t launch_wait_check(int* status, uint64_t limit_ns, cudaStream_t st);

// ---- small dense FP64 matrices (the exponentials of Sec. 3) ---------------
constexpr int kMaxBatch = 64;

struct GemmBatch {
  int count;
  int n[kMaxBatch];
  const double* A[kMaxBatch];
  const double* B[kMaxBatch];
  double* C[kMaxBatch];
  double alpha[kMaxBatch];
  double beta_I[kMaxBatch];          // coefficient of the identity
  const double* addm[kMaxBatch][3];  // optional addends (may be null)
  double addc[kMaxBatch][3];
};
// Batched C_k = alpha_k A_k B_k + beta_k I + sum_j addc_kj addm_kj
// (column-major n_k x n_k; alpha_k = 0 skips the product).
cudaError_t launch_gemm_batch_f64(const GemmBatch& gb, int nmax, cudaStream_t st);

// Batched matrix polynomials from stored powers:
//   Y_k = c_k0 I + sum_{i=1}^{m_k} c_ki P_ki   (column-major n_k x n_k),
// summed from the highest power down.
constexpr int kPolyBatch = 32;
constexpr int kPolyMax = 15;
struct PolyBatch {
  int count;
  int n[kPolyBatch];
  int m[kPolyBatch];
  double* Y[kPolyBatch];
  const double* P[kPolyBatch][kPolyMax];  // P[k][i - 1] = the i-th power
  double c[kPolyBatch][kPolyMax + 1];
};
cudaError_t launch_poly_batch_f64(const PolyBatch& pb, int nmax, cudaStream_t st);

}  // namespace phiks
