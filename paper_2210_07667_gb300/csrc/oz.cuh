// FP64 mu-mode products emulated on the tensor cores with exact integer
// slice products (the PHIKS_FP64_EMU dtype).
//
// Every fibre of the operand X (the n values contracted together) and every
// row of L is scaled by a power of two and written as seven balanced base-256
// digits c_0 .. c_6 (|c_s| <= 128), each stored exactly as a bf16:
//     x = 2^e_x sum_s c_s 2^(-8 s),     l = 2^e_l sum_s b_s 2^(-8 s).
// Then sum_j l x = 2^(e_x + e_l) sum_k 2^(-8 k) G_k with
// G_k = sum_{s + t = k} sum_j b_s c_t.  Each product of digits is below 2^14
// and (k + 1) n 2^14 < 2^24 for n <= 128, so the tensor cores accumulate
// every G_k (k = 0..6, 28 digit products) exactly in FP32; the epilogue
// assembles floor(sum_k 2^(8 (6 - k)) G_k / 2^8) in 64-bit integers and
// rounds it to FP64 (within (1/2 + 2^-8) ulp of the digit sum).  Per dot
// product of length n the error is at most
//   (7.03 n 2^-54 + 2^-52) max|x| max|l| + 2^-53 |result|:
// rounding x and l to the fibre's fixed point costs 2^-54 max|x| max|l| per
// term, the dropped digit products with s + t >= 7 at most 6.03 2^-54 per
// term (only when the low digit products all share a sign), the floor 2^-52.
// Between the passes of one Tucker operator (n_mu <= 64) the sum is kept
// exact: the next split takes S with its scale and rounds it once to that
// pass's fibre fixed point, so the last term applies to the last pass only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/phiks.h"
#include "kernels.cuh"

namespace phiks {

struct OzState;

constexpr int kOzSlices = 7;
constexpr int kOzMaxN = 128;
constexpr int kOzMaxBatch = 16;  // Tucker operators one oz_tucker call can run together
constexpr int kOzMaxSide = 8;    // extra combinations of its first split pass

// Workspace of oz_tucker for batches of up to `batch` (<= kOzMaxBatch) tensors.
size_t oz_workspace_bytes(int d, const int64_t* n, int64_t N, int batch);
phiks_status oz_create(OzState** out, int d, const int64_t* n, int64_t N);
void oz_destroy(OzState* s);
const char* oz_last_error();
void oz_bind_workspace(OzState* s, void* ws, double* tmp0, double* tmp1, int batch);

// Bytes of the B-operand slices of one n x n matrix (7 planes of n_pad x
// n_pad bf16 and n_pad row exponents), and their preparation from FP64
// column-major matrices: L[k] (n[k] x n[k]) into dst[k], k < count.
size_t oz_bplanes_bytes(int n);
cudaError_t oz_prepare_b(int count, const double* const* L, const int* n, void* const* dst,
                         cudaStream_t st);

// The B-operand planes (made by oz_prepare_b) of the d matrices of one Tucker
// operator.
struct OzMats {
  const void* B[PHIKS_MAX_D];
};

// Whether the tensors of one oz_tucker call may have different matrices:
// always (every tensor is tiled on its own, its last row tile partial).
bool oz_mixed_ok(const OzState* s);

// B Tucker operators run together (B at most the `batch` given to
// oz_bind_workspace): (combination in[b]) x_1 L_1 ... x_d L_d with the
// matrices mats[b] (the same for every b, or oz_mixed_ok), then through
// epi[b] (FP64).  Every pass treats the B tensors as one tensor with B times
// the fibres.  The bound workspace holds the digit planes of `batch` tensors,
// and tmp0 / tmp1 batch N doubles each.  With epi == nullptr no epilogue
// runs and *res receives the B results (tensor b at *res + b N, valid until
// the next call).  `ev` (2 d events, or null): ev[2 mu] and ev[2 mu + 1] are
// recorded around the tensor-core pass of mode mu.
// `pro` (or null) extends the first split pass: tensor b's input values are
// also stored to pro->store[b] (when not null), and pro->nside further
// combinations (FP64, as the inputs) are evaluated into pro->side_out[k] in
// the same launch; they may read the results of the previous call (its *res).
struct OzPrologue {
  double* store[kOzMaxBatch];
  int nside;
  Combo side[kOzMaxSide];
  double* side_out[kOzMaxSide];
};
cudaError_t oz_tucker(OzState* s, int B, const Combo* in, const OzMats* mats, const Epi* epi,
                      cudaStream_t st, const cudaEvent_t* ev = nullptr, const double** res = nullptr,
                      const OzPrologue* pro = nullptr);

int oz_read_status(OzState* s, cudaStream_t st);
// Rows of L per GEMM tile (16 or 32; 0 = by size).
void oz_set_ntile(OzState* s, int nt);
// The device status word the kernels record a failed wait in.
int* oz_status_word(OzState* s);

}  // namespace phiks
