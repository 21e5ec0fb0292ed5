// Split-precision mu-mode products on the tensor cores (tcgen05 / TMEM, fed by
// TMA): the PHIKS_TF32, PHIKS_TF32X3 and PHIKS_BF16X3 dtypes.
//
// A Tucker operator runs as d GEMM passes over "operand planes": the tensor is
// split once into hi (and lo) planes of bf16 or tf32 values, every pass
// contracts the contiguous mode on the tensor cores and writes its result,
// already split, with the contracted mode moved to the slowest position, so
// the next mode is contiguous in turn and after d passes the natural layout is
// back.  The last pass writes through the FP64 epilogue (Epi).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/phiks.h"
#include "kernels.cuh"

namespace phiks {

struct TcState;

// Tucker operators one tc_tucker call can run together, and extra
// combinations of its split pass.
constexpr int kTcMaxBatch = 16;
constexpr int kTcMaxSide = 8;

// Bytes of workspace the split path needs for `batch` tensors of N elements.
size_t tc_workspace_bytes(int64_t N, int batch);

phiks_status tc_create(TcState** out, int dtype, int d, const int64_t* n, int64_t N);
void tc_destroy(TcState* s);
const char* tc_last_error();
void tc_bind_workspace(TcState* s, void* ws, int batch);

// Bytes of the B-operand planes of one n x n matrix, and their preparation
// from an FP64 column-major matrix (row i of a plane holds L[i, 0..n_pad),
// zero padded to n_pad = n rounded up to 16).
size_t tc_bplanes_bytes(int dtype, int n);
cudaError_t tc_prepare_b(int dtype, const double* L, int n, void* dst, cudaStream_t st);
// The same for count matrices L[k] (n[k] x n[k]) into dst[k], in one launch per
// 32 matrices.
cudaError_t tc_prepare_b_many(int dtype, int count, const double* const* L, const int* n, void* const* dst,
                              cudaStream_t st);

// The B-operand planes of the d matrices of one Tucker operator.
struct TcMats {
  const void* B[PHIKS_MAX_D];
};

// Whether the tensors of one tc_tucker call may have different matrices
// (every mode's fibre count N / n_mu a multiple of 128).
bool tc_mixed_ok(const TcState* s);

// Extensions of the split pass: tensor b's input values are also stored to
// store[b] (FP64, or null); nside further combinations are evaluated into
// side_out[k] (float when bit k of side_f32 is set, else double) in the same
// launch, and may read the previous call's results.
struct TcPrologue {
  double* store[kTcMaxBatch];
  int nside;
  unsigned side_f32;
  Combo side[kTcMaxSide];
  void* side_out[kTcMaxSide];
};

// B Tucker operators run together (B at most the `batch` given to
// tc_bind_workspace): W_b = (combination in[b]) x_1 L_1 ... x_d L_d with the
// matrices mats[b] (B planes made by tc_prepare_b; the same for every b, or
// tc_mixed_ok), through epi[b] (FP64 arithmetic in the epilogue; outputs
// double or float as its masks say).  Every pass treats the B tensors as one
// tensor with B times the fibres.  With epi == nullptr no epilogue runs and
// *res receives the B results as float (tensor b at *res + b N, valid until
// the next call).  `pro` (or null) extends the split pass.  `ev` (2 d
// events, or null): ev[2 mu] and ev[2 mu + 1] are recorded around the GEMM
// pass of mode mu.
cudaError_t tc_tucker(TcState* s, int B, const Combo* in, const TcMats* mats, const Epi* epi,
                      cudaStream_t st, const float** res = nullptr, const TcPrologue* pro = nullptr,
                      const cudaEvent_t* ev = nullptr);

// Device-side status: 0, or the code of a bounded wait that gave up (the
// flag is cleared by the read).  Synchronises the stream.
int tc_read_status(TcState* s, cudaStream_t st);
// N tiles per GEMM pass as a multiple of the minimum ceil(n_pad / 256):
// 1, 2 or 4 (smaller tiles, more CTAs); 0 = by size (narrower tiles when the
// row tiles alone leave SMs idle).
void tc_set_ntiles(TcState* s, int mult);
// The device status word the kernels record a failed wait in.
int* tc_status_word(TcState* s);

// Largest n_mu the tensor-core path handles (N tiles of <= 256 rows beyond 256).
constexpr int kTcMaxN = 1024;

}  // namespace phiks
