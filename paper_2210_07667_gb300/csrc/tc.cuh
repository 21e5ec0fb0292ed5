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

// Tucker operators one tc_tucker call runs together.
constexpr int kTcMaxBatch = 4;

// Bytes of workspace the split path needs for kTcMaxBatch tensors of N elements.
size_t tc_workspace_bytes(int64_t N);

phiks_status tc_create(TcState** out, int dtype, int d, const int64_t* n, int64_t N);
void tc_destroy(TcState* s);
const char* tc_last_error();
void tc_bind_workspace(TcState* s, void* ws);

// Bytes of the B-operand planes of one n x n matrix, and their preparation
// from an FP64 column-major matrix (row i of a plane holds L[i, 0..n_pad),
// zero padded to n_pad = n rounded up to 16).
size_t tc_bplanes_bytes(int dtype, int n);
cudaError_t tc_prepare_b(int dtype, const double* L, int n, void* dst, cudaStream_t st);

// B <= kTcMaxBatch Tucker operators with the same matrices, run together:
// W_b = (combination in[b]) x_1 L_1 ... x_d L_d through epi[b] (FP64
// arithmetic in the epilogue; outputs double or float as its masks say).
// Every pass treats the B tensors as one tensor with B times the fibres.
// Bp[mu] are B planes made by tc_prepare_b for L_mu.
cudaError_t tc_tucker(TcState* s, int B, const Combo* in, const void* const* Bp, const Epi* epi,
                      cudaStream_t st);

// Device-side status: 0, or the code of a bounded wait that gave up (the
// flag is cleared by the read).  Synchronises the stream.
int tc_read_status(TcState* s, cudaStream_t st);

// Largest n_mu the tensor-core path handles (N tiles of <= 256 rows beyond 256).
constexpr int kTcMaxN = 1024;

}  // namespace phiks
