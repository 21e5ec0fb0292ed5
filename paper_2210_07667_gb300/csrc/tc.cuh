// Split-precision mu-mode products on the tensor cores (tcgen05 / TMEM, TMA):
// the PHIKS_TF32, PHIKS_TF32X3 and PHIKS_BF16X3 dtypes.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/phiks.h"
#include "kernels.cuh"

namespace phiks {

struct TcState;

// Extra device workspace the split path needs for a tensor of N elements.
size_t tc_workspace_bytes(int64_t N);

phiks_status tc_create(TcState** out, int d, const int64_t* n, int64_t N);
void tc_destroy(TcState* s);
const char* tc_last_error();
void tc_bind_workspace(TcState* s, void* ws);

// W = V x_mu L with V the combination `in` (float or double sources per
// in.f32mask), L FP64 column-major (rounded to the dtype's operands), result
// through `epi` (double or float outputs per its masks) or stored as float to
// W when epi is null / has no outputs.
cudaError_t tc_mode_product(TcState* s, int dtype, const Combo& in, const double* L, ModeGeom g,
                            void* W, const Epi* epi, cudaStream_t st);

}  // namespace phiks
