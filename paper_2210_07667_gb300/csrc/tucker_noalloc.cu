// phiks_tucker_noalloc: the FP64 Tucker operator W = V x_1 L_1 ... x_d L_d
// for callers that cannot allocate device memory themselves.
//
// Who needs it: a host application that hands all of its device memory to
// its own pool up front and forbids any other allocation, or a latency-bound
// loop that cannot afford cudaMalloc / cudaFree (they take locks in the driver
// and cudaFree synchronises the device).  phiks_tucker needs a plan, and the
// plan allocates its workspace; this entry point needs neither.
//
// Where its scratch lives: the d - 1 intermediate tensors of the mode-by-mode
// evaluation ping-pong between the two halves of one file-scope __device__
// array, kMaxElems doubles each (2 x 8 MiB).  Every GPU that loads this
// library holds those 16 MiB until the process exits.  Device code could name
// the array directly; host code cannot, because the array's name on the host
// is only a stand-in for the device object, so the host takes its device
// address once per device through cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/phiks.h"
#include "kernels.cuh"

namespace phiks {
namespace {

constexpr int64_t kMaxElems = int64_t(1) << 20;  // N limit: 1,048,576 elements
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[2 * kMaxElems];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

phiks_status noalloc_fail(phiks_status st, const char* msg) {
  char buf[320];
  std::snprintf(buf, sizeof buf, "phiks_tucker_noalloc: %s", msg);
  set_error_message(buf);
  return st;
}

// Device address of g_scratch on the current device; looked up on the first
// call per device (that call must not sit inside a stream capture).
phiks_status scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(PHIKS_ERR_CUDA, "no usable current device");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      char buf[256];
      std::snprintf(buf, sizeof buf, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return noalloc_fail(PHIKS_ERR_CUDA, buf);
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return PHIKS_OK;
}

}  // namespace
}  // namespace phiks

using namespace phiks;

extern "C" phiks_status phiks_tucker_noalloc(int d, const int64_t* n, const double* V, double* W,
                                             const double* const* L, void* stream) {
  set_error_message("");
  if (d < 1 || d > PHIKS_MAX_D) return noalloc_fail(PHIKS_ERR_INVALID, "d out of [1, PHIKS_MAX_D]");
  if (!n || !V || !W || !L) return noalloc_fail(PHIKS_ERR_INVALID, "NULL argument");
  int64_t N = 1;
  for (int mu = 0; mu < d; ++mu) {
    if (n[mu] < 1 || n[mu] > 65536) return noalloc_fail(PHIKS_ERR_INVALID, "n_mu out of [1, 65536]");
    if (!L[mu]) return noalloc_fail(PHIKS_ERR_INVALID, "L[mu] is NULL");
    if (N > kMaxElems / n[mu])
      return noalloc_fail(PHIKS_ERR_INVALID, "N = n_1 ... n_d exceeds the 1,048,576-element scratch");
    N *= n[mu];
  }
  {  // V and W may not share any element: with d == 1 the single mode
     // product would read V while it writes W
    const uintptr_t v0 = (uintptr_t)V, w0 = (uintptr_t)W, bytes = (uintptr_t)N * sizeof(double);
    if (v0 < w0 + bytes && w0 < v0 + bytes) return noalloc_fail(PHIKS_ERR_INVALID, "V and W overlap");
  }
  double* scratch = nullptr;
  phiks_status st = scratch_address(&scratch);
  if (st != PHIKS_OK) return st;
  double* half[2] = {scratch, scratch + kMaxElems};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Every mode product writes all N elements of its output, so nothing in the
  // scratch has to start at zero.
  Combo in;
  in.nsrc = 1;
  in.f32mask = 0;
  in.src[0] = V;
  in.coef[0] = 1.0;
  int64_t a = 1;
  for (int mu = 0; mu < d; ++mu) {
    int64_t b = N / (a * n[mu]);
    double* out = (mu == d - 1) ? W : half[mu & 1];
    ModeGeom g{a, (int)n[mu], b};
    cudaError_t e = launch_mode_product_f64(in, L[mu], g, out, nullptr, s);
    if (e != cudaSuccess) return noalloc_fail(PHIKS_ERR_CUDA, cudaGetErrorString(e));
    in.src[0] = out;
    a *= n[mu];
  }
  return PHIKS_OK;
}
