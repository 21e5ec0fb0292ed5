// Exponential integrators driving phiks on the device: exponential Euler and
// ETD2RK in their linear-combination forms (Sec. 2, eq. expEullc and
// eq. ETD2RKlc), with the nonlinear term evaluated by a CUDA kernel.
//
//   exponential Euler:  u_{n+1} = exp(tau K) u_n + tau phi_1(tau K) g(t_n, u_n)
//   ETD2RK:             u_n2    = exp(tau K) u_n + tau phi_1(tau K) g_n
//                       u_{n+1} = exp(tau K) u_n + tau phi_1(tau K) g_n
//                                 + tau phi_2(tau K) (g(t_n + tau, u_n2) - g_n)
// Every stage is one phiks_apply_ex call (a linear combination).
//
// Nonlinear terms:
//   PHIKS_NL_ADR_EXACT (Sec. 4.2): g = 1/(1 + u^2) + Psi(t, x) on the
//     Dirichlet grid x_i = i/(n+1) of [0,1]^3, Psi making e^t u_0,
//     u_0 = 64 prod x(1-x), the exact solution of u_t = eps Lap u +
//     alpha (d_1 + d_2 + d_3) u + g.
//   PHIKS_NL_ALLEN_CAHN (Sec. 4.3): g = -u^3 / eps^2 (K = Lap + I/eps^2).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/phiks.h"
#include "kernels.cuh"

namespace {

__global__ void g_adr_kernel(const double* __restrict__ u, double t, int n1, int n2, int n3,
                             double eps, double alpha, double scale, double* __restrict__ out) {
  const int64_t N = (int64_t)n1 * n2 * n3;
  const double et = exp(t);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i1 = (int)(idx % n1);
    const int i2 = (int)((idx / n1) % n2);
    const int i3 = (int)(idx / ((int64_t)n1 * n2));
    const double x1 = (i1 + 1.0) / (n1 + 1.0), x2 = (i2 + 1.0) / (n2 + 1.0),
                 x3 = (i3 + 1.0) / (n3 + 1.0);
    const double q1 = x1 * (1 - x1), q2 = x2 * (1 - x2), q3 = x3 * (1 - x3);
    const double u0 = 64.0 * q1 * q2 * q3;
    const double lap = -128.0 * (q2 * q3 + q1 * q3 + q1 * q2);
    const double grad = 64.0 * ((1 - 2 * x1) * q2 * q3 + q1 * (1 - 2 * x2) * q3 + q1 * q2 * (1 - 2 * x3));
    const double w = et * u0;
    const double psi = et * (u0 - eps * lap - alpha * grad) - 1.0 / (1.0 + w * w);
    const double v = u[idx];
    out[idx] = scale * (1.0 / (1.0 + v * v) + psi);
  }
}

__global__ void g_ac_kernel(const double* __restrict__ u, int64_t N, double eps, double scale,
                            double* __restrict__ out) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const double v = u[idx];
    out[idx] = -scale * v * v * v / (eps * eps);
  }
}

__global__ void axpby_kernel(const double* x, const double* y, double a, double b, int64_t N,
                             double* out) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N;
       idx += (int64_t)gridDim.x * blockDim.x)
    out[idx] = a * x[idx] + b * y[idx];
}

int grid_of(int64_t N) {
  int64_t g = (N + 255) / 256;
  return (int)(g > 152 * 16 ? 152 * 16 : (g < 1 ? 1 : g));
}

struct Fail {
  phiks_status st;
  std::string msg;
};

}  // namespace

extern "C" phiks_status phiks_integrate(phiks_plan_t plan, const int64_t* n, int d, int scheme,
                                        const phiks_nonlinear* g, double t0, double T, int steps,
                                        double* u, void* stream) {
  phiks::set_error_message("");
  auto fail = [](phiks_status s, const char* m) {
    phiks::set_error_message((std::string("phiks_integrate: ") + m).c_str());
    return s;
  };
  if (!plan || !n || !g || !u || steps < 1 || !(T > 0) || d < 1 || d > PHIKS_MAX_D)
    return fail(PHIKS_ERR_INVALID, "bad arguments");
  if (scheme != PHIKS_EXP_EULER && scheme != PHIKS_ETD2RK) return fail(PHIKS_ERR_INVALID, "scheme");
  if (g->kind == PHIKS_NL_ADR_EXACT && d != 3) return fail(PHIKS_ERR_INVALID, "ADR needs d = 3");
  if (g->kind != PHIKS_NL_ADR_EXACT && g->kind != PHIKS_NL_ALLEN_CAHN)
    return fail(PHIKS_ERR_INVALID, "nonlinearity kind");
  int64_t N = 1;
  for (int mu = 0; mu < d; ++mu) N *= n[mu];
  cudaStream_t st = (cudaStream_t)stream;
  double* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, 4 * (size_t)N * sizeof(double), st) != cudaSuccess)
    return fail(PHIKS_ERR_OOM, "workspace");
  double *g1 = buf, *g2 = buf + N, *u2 = buf + 2 * N, *un = buf + 3 * N;
  const double tau = T / steps;
  phiks_status res = PHIKS_OK;
  auto eval_g = [&](const double* x, double t, double* out) -> bool {
    phiks::count_launch();
    if (g->kind == PHIKS_NL_ADR_EXACT)
      g_adr_kernel<<<grid_of(N), 256, 0, st>>>(x, t, (int)n[0], (int)n[1], (int)n[2], g->eps,
                                               g->alpha, tau, out);
    else
      g_ac_kernel<<<grid_of(N), 256, 0, st>>>(x, N, g->eps, tau, out);
    return cudaGetLastError() == cudaSuccess;
  };
  double t = t0;
  for (int k = 0; k < steps && res == PHIKS_OK; ++k) {
    if (!eval_g(u, t, g1)) {
      res = fail(PHIKS_ERR_CUDA, "nonlinear term launch");
      break;
    }
    if (scheme == PHIKS_EXP_EULER) {
      const void* v[2] = {u, g1};
      res = phiks_apply(plan, tau, 1, v, 2, un, stream);
    } else {
      const void* v1[2] = {u, g1};
      res = phiks_apply(plan, tau, 1, v1, 2, u2, stream);
      if (res != PHIKS_OK) break;
      if (!eval_g(u2, t + tau, g2)) {
        res = fail(PHIKS_ERR_CUDA, "nonlinear term launch");
        break;
      }
      phiks::count_launch();
      axpby_kernel<<<grid_of(N), 256, 0, st>>>(g2, g1, 1.0, -1.0, N, g2);
      const void* v2[3] = {u, g1, g2};
      res = phiks_apply(plan, tau, 2, v2, 3, un, stream);
    }
    if (res != PHIKS_OK) break;
    if (cudaMemcpyAsync(u, un, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      res = fail(PHIKS_ERR_CUDA, "copy");
    t = t0 + (k + 1) * tau;
  }
  cudaFreeAsync(buf, st);
  return res;
}
