// Function posterior at new inputs (Sec. "Function posterior at new inputs",
// Eq. gp_posterior_newx): given f at the training inputs x (the Gibbs state)
// and K~ = tau2 C~,
//   mu*_j      = c(x*_j, x)^T C~^-1 f,
//   sigma*^2_j = tau2 (1 - || W_C^-1 c(x, x*_j) ||^2),   W_C W_C^T = C~,
// with the unit-variance kernel c (no nugget on the cross entries) evaluated
// by the same deterministic kernel entries as the assembly.
//   k_pred_mean : one CTA per new input, a fixed-order block sum over the n
//                 training inputs of c(x*_j, x_i) alpha_i (alpha = C~^-1 f).
//   k_pred_cols : the cross-kernel columns of two new inputs at a time, then
//                 one W_C^-1 sweep for both and their squared norms.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "../../include/fifa.h"
#include "fifa_api_internal.h"
#include "fifa_common.cuh"
#include "fifa_launch.h"

#define CK(call)                 \
  do {                           \
    cudaError_t e_ = (call);     \
    if (e_ != cudaSuccess) {     \
      ctx->last_cuda = e_;       \
      return FIFA_ERR_CUDA;      \
    }                            \
  } while (0)

__global__ void __launch_bounds__(256) k_pred_mean(const HmatDesc* __restrict__ Hd, const double* __restrict__ x,
                                                   const double* __restrict__ xs, const double* __restrict__ alpha,
                                                   double* __restrict__ mu) {
  __shared__ double red[40];
  const int j = blockIdx.x;
  const int64_t n = Hd->n;
  const double xj = xs[j], kc = Hd->kc;
  const int kind = Hd->kind;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += kern_entry(kind, kc, xj, x[i]) * alpha[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) mu[j] = acc;
}

// cols[q * n + i] = c(x*_{j0 + q}, x_i) for q < cnt (cnt <= 2)
__global__ void k_pred_cols(const HmatDesc* __restrict__ Hd, const double* __restrict__ x,
                            const double* __restrict__ xs, int64_t j0, int cnt, double* __restrict__ cols) {
  const int64_t n = Hd->n;
  const double kc = Hd->kc;
  const int kind = Hd->kind;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int q = 0; q < cnt; ++q) cols[q * n + i] = kern_entry(kind, kc, xs[j0 + q], x[i]);
}

// var[j0 + q] = tau2 (1 - qsum[q])
__global__ void k_pred_var(const double* __restrict__ qsum, int cnt, double tau2, double* __restrict__ var,
                           int64_t j0) {
  const int q = threadIdx.x;
  if (q < cnt) var[j0 + q] = tau2 * (1.0 - qsum[q]);
}

extern "C" fifa_status fifa_predict(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, const double* x_dev,
                                    const double* f_dev, const double* xstar_dev, int64_t nstar, double tau2,
                                    double* mu_dev, double* var_dev) {
  if (!ctx || !C || !WC || !x_dev || !f_dev || !xstar_dev || nstar < 0 || !(tau2 > 0.0)) return FIFA_ERR_INVALID_ARG;
  if (C->plan != WC->plan || C->host.shift != 0.0 || C->host.scale != 1.0 || C->host.diag) return FIFA_ERR_INVALID_ARG;
  if (nstar == 0 || (!mu_dev && !var_dev)) return FIFA_OK;
  if (nstar > (1 << 30)) return FIFA_ERR_UNSUPPORTED;
  Plan* P = C->plan;
  fifa_status st = ensure_scratch(ctx, P);
  if (st != FIFA_OK) return st;
  Scratch S = carve(ctx, P);
  const int64_t n = P->n;
  cudaStream_t s = ctx->stream;
  double* alpha = S.vec;     // n: C~^-1 f
  double* cols = S.vec + n;  // 2n: cross-kernel columns, then W_C^-1 of them
  if (mu_dev) {
    CK(cudaMemcpyAsync(alpha, f_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if ((st = sweep_enqueue_desc(ctx, P, WC->dev, 0, 4, alpha, 1)) != FIFA_OK) return st;  // W^-T W^-1 f
    k_pred_mean<<<(unsigned)nstar, 256, 0, s>>>(C->dev, x_dev, xstar_dev, alpha, mu_dev);
    CK(cudaGetLastError());
  }
  if (var_dev) {
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, 4096);
    for (int64_t j0 = 0; j0 < nstar; j0 += 2) {
      const int cnt = (int)std::min<int64_t>(2, nstar - j0);
      k_pred_cols<<<blocks, threads, 0, s>>>(C->dev, x_dev, xstar_dev, j0, cnt, cols);
      CK(cudaGetLastError());
      if ((st = sweep_enqueue(ctx, WC, 0, 1, cols, cnt)) != FIFA_OK) return st;  // W_C^-1 c
      for (int q = 0; q < cnt; ++q) CK(launch_sumsq(cols + (size_t)q * n, nullptr, n, S.red, S.red + 300 + q, s));
      k_pred_var<<<1, 32, 0, s>>>(S.red + 300, cnt, tau2, var_dev, j0);
      CK(cudaGetLastError());
    }
  }
  return FIFA_OK;
}
