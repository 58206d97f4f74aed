// Length-scale on a discrete grid (Eq. posterior_gibs4, the sampler the paper
// times): with a prior over the grid {s_1, ..., s_G} and K_h = tau2 C~(s_h),
//   Pr(rho = s_h | f, tau2) ~ prior_h det(K_h)^-1/2 exp(-f^T K_h^-1 f / 2),
// so with the factors W_h W_h^T = C~(s_h) computed once,
//   log w_h = log prior_h - logdet C~_h / 2 - ||W_h^-1 f||^2 / (2 tau2)
// (the common -n log(tau2) / 2 cancels).  A draw costs one W_h^-1 sweep per
// grid point and a categorical draw from a Philox uniform on the device.
#include <cuda_runtime.h>
#include <math.h>

#include <new>
#include <vector>

#include "../../include/fifa.h"
#include "fifa_api_internal.h"
#include "fifa_common.cuh"
#include "fifa_launch.h"
#include "fifa_rng.cuh"

#define CK(call)                 \
  do {                           \
    cudaError_t e_ = (call);     \
    if (e_ != cudaSuccess) {     \
      ctx->last_cuda = e_;       \
      return FIFA_ERR_CUDA;      \
    }                            \
  } while (0)

struct fifa_grid {
  int G = 0;
  std::vector<fifa_hmat*> H;
  std::vector<fifa_fact*> F;
  double* x = nullptr;         // n (arena copy of the inputs)
  double* logdet = nullptr;    // G, device
  double* quad = nullptr;      // G, device: ||W_h^-1 f||^2 of the last draw
  double* lprior = nullptr;    // G, device
  double* probs = nullptr;     // G, device
  int* index = nullptr;        // 1, device
  double* tmp = nullptr;       // n, device
};

__global__ void k_grid_gather_logdet(const FactDesc* __restrict__ Fd, double* __restrict__ out) {
  if (threadIdx.x == 0) *out = *Fd->logdet;
}

// One thread: normalised weights (largest log-weight subtracted), their
// cumulative sum in grid order, and the first index whose cumulative sum
// exceeds u (the last one if rounding leaves the total below u).
__global__ void k_grid_draw(const double* __restrict__ logdet, const double* __restrict__ quad,
                            const double* __restrict__ lprior, int G, double tau2, uint64_t seed, uint64_t it,
                            uint64_t sid, double* __restrict__ probs, int* __restrict__ index) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double m = -INFINITY;
  for (int h = 0; h < G; ++h) {
    const double lw = lprior[h] - 0.5 * logdet[h] - 0.5 * quad[h] / tau2;
    probs[h] = lw;
    m = fmax(m, lw);
  }
  double tot = 0.0;
  for (int h = 0; h < G; ++h) {
    probs[h] = exp(probs[h] - m);
    tot += probs[h];
  }
  const double u = philox_uniform(seed, 0u, 5u, it, sid);
  double cdf = 0.0;
  int pick = G - 1;
  for (int h = 0; h < G; ++h) {
    probs[h] /= tot;
    cdf += probs[h];
    if (cdf > u && pick == G - 1 && h < G - 1) pick = h;
  }
  *index = pick;
}

extern "C" fifa_status fifa_grid_create(fifa_ctx* ctx, const double* x_dev, int64_t n, int kernel, double nugget,
                                        const double* rho_host, int G, const double* log_prior_host,
                                        fifa_grid** out) {
  if (!ctx || !x_dev || !rho_host || !out || n < 1 || G < 1 || G > 4096 || !(nugget >= 0.0)) return FIFA_ERR_INVALID_ARG;
  if (kernel != 0 && kernel != 1) return FIFA_ERR_INVALID_ARG;
  for (int h = 0; h < G; ++h)
    if (!(rho_host[h] > 0.0) || !isfinite(rho_host[h])) return FIFA_ERR_INVALID_ARG;
  *out = nullptr;
  fifa_grid* g = new (std::nothrow) fifa_grid();
  if (!g) return FIFA_ERR_OOM;
  auto fail = [&](fifa_status e) {
    fifa_destroy_grid(ctx, g);
    return e;
  };
  g->G = G;
  cudaStream_t s = ctx->stream;
  g->x = (double*)ctx->arena.alloc(sizeof(double) * n);
  g->tmp = (double*)ctx->arena.alloc(sizeof(double) * n);
  g->logdet = (double*)ctx->arena.alloc(sizeof(double) * G);
  g->quad = (double*)ctx->arena.alloc(sizeof(double) * G);
  g->lprior = (double*)ctx->arena.alloc(sizeof(double) * G);
  g->probs = (double*)ctx->arena.alloc(sizeof(double) * G);
  g->index = (int*)ctx->arena.alloc(sizeof(int));
  if (!g->x || !g->tmp || !g->logdet || !g->quad || !g->lprior || !g->probs || !g->index) return fail(FIFA_ERR_OOM);
  CK(cudaMemcpyAsync(g->x, x_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  std::vector<double> lp(G, 0.0);
  if (log_prior_host)
    for (int h = 0; h < G; ++h) lp[h] = log_prior_host[h];
  CK(cudaMemcpyAsync(g->lprior, lp.data(), sizeof(double) * G, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  for (int h = 0; h < G; ++h) {
    fifa_hyper hy{kernel, 1.0, rho_host[h], 1.0, nugget};
    fifa_hmat* H = nullptr;
    fifa_status st = fifa_assemble(ctx, g->x, n, &hy, &H);
    if (st != FIFA_OK) return fail(st);
    g->H.push_back(H);
    fifa_fact* F = nullptr;
    st = fact_alloc(ctx, H->plan, 0, &F);
    if (st != FIFA_OK) return fail(st);
    F->src = H;
    g->F.push_back(F);
    if ((st = fact_enqueue(ctx, F, H->dev)) != FIFA_OK) return fail(st);
    k_grid_gather_logdet<<<1, 32, 0, s>>>(F->dev, g->logdet + h);
    CK(cudaGetLastError());
  }
  // every grid matrix must have factored: a non-positive pivot is an error here
  int bad = 0;
  for (int h = 0; h < G; ++h) {
    double ld = 0.0;
    fifa_status st = fifa_logdet(ctx, g->F[h], &ld);
    if (st == FIFA_ERR_NOT_SPD || st == FIFA_ERR_TIMEOUT) bad = st;
  }
  if (bad) return fail((fifa_status)bad);
  *out = g;
  return FIFA_OK;
}

extern "C" fifa_status fifa_grid_draw(fifa_ctx* ctx, fifa_grid* g, const double* f_dev, double tau2, uint64_t seed,
                                      uint64_t stream_id, uint64_t iter, int* index_host, double* probs_host) {
  if (!ctx || !g || !f_dev || !index_host || !(tau2 > 0.0)) return FIFA_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  Plan* P = g->F[0]->plan;
  const int64_t n = P->n;
  fifa_status st = ensure_scratch(ctx, P);
  if (st != FIFA_OK) return st;
  Scratch S = carve(ctx, P);
  for (int h = 0; h < g->G; ++h) {
    CK(cudaMemcpyAsync(g->tmp, f_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if ((st = sweep_enqueue(ctx, g->F[h], 0, 1, g->tmp, 1)) != FIFA_OK) return st;
    CK(launch_sumsq(g->tmp, nullptr, n, S.red, g->quad + h, s));
  }
  k_grid_draw<<<1, 32, 0, s>>>(g->logdet, g->quad, g->lprior, g->G, tau2, seed, iter, stream_id, g->probs, g->index);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->host_flags, g->index, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (probs_host) CK(cudaMemcpyAsync(probs_host, g->probs, sizeof(double) * g->G, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *index_host = ctx->host_flags[0];
  return FIFA_OK;
}

extern "C" fifa_status fifa_grid_get(const fifa_grid* g, int h, const fifa_hmat** C, const fifa_fact** W) {
  if (!g || h < 0 || h >= g->G) return FIFA_ERR_INVALID_ARG;
  if (C) *C = g->H[h];
  if (W) *W = g->F[h];
  return FIFA_OK;
}

extern "C" void fifa_destroy_grid(fifa_ctx* ctx, fifa_grid* g) {
  if (!ctx || !g) return;
  cudaStreamSynchronize(ctx->stream);
  for (fifa_fact* F : g->F) fifa_destroy_fact(ctx, F);
  for (fifa_hmat* H : g->H) fifa_destroy_hmat(ctx, H);
  ctx->arena.release(g->x);
  ctx->arena.release(g->tmp);
  ctx->arena.release(g->logdet);
  ctx->arena.release(g->quad);
  ctx->arena.release(g->lprior);
  ctx->arena.release(g->probs);
  ctx->arena.release(g->index);
  delete g;
}
