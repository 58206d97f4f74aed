// Tensor product of 1-D GPs for d-dimensional inputs (Sec. 4.2, Eq.
// tensor_prod):
//   y_i = beta f_1(x_{1,i}) ... f_d(x_{d,i}) + e_i,  e_i ~ N(0, sigma2),
//   f_h ~ GP(m_h, C(rho_h))  (unit variance; m_h = 1).
// Block update of f_h: with g_i = beta prod_{k != h} f_k(x_{k,i}), y_i / g_i
// observes f_h(x_{h,i}) with precision d_i = g_i^2 / sigma2, so f_h - m_h is
// drawn by Algorithm 1.h (Appendix "Heteroskedastic noise derivation") with
// K~ = C~(rho_h), D = diag(d) and data y / g - m_h, on the sorted x_h.
// One sweep: f_1 .. f_d; beta | y, F (normal prior, conjugate); sigma2 | y, F,
// beta; then for every block the Metropolis step on log rho_h with tau2 = 1 and
// q = (f_h - m_h)^T C~_h^-1 (f_h - m_h).  Block h draws from Philox stream id h,
// sigma2 from stream id d, beta from stream id d + 1 (tag 0), all at the sweep
// index.  A zero product g_i carries no information on f_h: the sweep reports
// FIFA_ERR_INVALID_ARG.
//
// Each block is a Gibbs chain on its sorted coordinate (its C~, factor, the
// proposal and the Metropolis state); its M~ view holds P~ = C~ + D^-1 (the
// per-row diagonal 1/d), refactored every sweep.  The sweep is one CUDA graph.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/fifa.h"
#include "fifa_api_internal.h"
#include "fifa_chain.h"
#include "fifa_chain_impl.h"
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

#define TENSOR_RED_BLOCKS 128
#define TENSOR_TRACE_G 4  // sweep, beta, sigma2, rss

// Shared state of the model (device): beta and its prior, sigma2 and its prior.
struct TensorDev {
  double beta, beta_mu, beta_sd;
  double sigma2, a_sigma2, b_sigma2;
  double gg, gy, rss;
  uint64_t seed, iter;
  int64_t n;
  int d, status;
  double* trace;  // CHAIN_TRACE_CAP rows of TENSOR_TRACE_G
};

struct fifa_tensor {
  int d = 0;
  int64_t n = 0;
  fifa_chain* blk[FIFA_ADDITIVE_MAX_D] = {};
  int64_t* perm = nullptr;  // d x n
  double* F = nullptr;      // n x d, column h at F + h n, original order
  double* y = nullptr;
  double* dd = nullptr;     // d x n: precisions of each block, sorted order
  double* dinv = nullptr;   // d x n: their inverses (the diagonal of P~)
  double* part = nullptr;   // 2 x TENSOR_RED_BLOCKS partial sums
  TensorDev* g = nullptr;
  ChainDev** blk_dev = nullptr;
  double* gtrace = nullptr;
  uint64_t iter_host = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_failed = false;
};

static inline int tgrid(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 8); }

// Block h's data in its sorted order: g = beta prod_{k != h} F[p, k] (k
// ascending), yt = y[p] / g - m, d = g^2 / sigma2, dinv = 1 / d.
__global__ void k_tensor_data(const double* __restrict__ y, const double* __restrict__ F,
                              const int64_t* __restrict__ perm, int64_t n, int d, int h, double m,
                              TensorDev* __restrict__ G, double* __restrict__ yt, double* __restrict__ dd,
                              double* __restrict__ dinv) {
  const double beta = G->beta, s2 = G->sigma2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = perm[i];
    double prod = 1.0;
    for (int k = 0; k < d; ++k)
      if (k != h) prod *= F[(int64_t)k * n + p];
    const double g = beta * prod;
    if (g == 0.0) {
      atomicOr(&G->status, 1);
      yt[i] = 0.0;
      dd[i] = 1.0;
      dinv[i] = 1.0;
      continue;
    }
    yt[i] = y[p] / g - m;
    const double di = g * g / s2;
    dd[i] = di;
    dinv[i] = 1.0 / di;
  }
}

// P~ = C~ + diag(dinv) (tau2 = 1), refactored this sweep.
__global__ void k_tensor_view(const HmatDesc* __restrict__ Hc, HmatDesc* __restrict__ Pv, const double* dinv,
                              ChainDev* __restrict__ c) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  HmatDesc v = *Hc;
  v.scale = 1.0;
  v.shift = 0.0;
  v.diag = dinv;
  *Pv = v;
  c->fm_skip = 0;
  c->refreshed = 1;
}

// F[perm[i], h] = m + g[i]
__global__ void k_tensor_scatter(const double* __restrict__ g, const int64_t* __restrict__ perm, int64_t n, double m,
                                 double* __restrict__ Fh) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Fh[perm[i]] = m + g[i];
}

// Partial sums of G^2 and G y, G_i = prod_h F[i, h] (h ascending).
__global__ void k_tensor_gsums(const double* __restrict__ y, const double* __restrict__ F, int64_t n, int d,
                               double* __restrict__ part) {
  __shared__ double red[40];
  double gg = 0.0, gy = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double G = 1.0;
    for (int k = 0; k < d; ++k) G *= F[(int64_t)k * n + i];
    gg += G * G;
    gy += G * y[i];
  }
  gg = block_sum(gg, red);
  gy = block_sum(gy, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = gg;
    part[TENSOR_RED_BLOCKS + blockIdx.x] = gy;
  }
}

// beta | y, F: prior N(mu, sd^2), data y = beta G + e  (one thread).
__global__ void k_tensor_beta(TensorDev* __restrict__ G, const double* __restrict__ part) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double gg = 0.0, gy = 0.0;
  for (int b = 0; b < TENSOR_RED_BLOCKS; ++b) {
    gg += part[b];
    gy += part[TENSOR_RED_BLOCKS + b];
  }
  G->gg = gg;
  G->gy = gy;
  const double prec = 1.0 / (G->beta_sd * G->beta_sd) + gg / G->sigma2;
  const double v = 1.0 / prec;
  const double m = v * (G->beta_mu / (G->beta_sd * G->beta_sd) + gy / G->sigma2);
  G->beta = m + sqrt(v) * philox_normal(G->seed, 0u, 0u, G->iter, (uint64_t)G->d + 1);
}

// Partial sums of (y - beta G)^2.
__global__ void k_tensor_rss(const double* __restrict__ y, const double* __restrict__ F, int64_t n, int d,
                             const TensorDev* __restrict__ G, double* __restrict__ part) {
  __shared__ double red[40];
  const double beta = G->beta;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double P = 1.0;
    for (int k = 0; k < d; ++k) P *= F[(int64_t)k * n + i];
    const double r = y[i] - beta * P;
    acc += r * r;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// sigma2 | y, F, beta (stream id d), copied into every block; the trace row
// (sweep, beta, sigma2, rss); the sweep counter advances.
__global__ void k_tensor_sigma2(TensorDev* __restrict__ G, const double* __restrict__ part, ChainDev* const* blocks) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double rss = 0.0;
  for (int b = 0; b < TENSOR_RED_BLOCKS; ++b) rss += part[b];
  G->rss = rss;
  const double shape = G->a_sigma2 + 0.5 * (double)G->n;
  const double scale = G->b_sigma2 + 0.5 * rss;
  const double s2 = scale / gamma_mt(shape, G->seed, 2u, G->iter, (uint64_t)G->d);
  G->sigma2 = s2;
  for (int k = 0; k < G->d; ++k) blocks[k]->sigma2 = s2;
  if (G->trace) {
    double* row = G->trace + (size_t)(G->iter % CHAIN_TRACE_CAP) * TENSOR_TRACE_G;
    row[0] = (double)G->iter;
    row[1] = G->beta;
    row[2] = s2;
    row[3] = rss;
  }
  G->iter += 1;
}

static fifa_status tensor_sweep_enqueue(fifa_ctx* ctx, fifa_tensor* T) {
  const int64_t n = T->n;
  const int d = T->d;
  cudaStream_t s = ctx->stream;
  fifa_status st = FIFA_OK;
  for (int h = 0; h < d && st == FIFA_OK; ++h) {
    fifa_chain* ch = T->blk[h];
    double* dd = T->dd + (size_t)h * n;
    double* di = T->dinv + (size_t)h * n;
    k_tensor_data<<<tgrid(n), 256, 0, s>>>(T->y, T->F, T->perm + (size_t)h * n, n, d, h, 1.0, T->g, ch->y, dd, di);
    k_tensor_view<<<1, 32, 0, s>>>(ch->H[0]->dev, ch->Mv->dev, di, ch->dev);
    CK(cudaGetLastError());
    ctx->active_scratch = ch->scratch;
    st = fact_enqueue(ctx, ch->FM, ch->Mv->dev);
    if (st == FIFA_OK)
      st = sample_hetero_enqueue(ctx, ch->H[0], ch->F[0], ch->FM, ch->y, 1.0, dd, ch->init.seed, (uint64_t)h,
                                 &ch->dev->iter, 0, ch->f, ch->mean, &ch->dev->refine_res, &ch->dev->pcg_iters);
    if (st == FIFA_OK) {
      k_tensor_scatter<<<tgrid(n), 256, 0, s>>>(ch->f, T->perm + (size_t)h * n, n, 1.0, T->F + (size_t)h * n);
      CK(cudaGetLastError());
    }
  }
  if (st == FIFA_OK) {
    k_tensor_gsums<<<TENSOR_RED_BLOCKS, 256, 0, s>>>(T->y, T->F, n, d, T->part);
    k_tensor_beta<<<1, 32, 0, s>>>(T->g, T->part);
    k_tensor_rss<<<TENSOR_RED_BLOCKS, 256, 0, s>>>(T->y, T->F, n, d, T->g, T->part);
    k_tensor_sigma2<<<1, 32, 0, s>>>(T->g, T->part, T->blk_dev);
    CK(cudaGetLastError());
  }
  // the Metropolis step on every log rho_h (tau2 = 1: the block's tau2 is never drawn)
  for (int h = 0; h < d && st == FIFA_OK; ++h) {
    fifa_chain* ch = T->blk[h];
    ctx->active_scratch = ch->scratch;
    Scratch S = carve(ctx, ch->plan);
    CK(cudaMemcpyAsync(ch->tmp, ch->f, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    st = sweep_enqueue(ctx, ch->F[0], 0, 1, ch->tmp, 1);
    if (st == FIFA_OK) {
      CK(launch_sumsq(ch->tmp, nullptr, n, S.red, &ch->dev->q, s));
      CK(launch_chain_propose(ch->dev, ch->H[1]->dev, s));
      st = hmat_assemble_enqueue(ctx, ch->H[1]);
    }
    if (st == FIFA_OK) st = fact_enqueue(ctx, ch->F[1], ch->H[1]->dev);
    if (st == FIFA_OK) st = chain_phase_hyper_post(ctx, ch, S);
  }
  ctx->active_scratch = nullptr;
  if (st == FIFA_ERR_CUDA) ctx->last_cuda = cudaGetLastError();
  return st;
}

extern "C" fifa_status fifa_tensor_create(fifa_ctx* ctx, const double* X_dev, const double* y_dev, int64_t n, int d,
                                          const fifa_hyper* init, const fifa_prior* prior, double beta0,
                                          double beta_mu, double beta_sd, uint64_t seed, fifa_tensor** out) {
  if (!ctx || !X_dev || !y_dev || !init || !prior || !out || n < 2 || d < 1 || d > FIFA_ADDITIVE_MAX_D)
    return FIFA_ERR_INVALID_ARG;
  if (!(beta_sd > 0.0) || !isfinite(beta0) || !isfinite(beta_mu)) return FIFA_ERR_INVALID_ARG;
  *out = nullptr;
  if (ctx->capturing) return FIFA_ERR_INVALID_ARG;
  fifa_tensor* T = new (std::nothrow) fifa_tensor();
  if (!T) return FIFA_ERR_OOM;
  T->d = d;
  T->n = n;
  auto fail = [&](fifa_status e) {
    fifa_destroy_tensor(ctx, T);
    return e;
  };
  cudaStream_t s = ctx->stream;
  T->perm = (int64_t*)ctx->arena.alloc(sizeof(int64_t) * n * d);
  T->F = (double*)ctx->arena.alloc(sizeof(double) * n * d);
  T->y = (double*)ctx->arena.alloc(sizeof(double) * n);
  T->dd = (double*)ctx->arena.alloc(sizeof(double) * n * d);
  T->dinv = (double*)ctx->arena.alloc(sizeof(double) * n * d);
  T->part = (double*)ctx->arena.alloc(sizeof(double) * 2 * TENSOR_RED_BLOCKS);
  T->g = (TensorDev*)ctx->arena.alloc(sizeof(TensorDev));
  T->blk_dev = (ChainDev**)ctx->arena.alloc(sizeof(ChainDev*) * FIFA_ADDITIVE_MAX_D);
  T->gtrace = (double*)ctx->arena.alloc(sizeof(double) * CHAIN_TRACE_CAP * TENSOR_TRACE_G);
  if (!T->perm || !T->F || !T->y || !T->dd || !T->dinv || !T->part || !T->g || !T->blk_dev || !T->gtrace)
    return fail(FIFA_ERR_OOM);
  CK(cudaMemcpyAsync(T->y, y_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  std::vector<double> ones((size_t)n * d, 1.0);  // every f_h starts at its prior mean 1
  CK(cudaMemcpyAsync(T->F, ones.data(), sizeof(double) * n * d, cudaMemcpyHostToDevice, s));
  std::vector<double> xk(n), xs(n);
  std::vector<int64_t> idx(n);
  fifa_hyper bi = *init;
  bi.tau2 = 1.0;  // unit-variance blocks
  for (int h = 0; h < d; ++h) {
    CK(cudaMemcpyAsync(xk.data(), X_dev + (size_t)h * n, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < n; ++i)
      if (!std::isfinite(xk[i])) return fail(FIFA_ERR_INVALID_ARG);
    std::iota(idx.begin(), idx.end(), (int64_t)0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return xk[a] < xk[b]; });
    for (int64_t i = 0; i < n; ++i) xs[i] = xk[idx[i]];
    CK(cudaMemcpyAsync(T->perm + (size_t)h * n, idx.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(T->dd, xs.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));  // staging
    CK(cudaStreamSynchronize(s));
    // blocks are stepped phase by phase: no proposal-overlap resources
    const int ov = ctx->opts.overlap_proposal;
    ctx->opts.overlap_proposal = 0;
    fifa_status st = fifa_chain_create(ctx, T->dd, T->y, n, &bi, prior, seed, (uint64_t)h, &T->blk[h]);
    ctx->opts.overlap_proposal = ov;
    if (st != FIFA_OK) return fail(st);
  }
  ChainDev* ptrs[FIFA_ADDITIVE_MAX_D] = {};
  for (int h = 0; h < d; ++h) ptrs[h] = T->blk[h]->dev;
  CK(cudaMemcpyAsync(T->blk_dev, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice, s));
  TensorDev g;
  memset(&g, 0, sizeof(g));
  g.beta = beta0;
  g.beta_mu = beta_mu;
  g.beta_sd = beta_sd;
  g.sigma2 = init->sigma2;
  g.a_sigma2 = prior->a_sigma2;
  g.b_sigma2 = prior->b_sigma2;
  g.seed = seed;
  g.n = n;
  g.d = d;
  g.trace = T->gtrace;
  CK(cudaMemcpyAsync(T->g, &g, sizeof(TensorDev), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  *out = T;
  return FIFA_OK;
}

static void tensor_build_graph(fifa_ctx* ctx, fifa_tensor* T) {
  if (T->exec || T->graph_failed) return;
  cudaStream_t s = ctx->stream;
  if (s == nullptr || cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    T->graph_failed = true;
    return;
  }
  ctx->capturing = true;
  fifa_status st = tensor_sweep_enqueue(ctx, T);
  ctx->capturing = false;
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &gr);
  if (st != FIFA_OK || e != cudaSuccess || !gr || cudaGraphInstantiate(&T->exec, gr, 0) != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    T->exec = nullptr;
    T->graph_failed = true;
    return;
  }
  T->graph = gr;
}

extern "C" fifa_status fifa_tensor_sweep(fifa_ctx* ctx, fifa_tensor* T, int sweeps, double* trace_host) {
  if (!ctx || !T || sweeps < 0 || ctx->capturing) return FIFA_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  tensor_build_graph(ctx, T);
  const int d = T->d;
  const int TF = FIFA_TENSOR_TRACE_FIELDS(d);
  std::vector<double> gt, bt;
  int done = 0;
  while (done < sweeps) {
    const int chunk = std::min(sweeps - done, CHAIN_TRACE_CAP);
    for (int k = 0; k < chunk; ++k) {
      if (T->exec) {
        CK(cudaGraphLaunch(T->exec, s));
      } else {
        fifa_status st = tensor_sweep_enqueue(ctx, T);
        if (st != FIFA_OK) return st;
      }
    }
    if (trace_host) {
      gt.assign((size_t)chunk * TENSOR_TRACE_G, 0.0);
      bt.assign((size_t)chunk * CHAIN_TRACE_FIELDS * d, 0.0);
      const uint64_t first = T->iter_host % CHAIN_TRACE_CAP;
      const uint64_t n1 = std::min<uint64_t>(chunk, CHAIN_TRACE_CAP - first);
      auto fetch = [&](double* dst, const double* ring, int fields) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dst, ring + first * fields, sizeof(double) * n1 * fields,
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && n1 < (uint64_t)chunk)
          e = cudaMemcpyAsync(dst + n1 * fields, ring, sizeof(double) * (chunk - n1) * fields, cudaMemcpyDeviceToHost,
                              s);
        return e;
      };
      CK(fetch(gt.data(), T->gtrace, TENSOR_TRACE_G));
      for (int h = 0; h < d; ++h)
        CK(fetch(bt.data() + (size_t)h * chunk * CHAIN_TRACE_FIELDS, T->blk[h]->trace, CHAIN_TRACE_FIELDS));
      CK(cudaStreamSynchronize(s));
      for (int t = 0; t < chunk; ++t) {
        double* row = trace_host + (size_t)(done + t) * TF;
        for (int q = 0; q < TENSOR_TRACE_G; ++q) row[q] = gt[(size_t)t * TENSOR_TRACE_G + q];
        int status = 0;
        for (int h = 0; h < d; ++h) {
          const double* br = bt.data() + ((size_t)h * chunk + t) * CHAIN_TRACE_FIELDS;
          status |= (int)br[10];
          row[5 + h] = br[3];
          row[5 + d + h] = br[4];
        }
        row[4] = (double)status;
      }
    }
    T->iter_host += chunk;
    for (int h = 0; h < d; ++h) T->blk[h]->iter_host += chunk;
    done += chunk;
  }
  TensorDev g;
  CK(cudaMemcpyAsync(&g, T->g, sizeof(TensorDev), cudaMemcpyDeviceToHost, s));
  int cs = 0;
  for (int h = 0; h < d; ++h) {
    CK(cudaMemcpyAsync(ctx->host_flags + h % 32, &T->blk[h]->dev->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    cs |= ctx->host_flags[h % 32];
  }
  if (g.status) return FIFA_ERR_INVALID_ARG;
  if (cs & FIFA_DEV_TIMEOUT) return FIFA_ERR_TIMEOUT;
  if (cs & FIFA_DEV_NOT_SPD) return FIFA_ERR_NOT_SPD;
  return FIFA_OK;
}

extern "C" fifa_status fifa_tensor_get(fifa_ctx* ctx, const fifa_tensor* T, double* F_dev, double* beta_host,
                                       double* sigma2_host, fifa_hyper* blocks_host) {
  if (!ctx || !T) return FIFA_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  if (F_dev) CK(cudaMemcpyAsync(F_dev, T->F, sizeof(double) * T->n * T->d, cudaMemcpyDeviceToDevice, s));
  TensorDev g;
  CK(cudaMemcpyAsync(&g, T->g, sizeof(TensorDev), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (beta_host) *beta_host = g.beta;
  if (sigma2_host) *sigma2_host = g.sigma2;
  if (blocks_host)
    for (int h = 0; h < T->d; ++h) {
      fifa_status st = fifa_chain_get(ctx, T->blk[h], nullptr, nullptr, &blocks_host[h]);
      if (st != FIFA_OK) return st;
    }
  return FIFA_OK;
}

extern "C" void fifa_destroy_tensor(fifa_ctx* ctx, fifa_tensor* T) {
  if (!ctx || !T) return;
  cudaStreamSynchronize(ctx->stream);
  if (T->exec) cudaGraphExecDestroy(T->exec);
  if (T->graph) cudaGraphDestroy(T->graph);
  for (int h = 0; h < T->d; ++h)
    if (T->blk[h]) fifa_destroy_chain(ctx, T->blk[h]);
  ctx->arena.release(T->perm);
  ctx->arena.release(T->F);
  ctx->arena.release(T->y);
  ctx->arena.release(T->dd);
  ctx->arena.release(T->dinv);
  ctx->arena.release(T->part);
  ctx->arena.release(T->g);
  ctx->arena.release(T->blk_dev);
  ctx->arena.release(T->gtrace);
  delete T;
}
