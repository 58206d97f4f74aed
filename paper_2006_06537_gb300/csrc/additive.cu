// Additive model of d one-dimensional GP blocks (Sec. 4.2 allows an additive
// model in place of the tensor-product kernel):
//   y = sum_k f_k(x_k) + e,  e ~ N(0, sigma2 I),  f_k ~ GP(0, tau2_k C(rho_k)).
// One block-Gibbs sweep:
//   for k = 0..d-1: r = y - sum_{j != k} f_j, sorted by x_k; f_k | r by
//                   Algorithm 1 with (tau2_k, sigma2, rho_k); scattered back
//   sigma2 | y, f_1..f_d
//   for k:          tau2_k | f_k, then the Metropolis step on log rho_k
// Each block is a Gibbs chain on its sorted coordinate (Philox stream id k);
// the shared sigma2 has its own small state (stream id d).  The sweep is
// captured once in a CUDA graph and replayed.  The blocks' M~ factorizations
// depend only on the hyperparameters: all d are factored in one batched pass
// (one launch per step and tree level for every block, the blocks' descriptors
// and scratch laid out contiguously); so are the d proposals C~(rho'_k).  On a context with independent CTAs the
// factorizations and the blocks' tau2 / rho updates instead run as concurrent
// graph branches, one per block.
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

#define CK(call)                 \
  do {                           \
    cudaError_t e_ = (call);     \
    if (e_ != cudaSuccess) {     \
      ctx->last_cuda = e_;       \
      return FIFA_ERR_CUDA;      \
    }                            \
  } while (0)

#define ADD_TRACE_FIELDS_G 3

struct fifa_additive {
  int d = 0;
  int64_t n = 0;
  fifa_chain* blk[FIFA_ADDITIVE_MAX_D] = {};
  int64_t* perm = nullptr;  // d x n
  double* F = nullptr;      // n x d, column k at F + k n, original order
  double* y = nullptr;
  double* res = nullptr;
  ChainDev* g = nullptr;  // shared sigma2 state
  ChainDev** blk_dev = nullptr;
  double* gtrace = nullptr;
  uint64_t iter_host = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_failed = false;
  // concurrent branches (contexts with independent CTAs only): one stream and
  // fork / join events per block
  cudaStream_t side[FIFA_ADDITIVE_MAX_D] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[FIFA_ADDITIVE_MAX_D] = {};
  bool branches = false;
  // batched factorization of the blocks' M~ (all blocks share one plan): the
  // blocks' M~ factor and view descriptors and their scratch are contiguous
  FactDesc* fm_desc = nullptr;  // d
  FactDesc* fm32_desc = nullptr;  // d: their FP32 copies (mixed precision), else null
  HmatDesc* mv_desc = nullptr;  // d
  FactDesc* f_desc[2] = {nullptr, nullptr};  // d each: current / proposal factor of C~
  HmatDesc* h_desc[2] = {nullptr, nullptr};  // d each: current / proposal C~
  char* scratch = nullptr;      // d * scratch_stride
  size_t scratch_stride = 0;
  // the blocks' tau2 / rho sweeps of f as one launch (sweep_batch_config;
  // fsb_ls < 0: one sweep per block): the blocks' copies of f
  double** tmp_list = nullptr;  // d device pointers
  int fsb_ls = -1, fsb_rows = 0;
  // the prior part of every block's Algorithm 1 (normals, C~ a, W_C b, rhs0)
  // in shared launches: the blocks' vectors (device arrays) and the fused
  // product's grid for d problems (mvb_ls < 0: one product per block)
  Alg1Prior* prior = nullptr;    // d
  double** vec_lists = nullptr;  // 3 d: a, b, Ca of every block
  int mvb_ls = -1, mvb_rows = 0;
};

// Enqueue fn(k) for every block k, as concurrent branches forked from and
// joined back into ctx->stream when the model has branches, else in order.
template <typename Fn>
static fifa_status for_blocks(fifa_ctx* ctx, fifa_additive* A, Fn fn) {
  if (!A->branches) {
    for (int k = 0; k < A->d; ++k) {
      fifa_status st = fn(k);
      if (st != FIFA_OK) return st;
    }
    return FIFA_OK;
  }
  cudaStream_t main = ctx->stream;
  if (cudaEventRecord(A->ev_fork, main) != cudaSuccess) return FIFA_ERR_CUDA;
  fifa_status st = FIFA_OK;
  for (int k = 0; k < A->d && st == FIFA_OK; ++k) {
    if (cudaStreamWaitEvent(A->side[k], A->ev_fork, 0) != cudaSuccess) {
      st = FIFA_ERR_CUDA;
      break;
    }
    ctx->stream = A->side[k];
    st = fn(k);
    ctx->stream = main;
    if (st == FIFA_OK && (cudaEventRecord(A->ev_join[k], A->side[k]) != cudaSuccess ||
                          cudaStreamWaitEvent(main, A->ev_join[k], 0) != cudaSuccess))
      st = FIFA_ERR_CUDA;
  }
  ctx->stream = main;
  return st;
}

static fifa_status additive_sweep_enqueue(fifa_ctx* ctx, fifa_additive* A) {
  const int64_t n = A->n;
  const int d = A->d;
  fifa_status st = FIFA_OK;
  // M~_k = (tau2_k / sigma2) C~_k + I and its factor for every block: they
  // depend only on the hyperparameters, so all blocks are factored together,
  // one launch per tree level for all d blocks
  if (A->fm_desc) {
    for (int k = 0; k < d && st == FIFA_OK; ++k) {
      fifa_chain* ch = A->blk[k];
      if (launch_chain_make_view(ch->H[0]->dev, ch->Mv->dev, ch->dev, ctx->stream) != cudaSuccess) st = FIFA_ERR_CUDA;
    }
    if (st == FIFA_OK)
      st = fact_enqueue_batched(ctx, A->blk[0]->plan, A->fm_desc, A->mv_desc, d, A->scratch, A->scratch_stride,
                                A->fm32_desc);
  } else {
    st = for_blocks(ctx, A, [&](int k) {
      ctx->active_scratch = A->blk[k]->scratch;
      return chain_phase_factor_m(ctx, A->blk[k]);
    });
  }
  // the data-independent part of every block's draw (normals, C~_k a_k,
  // W_{C,k} b_k and the first right-hand side) at once
  if (st == FIFA_OK && A->prior) {
    const fifa_hmat* Ce[FIFA_ADDITIVE_MAX_D];
    const fifa_fact* We[FIFA_ADDITIVE_MAX_D];
    for (int k = 0; k < d; ++k) {
      Ce[k] = A->blk[k]->H[0];
      We[k] = A->blk[k]->F[0];
    }
    st = sample_prior_batched(ctx, A->blk[0]->plan, A->h_desc[0], A->f_desc[0], A->prior, A->vec_lists,
                              A->vec_lists + d, A->vec_lists + 2 * d, d, A->blk[0]->init.seed, A->fsb_ls, A->fsb_rows,
                              A->mvb_ls, A->mvb_rows, A->scratch, A->scratch_stride, Ce, We);
  }
  // f_k | y - sum_{j != k} f_j, blocks in order (block Gibbs)
  for (int k = 0; k < d && st == FIFA_OK; ++k) {
    fifa_chain* ch = A->blk[k];
    if (launch_add_gather(A->y, A->F, A->perm + (size_t)k * n, n, d, k, ch->y, ctx->stream) != cudaSuccess) {
      st = FIFA_ERR_CUDA;
      break;
    }
    ctx->active_scratch = ch->scratch;
    st = A->prior ? chain_phase_sample_data(ctx, ch) : chain_phase_sample(ctx, ch);
    if (st == FIFA_OK &&
        launch_add_scatter(ch->f, A->perm + (size_t)k * n, n, A->F + (size_t)k * n, ctx->stream) != cudaSuccess)
      st = FIFA_ERR_CUDA;
  }
  // shared sigma2
  if (st == FIFA_OK) {
    ctx->active_scratch = A->blk[0]->scratch;
    Scratch S = carve(ctx, A->blk[0]->plan);
    if (launch_add_residual(A->y, A->F, n, d, A->res, ctx->stream) != cudaSuccess ||
        launch_sumsq(A->res, A->F + (size_t)(d - 1) * n, n, S.red, &A->g->rss, ctx->stream) != cudaSuccess ||
        launch_add_sigma2(A->g, A->blk_dev, d, ctx->stream) != cudaSuccess)
      st = FIFA_ERR_CUDA;
  }
  // tau2_k and rho_k of every block: the blocks' sweeps of f, the proposals'
  // assemblies and their factorizations each in shared launches for all d
  // blocks (they do not depend on one another)
  if (st == FIFA_OK && A->fm_desc) {
    Plan* P = A->blk[0]->plan;
    auto sweeps = [&](int q) -> fifa_status {  // tmp_k = W_{C,k}^-1 f_k with the current (0) / proposal (1) factors
      for (int k = 0; k < d; ++k) {
        fifa_chain* ch = A->blk[k];
        if (cudaMemcpyAsync(ch->tmp, ch->f, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
          return FIFA_ERR_CUDA;
      }
      if (A->fsb_ls >= 0)
        return sweep_enqueue_batched(ctx, P, A->f_desc[q], A->tmp_list, d, 1, A->fsb_ls, A->fsb_rows, A->scratch,
                                     A->scratch_stride);
      for (int k = 0; k < d; ++k) {
        fifa_chain* ch = A->blk[k];
        ctx->active_scratch = ch->scratch;
        fifa_status e = sweep_enqueue(ctx, ch->F[q], 0, 1, ch->tmp, 1);
        if (e != FIFA_OK) return e;
      }
      return FIFA_OK;
    };
    st = sweeps(0);
    for (int k = 0; k < d && st == FIFA_OK; ++k) {
      fifa_chain* ch = A->blk[k];
      ctx->active_scratch = ch->scratch;
      st = chain_hyper_tau2_propose(ctx, ch, carve(ctx, P));
    }
    if (st == FIFA_OK) st = hmat_assemble_batched(ctx, P, A->h_desc[1], d, A->scratch, A->scratch_stride);
    if (st == FIFA_OK) st = fact_enqueue_batched(ctx, P, A->f_desc[1], A->h_desc[1], d, A->scratch, A->scratch_stride);
    if (st == FIFA_OK) st = sweeps(1);
    for (int k = 0; k < d && st == FIFA_OK; ++k) {
      fifa_chain* ch = A->blk[k];
      ctx->active_scratch = ch->scratch;
      st = chain_hyper_mh(ctx, ch, carve(ctx, P));
    }
  } else if (st == FIFA_OK) {
    st = for_blocks(ctx, A, [&](int k) {
      fifa_chain* ch = A->blk[k];
      ctx->active_scratch = ch->scratch;
      Scratch S = carve(ctx, ch->plan);
      return chain_phase_hyper(ctx, ch, S);
    });
  }
  ctx->active_scratch = nullptr;
  if (st == FIFA_ERR_CUDA) ctx->last_cuda = cudaGetLastError();
  return st;
}

extern "C" fifa_status fifa_additive_create(fifa_ctx* ctx, const double* X_dev, const double* y_dev, int64_t n,
                                            int d, const fifa_hyper* init, const fifa_prior* prior, uint64_t seed,
                                            fifa_additive** out) {
  if (!ctx || !X_dev || !y_dev || !init || !prior || !out || n < 2 || d < 1 || d > FIFA_ADDITIVE_MAX_D)
    return FIFA_ERR_INVALID_ARG;
  *out = nullptr;
  if (ctx->capturing) return FIFA_ERR_INVALID_ARG;
  fifa_additive* A = new (std::nothrow) fifa_additive();
  if (!A) return FIFA_ERR_OOM;
  A->d = d;
  A->n = n;
  auto fail = [&](fifa_status e) {
    fifa_destroy_additive(ctx, A);
    return e;
  };
  cudaStream_t s = ctx->stream;
  A->perm = (int64_t*)ctx->arena.alloc(sizeof(int64_t) * n * d);
  A->F = (double*)ctx->arena.alloc(sizeof(double) * n * d);
  A->y = (double*)ctx->arena.alloc(sizeof(double) * n);
  A->res = (double*)ctx->arena.alloc(sizeof(double) * n);
  A->g = (ChainDev*)ctx->arena.alloc(sizeof(ChainDev));
  A->blk_dev = (ChainDev**)ctx->arena.alloc(sizeof(ChainDev*) * FIFA_ADDITIVE_MAX_D);
  A->gtrace = (double*)ctx->arena.alloc(sizeof(double) * CHAIN_TRACE_CAP * ADD_TRACE_FIELDS_G);
  if (!A->perm || !A->F || !A->y || !A->res || !A->g || !A->blk_dev || !A->gtrace) return fail(FIFA_ERR_OOM);
  CK(cudaMemcpyAsync(A->y, y_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(A->F, 0, sizeof(double) * n * d, s));
  CK(cudaMemsetAsync(A->res, 0, sizeof(double) * n, s));
  // per block: stable sort of coordinate k (ties keep the lower point index first)
  std::vector<double> xk(n), xs(n);
  std::vector<int64_t> idx(n);
  for (int k = 0; k < d; ++k) {
    CK(cudaMemcpyAsync(xk.data(), X_dev + (size_t)k * n, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < n; ++i)
      if (!std::isfinite(xk[i])) return fail(FIFA_ERR_INVALID_ARG);
    std::iota(idx.begin(), idx.end(), (int64_t)0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return xk[a] < xk[b]; });
    for (int64_t i = 0; i < n; ++i) xs[i] = xk[idx[i]];
    CK(cudaMemcpyAsync(A->perm + (size_t)k * n, idx.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(A->res, xs.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    // the block's data buffer is overwritten by the partial residual every sweep;
    // blocks are stepped phase by phase, so they take no proposal-overlap resources
    const int ov = ctx->opts.overlap_proposal;
    ctx->opts.overlap_proposal = 0;
    fifa_status st = fifa_chain_create(ctx, A->res, A->y, n, init, prior, seed, (uint64_t)k, &A->blk[k]);
    ctx->opts.overlap_proposal = ov;
    if (st != FIFA_OK) return fail(st);
  }
  // concurrent block branches only where no kernel's CTAs wait on each other
  if (ctx->opts.independent_ctas && d > 1) {
    A->branches = cudaEventCreateWithFlags(&A->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < d && A->branches; ++k)
      A->branches = cudaStreamCreateWithFlags(&A->side[k], cudaStreamNonBlocking) == cudaSuccess &&
                    cudaEventCreateWithFlags(&A->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!A->branches) return fail(FIFA_ERR_CUDA);
  }
  // contiguous M~ factor / view descriptors and scratch for the batched
  // factorization (the graph is built later, so re-pointing is safe now)
  if (!A->branches && d > 1) {
    const Plan* P = A->blk[0]->plan;
    A->scratch_stride = (P->scratch_bytes + 255) & ~(size_t)255;
    A->fm_desc = (FactDesc*)ctx->arena.alloc(sizeof(FactDesc) * d);
    A->mv_desc = (HmatDesc*)ctx->arena.alloc(sizeof(HmatDesc) * d);
    for (int q = 0; q < 2; ++q) {
      A->f_desc[q] = (FactDesc*)ctx->arena.alloc(sizeof(FactDesc) * d);
      A->h_desc[q] = (HmatDesc*)ctx->arena.alloc(sizeof(HmatDesc) * d);
    }
    A->scratch = (char*)ctx->arena.alloc(A->scratch_stride * d);
    if (!A->fm_desc || !A->mv_desc || !A->f_desc[0] || !A->f_desc[1] || !A->h_desc[0] || !A->h_desc[1] || !A->scratch)
      return fail(FIFA_ERR_OOM);
    if (A->blk[0]->FM->has32 && !(A->fm32_desc = (FactDesc*)ctx->arena.alloc(sizeof(FactDesc) * d)))
      return fail(FIFA_ERR_OOM);
    for (int k = 0; k < d; ++k) {
      fifa_chain* ch = A->blk[k];
      CK(cudaMemcpyAsync(A->fm_desc + k, ch->FM->dev, sizeof(FactDesc), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(A->mv_desc + k, ch->Mv->dev, sizeof(HmatDesc), cudaMemcpyDeviceToDevice, s));
      for (int q = 0; q < 2; ++q) {
        CK(cudaMemcpyAsync(A->f_desc[q] + k, ch->F[q]->dev, sizeof(FactDesc), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(A->h_desc[q] + k, ch->H[q]->dev, sizeof(HmatDesc), cudaMemcpyDeviceToDevice, s));
      }
      if (A->fm32_desc)
        CK(cudaMemcpyAsync(A->fm32_desc + k, ch->FM->dev32, sizeof(FactDesc), cudaMemcpyDeviceToDevice, s));
      CK(cudaStreamSynchronize(s));
      ctx->arena.release(ch->FM->dev);
      ctx->arena.release(ch->Mv->dev);
      ctx->arena.release(ch->scratch);
      if (A->fm32_desc) {
        ctx->arena.release(ch->FM->dev32);
        ch->FM->dev32 = A->fm32_desc + k;
      }
      ch->FM->dev = A->fm_desc + k;
      ch->Mv->dev = A->mv_desc + k;
      for (int q = 0; q < 2; ++q) {
        ctx->arena.release(ch->F[q]->dev);
        ctx->arena.release(ch->H[q]->dev);
        ch->F[q]->dev = A->f_desc[q] + k;
        ch->H[q]->dev = A->h_desc[q] + k;
      }
      ch->scratch = A->scratch + (size_t)k * A->scratch_stride;
    }
    // the blocks' copies of f, for the batched sweeps
    double* tl[FIFA_ADDITIVE_MAX_D] = {};
    for (int k = 0; k < d; ++k) tl[k] = A->blk[k]->tmp;
    if (!(A->tmp_list = (double**)ctx->arena.alloc(sizeof(double*) * d))) return fail(FIFA_ERR_OOM);
    CK(cudaMemcpyAsync(A->tmp_list, tl, sizeof(double*) * d, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    if (!sweep_batch_config(ctx, P, d, &A->fsb_ls, &A->fsb_rows)) A->fsb_ls = -1;
    if (!mv_batch_config(ctx, P, d, &A->mvb_ls, &A->mvb_rows)) A->mvb_ls = -1;
    // the blocks' Algorithm 1 vectors in their scratch (the layout of
    // sample_prior_enqueue: a, b, Ca, rhs at 0, n, 2n, 3n of the scratch vectors)
    Alg1Prior pr[FIFA_ADDITIVE_MAX_D];
    double* vl[3 * FIFA_ADDITIVE_MAX_D];
    for (int k = 0; k < d; ++k) {
      fifa_chain* ch = A->blk[k];
      ctx->active_scratch = ch->scratch;
      Scratch S = carve(ctx, ch->plan);
      ctx->active_scratch = nullptr;
      pr[k] = Alg1Prior{&ch->dev->iter, ch->init.chain_id, S.vec, S.vec + n, S.vec + 2 * n, S.vec + 3 * n,
                        &ch->dev->tau2};
      vl[k] = S.vec;
      vl[d + k] = S.vec + n;
      vl[2 * d + k] = S.vec + 2 * n;
    }
    A->prior = (Alg1Prior*)ctx->arena.alloc(sizeof(Alg1Prior) * d);
    A->vec_lists = (double**)ctx->arena.alloc(sizeof(double*) * 3 * d);
    if (!A->prior || !A->vec_lists) return fail(FIFA_ERR_OOM);
    CK(cudaMemcpyAsync(A->prior, pr, sizeof(Alg1Prior) * d, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(A->vec_lists, vl, sizeof(double*) * 3 * d, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  ChainDev* ptrs[FIFA_ADDITIVE_MAX_D] = {};
  for (int k = 0; k < d; ++k) ptrs[k] = A->blk[k]->dev;
  CK(cudaMemcpyAsync(A->blk_dev, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice, s));
  ChainDev g = A->blk[0]->init;
  g.chain_id = (uint64_t)d;
  g.iter = 0;
  g.rss = 0.0;
  g.trace = A->gtrace;
  g.trace_cap = CHAIN_TRACE_CAP;
  CK(cudaMemcpyAsync(A->g, &g, sizeof(ChainDev), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(A->res, 0, sizeof(double) * n, s));
  CK(cudaStreamSynchronize(s));
  *out = A;
  return FIFA_OK;
}

static void additive_build_graph(fifa_ctx* ctx, fifa_additive* A) {
  if (A->exec || A->graph_failed) return;
  cudaStream_t s = ctx->stream;
  if (s == nullptr || cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    A->graph_failed = true;
    return;
  }
  ctx->capturing = true;
  fifa_status st = additive_sweep_enqueue(ctx, A);
  ctx->capturing = false;
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &gr);
  if (st != FIFA_OK || e != cudaSuccess || !gr || cudaGraphInstantiate(&A->exec, gr, 0) != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    A->exec = nullptr;
    A->graph_failed = true;
    return;
  }
  A->graph = gr;
}

extern "C" fifa_status fifa_additive_sweep(fifa_ctx* ctx, fifa_additive* A, int sweeps, double* trace_host) {
  if (!ctx || !A || sweeps < 0 || ctx->capturing) return FIFA_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  additive_build_graph(ctx, A);
  const int d = A->d;
  const int TF = FIFA_ADDITIVE_TRACE_FIELDS(d);
  std::vector<double> gt, bt;
  int done = 0;
  while (done < sweeps) {
    const int chunk = std::min(sweeps - done, CHAIN_TRACE_CAP);
    for (int k = 0; k < chunk; ++k) {
      if (A->exec) {
        CK(cudaGraphLaunch(A->exec, s));
      } else {
        fifa_status st = additive_sweep_enqueue(ctx, A);
        if (st != FIFA_OK) return st;
      }
    }
    if (trace_host) {
      // rows [first, first + chunk) of the rings, possibly wrapping
      gt.assign((size_t)chunk * ADD_TRACE_FIELDS_G, 0.0);
      bt.assign((size_t)chunk * CHAIN_TRACE_FIELDS * d, 0.0);
      const uint64_t first = A->iter_host % CHAIN_TRACE_CAP;
      const uint64_t n1 = std::min<uint64_t>(chunk, CHAIN_TRACE_CAP - first);
      auto fetch = [&](double* dst, const double* ring, int fields) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dst, ring + first * fields, sizeof(double) * n1 * fields,
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && n1 < (uint64_t)chunk)
          e = cudaMemcpyAsync(dst + n1 * fields, ring, sizeof(double) * (chunk - n1) * fields, cudaMemcpyDeviceToHost,
                              s);
        return e;
      };
      CK(fetch(gt.data(), A->gtrace, ADD_TRACE_FIELDS_G));
      for (int k = 0; k < d; ++k)
        CK(fetch(bt.data() + (size_t)k * chunk * CHAIN_TRACE_FIELDS, A->blk[k]->trace, CHAIN_TRACE_FIELDS));
      CK(cudaStreamSynchronize(s));
      for (int t = 0; t < chunk; ++t) {
        double* row = trace_host + (size_t)(done + t) * TF;
        row[0] = gt[(size_t)t * ADD_TRACE_FIELDS_G + 0];
        row[1] = gt[(size_t)t * ADD_TRACE_FIELDS_G + 1];
        row[2] = gt[(size_t)t * ADD_TRACE_FIELDS_G + 2];
        int status = 0;
        double res = 0.0;
        for (int k = 0; k < d; ++k) {
          const double* br = bt.data() + ((size_t)k * chunk + t) * CHAIN_TRACE_FIELDS;
          status |= (int)br[10];
          res = std::max(res, br[9]);
          row[5 + k] = br[2];
          row[5 + d + k] = br[3];
          row[5 + 2 * d + k] = br[4];
        }
        row[3] = (double)status;
        row[4] = res;
      }
    }
    A->iter_host += chunk;
    for (int k = 0; k < d; ++k) A->blk[k]->iter_host += chunk;
    done += chunk;
  }
  int cs = 0;
  for (int k = 0; k < d; ++k) {
    CK(cudaMemcpyAsync(ctx->host_flags, &A->blk[k]->dev->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    cs |= ctx->host_flags[0];
  }
  if (cs & FIFA_DEV_TIMEOUT) return FIFA_ERR_TIMEOUT;
  if (cs & FIFA_DEV_NOT_SPD) return FIFA_ERR_NOT_SPD;
  return FIFA_OK;
}

extern "C" fifa_status fifa_additive_get(fifa_ctx* ctx, const fifa_additive* A, double* F_dev, double* sigma2_host,
                                         fifa_hyper* blocks_host) {
  if (!ctx || !A) return FIFA_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  if (F_dev) CK(cudaMemcpyAsync(F_dev, A->F, sizeof(double) * A->n * A->d, cudaMemcpyDeviceToDevice, s));
  ChainDev g;
  CK(cudaMemcpyAsync(&g, A->g, sizeof(ChainDev), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (sigma2_host) *sigma2_host = g.sigma2;
  if (blocks_host)
    for (int k = 0; k < A->d; ++k) {
      fifa_status st = fifa_chain_get(ctx, A->blk[k], nullptr, nullptr, &blocks_host[k]);
      if (st != FIFA_OK) return st;
    }
  return FIFA_OK;
}

extern "C" fifa_status fifa_additive_kernel_nodes(const fifa_additive* A, int* out_host) {
  if (!A || !out_host) return FIFA_ERR_INVALID_ARG;
  *out_host = -1;
  if (!A->graph) return FIFA_OK;
  size_t count = 0;
  if (cudaGraphGetNodes(A->graph, nullptr, &count) != cudaSuccess) return FIFA_ERR_CUDA;
  std::vector<cudaGraphNode_t> nodes(count);
  if (count && cudaGraphGetNodes(A->graph, nodes.data(), &count) != cudaSuccess) return FIFA_ERR_CUDA;
  int kernels = 0;
  for (size_t i = 0; i < count; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
  }
  *out_host = kernels;
  return FIFA_OK;
}

extern "C" void fifa_destroy_additive(fifa_ctx* ctx, fifa_additive* A) {
  if (!ctx || !A) return;
  cudaStreamSynchronize(ctx->stream);
  if (A->exec) cudaGraphExecDestroy(A->exec);
  if (A->graph) cudaGraphDestroy(A->graph);
  for (int k = 0; k < A->d; ++k)
    if (A->blk[k]) {
      if (A->fm_desc) {  // these point into the model's shared arrays, released below
        A->blk[k]->FM->dev = nullptr;
        if (A->fm32_desc) A->blk[k]->FM->dev32 = nullptr;
        A->blk[k]->Mv->dev = nullptr;
        for (int q = 0; q < 2; ++q) {
          A->blk[k]->F[q]->dev = nullptr;
          A->blk[k]->H[q]->dev = nullptr;
        }
        A->blk[k]->scratch = nullptr;
      }
      fifa_destroy_chain(ctx, A->blk[k]);
    }
  ctx->arena.release(A->fm_desc);
  ctx->arena.release(A->fm32_desc);
  ctx->arena.release(A->mv_desc);
  for (int q = 0; q < 2; ++q) {
    ctx->arena.release(A->f_desc[q]);
    ctx->arena.release(A->h_desc[q]);
  }
  ctx->arena.release(A->scratch);
  ctx->arena.release(A->tmp_list);
  ctx->arena.release(A->prior);
  ctx->arena.release(A->vec_lists);
  for (int k = 0; k < FIFA_ADDITIVE_MAX_D; ++k) {
    if (A->side[k]) cudaStreamDestroy(A->side[k]);
    if (A->ev_join[k]) cudaEventDestroy(A->ev_join[k]);
  }
  if (A->ev_fork) cudaEventDestroy(A->ev_fork);
  ctx->arena.release(A->perm);
  ctx->arena.release(A->F);
  ctx->arena.release(A->y);
  ctx->arena.release(A->res);
  ctx->arena.release(A->g);
  ctx->arena.release(A->blk_dev);
  ctx->arena.release(A->gtrace);
  delete A;
}
