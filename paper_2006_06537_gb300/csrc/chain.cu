// Gibbs chain: device-resident state and one iteration captured in a CUDA graph.
//
// Per iteration (Sec. 4.1, in the order of Eqs. posterior_gibs1-4):
//   M~ = s C~ + I view (s = tau2 / sigma2) and its FP64 factor (mixed: kept from
//   an earlier iteration unless it must be refreshed, plus its FP32 copy)
//   f by Algorithm 1 (Philox a, b; C~ a, W_C b, two-right-hand-side solve, C~ r)
//   sigma2 | y, f ;  q = ||W_C^-1 f||^2 ;  tau2 | f
//   propose rho', assemble C~(rho') (leaves + ACA), factor it, q' = ||W'^-1 f||^2
//   Metropolis accept / reject (descriptor swap on the device)
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
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

// Phase 1a: M~ = (tau2 / sigma2) C~ + I and its factor.
fifa_status chain_phase_factor_m(fifa_ctx* ctx, fifa_chain* ch) {
  if (launch_chain_make_view(ch->H[0]->dev, ch->Mv->dev, ch->dev, ctx->stream) != cudaSuccess) return FIFA_ERR_CUDA;
  return fact_enqueue(ctx, ch->FM, ch->Mv->dev);
}

// Phase 1b: f | y by Algorithm 1 (after phase 1a).  A mixed chain's M~ solves
// iterate on the current M~ view with its kept factor as preconditioner.
fifa_status chain_phase_sample(fifa_ctx* ctx, fifa_chain* ch) {
  ChainDev* c = ch->dev;
  return sample_enqueue(ctx, ch->H[0], ch->F[0], ch->FM, ch->y, 0.0, 0.0, ch->init.seed, ch->init.chain_id, &c->iter,
                        0, ch->f, ch->mean, &c->tau2, &c->refine_res, &c->pcg_iters, ch->Mv);
}

// Phase 1b's data part (after the prior part has run for this chain,
// sample_prior_enqueue or sample_prior_batched).
fifa_status chain_phase_sample_data(fifa_ctx* ctx, fifa_chain* ch) {
  ChainDev* c = ch->dev;
  return sample_data_enqueue(ctx, ch->H[0], ch->FM, ch->y, 0.0, 0.0, ch->f, ch->mean, &c->tau2, &c->refine_res,
                             &c->pcg_iters, ch->Mv);
}

// Phase 1: phases 1a and 1b.
fifa_status chain_phase_draw(fifa_ctx* ctx, fifa_chain* ch) {
  fifa_status st = chain_phase_factor_m(ctx, ch);
  return st == FIFA_OK ? chain_phase_sample(ctx, ch) : st;
}

// Phase 2: sigma2 | y, f.
fifa_status chain_phase_sigma2(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S) {
  if (launch_sumsq(ch->y, ch->f, ch->plan->n, S.red, &ch->dev->rss, ctx->stream) != cudaSuccess) return FIFA_ERR_CUDA;
  if (launch_chain_sigma2(ch->dev, ctx->stream) != cudaSuccess) return FIFA_ERR_CUDA;
  return FIFA_OK;
}

// Phase 3: tau2 | f, rho, then the Metropolis step on log rho (advances the
// chain's iteration counter).
// Phase 3a: q, tau2 | f, rho, the proposal rho' and the assembly of C~(rho').
fifa_status chain_phase_hyper_pre(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S) {
  if (cudaMemcpyAsync(ch->tmp, ch->f, sizeof(double) * ch->plan->n, cudaMemcpyDeviceToDevice, ctx->stream) !=
      cudaSuccess)
    return FIFA_ERR_CUDA;
  fifa_status st = sweep_enqueue(ctx, ch->F[0], 0, 1, ch->tmp, 1);
  if (st == FIFA_OK) st = chain_hyper_tau2_propose(ctx, ch, S);
  return st == FIFA_OK ? hmat_assemble_enqueue(ctx, ch->H[1]) : st;
}

// Phase 3a's middle: q = |W_C^-1 f|^2 from the swept copy of f in tmp, tau2 |
// f, rho, and the proposal rho' (written into the proposal's descriptor).
fifa_status chain_hyper_tau2_propose(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S) {
  fifa_status st = chain_hyper_tau2(ctx, ch, S);
  if (st != FIFA_OK) return st;
  if (launch_chain_propose(ch->dev, ch->H[1]->dev, ctx->stream) != cudaSuccess) return FIFA_ERR_CUDA;
  return FIFA_OK;
}

// q = |W_C^-1 f|^2 from the swept copy of f in tmp and tau2 | f, rho.
fifa_status chain_hyper_tau2(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S) {
  cudaStream_t s = ctx->stream;
  ChainDev* c = ch->dev;
  if (launch_sumsq(ch->tmp, nullptr, ch->plan->n, S.red, &c->q, s) != cudaSuccess) return FIFA_ERR_CUDA;
  if (launch_chain_tau2(c, s) != cudaSuccess) return FIFA_ERR_CUDA;
  return FIFA_OK;
}

// Phase 3c (after the factorization of C~(rho'), phase 3b): q' and the
// Metropolis step on log rho (advances the chain's iteration counter).
fifa_status chain_phase_hyper_post(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S) {
  if (cudaMemcpyAsync(ch->tmp, ch->f, sizeof(double) * ch->plan->n, cudaMemcpyDeviceToDevice, ctx->stream) !=
      cudaSuccess)
    return FIFA_ERR_CUDA;
  fifa_status st = sweep_enqueue(ctx, ch->F[1], 0, 1, ch->tmp, 1);
  return st == FIFA_OK ? chain_hyper_mh(ctx, ch, S) : st;
}

// Phase 3c's end: q' = |W_C'^-1 f|^2 from the swept copy of f in tmp and the
// Metropolis step.
fifa_status chain_hyper_mh(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S) {
  cudaStream_t s = ctx->stream;
  ChainDev* c = ch->dev;
  if (launch_sumsq(ch->tmp, nullptr, ch->plan->n, S.red, &c->q_prop, s) != cudaSuccess) return FIFA_ERR_CUDA;
  if (launch_chain_mh(c, ch->H[0]->dev, ch->H[1]->dev, ch->F[0]->dev, ch->F[1]->dev, ch->FM->dev, s) != cudaSuccess)
    return FIFA_ERR_CUDA;
  return FIFA_OK;
}

// Phase 3: tau2 | f, rho, then the Metropolis step on log rho (advances the
// chain's iteration counter).
fifa_status chain_phase_hyper(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S) {
  fifa_status st = chain_phase_hyper_pre(ctx, ch, S);
  if (st == FIFA_OK) st = fact_enqueue(ctx, ch->F[1], ch->H[1]->dev);
  if (st == FIFA_OK) st = chain_phase_hyper_post(ctx, ch, S);
  return st;
}

// One iteration with the proposal's assembly and factorization beside the draw
// (overlap_proposal).  rho' depends only on the state the previous iteration
// left, so C~(rho') can be built while f, sigma2 and tau2 are drawn.
//   ctx->stream: rho'; fork
//   draw stream (highest priority): grouped ACA of C~(rho'); draw, sigma2, q,
//     tau2; then, once the branch is done, the leaves and CTA-local levels of
//     W'^-1 f (independent CTAs, on the branch's idle scratch)
//   branch stream (lowest priority, own scratch): dense leaves, one-CTA and
//     one-warp ACA blocks; after the grouped ACA, the factorization's leaves
//     and ungrouped levels
//   ctx->stream: after the branch and the draw's last waiting launch, the
//     grouped levels of C~(rho') (beside the first part of W'^-1 f); join; the
//     rest of W'^-1 f, q' and the Metropolis step.
// Whenever a launch whose CTAs wait on each other runs, every other stream runs
// only kernels whose CTAs never wait, so the waiting launches keep their sizes
// and always become co-resident; the priorities let the draw's CTAs take SMs
// first as the branch's CTAs finish.  Every kernel, size and result is that of
// the serial order (W'^-1 f in two launches has the one-launch arithmetic).
static fifa_status chain_iteration_overlap(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S) {
  cudaStream_t ms = ctx->stream, ds = ch->draw_stream, ps = ch->prop_stream;
  CK(launch_chain_propose(ch->dev, ch->H[1]->dev, ms));
  CK(cudaEventRecord(ch->ev_fork, ms));
  CK(cudaStreamWaitEvent(ds, ch->ev_fork, 0));
  CK(cudaStreamWaitEvent(ps, ch->ev_fork, 0));
  // draw stream: grouped ACA, then the draw (ctx->stream points at it meanwhile)
  ctx->stream = ds;
  fifa_status st = hmat_assemble_grouped_enqueue(ctx, ch->H[1]);
  cudaError_t e = st == FIFA_OK ? cudaEventRecord(ch->ev_aca, ds) : cudaSuccess;
  if (st == FIFA_OK && e == cudaSuccess) {
    // branch: its own stream and scratch
    ctx->stream = ps;
    ctx->active_scratch = ch->scratch_prop;
    st = hmat_assemble_rest_enqueue(ctx, ch->H[1]);
    if (st == FIFA_OK) e = cudaStreamWaitEvent(ps, ch->ev_aca, 0);
    if (st == FIFA_OK && e == cudaSuccess) st = fact_enqueue_part(ctx, ch->F[1], ch->H[1]->dev, 0);
    ctx->stream = ds;
    ctx->active_scratch = ch->scratch;
  }
  const cudaError_t e_branch = cudaEventRecord(ch->ev_join_prop, ps);  // the branch ends here
  bool go = st == FIFA_OK && e == cudaSuccess && e_branch == cudaSuccess;
  if (go) st = chain_phase_draw(ctx, ch);
  if (go && st == FIFA_OK) st = chain_phase_sigma2(ctx, ch, S);
  if (go && st == FIFA_OK)
    st = cudaMemcpyAsync(ch->tmp, ch->f, sizeof(double) * ch->plan->n, cudaMemcpyDeviceToDevice, ds) == cudaSuccess
             ? sweep_enqueue(ctx, ch->F[0], 0, 1, ch->tmp, 1)
             : FIFA_ERR_CUDA;
  if (go && st == FIFA_OK) st = chain_hyper_tau2(ctx, ch, S);
  go = go && st == FIFA_OK;
  // the draw's last waiting launch is behind this event
  cudaError_t e_done = cudaEventRecord(ch->ev_draw_done, ds);
  const bool split = sweep_inverse_split_ok(ch->plan);
  if (go && split && e_done == cudaSuccess) {
    // first part of q' = |W'^-1 f|^2 beside the grouped levels: it reads only
    // the factor's levels the branch has finished
    e_done = cudaStreamWaitEvent(ds, ch->ev_join_prop, 0);
    if (e_done == cudaSuccess)
      e_done = cudaMemcpyAsync(ch->tmp, ch->f, sizeof(double) * ch->plan->n, cudaMemcpyDeviceToDevice, ds);
    if (e_done == cudaSuccess) {
      ctx->active_scratch = ch->scratch_prop;
      st = sweep_inverse_part_enqueue(ctx, ch->F[1], ch->tmp, 0);
      ctx->active_scratch = ch->scratch;
    }
  }
  const cudaError_t e_draw = cudaEventRecord(ch->ev_join_draw, ds);
  ctx->stream = ms;
  // the grouped levels wait for the branch and for the draw's last waiting launch
  const cudaError_t e3 = cudaStreamWaitEvent(ms, ch->ev_draw_done, 0);
  const cudaError_t e4 = cudaStreamWaitEvent(ms, ch->ev_join_prop, 0);
  if (go && st == FIFA_OK && e_done == cudaSuccess && e3 == cudaSuccess && e4 == cudaSuccess)
    st = fact_enqueue_part(ctx, ch->F[1], ch->H[1]->dev, 1);
  // join the draw stream whatever happened above (a capture must end joined)
  const cudaError_t e5 = cudaStreamWaitEvent(ms, ch->ev_join_draw, 0);
  if (st != FIFA_OK) return st;
  CK(e);
  CK(e_branch);
  CK(e_done);
  CK(e_draw);
  CK(e3);
  CK(e4);
  CK(e5);
  if (!split) return chain_phase_hyper_post(ctx, ch, S);
  st = sweep_inverse_part_enqueue(ctx, ch->F[1], ch->tmp, 1);
  return st == FIFA_OK ? chain_hyper_mh(ctx, ch, S) : st;
}

static fifa_status chain_iteration_enqueue(fifa_ctx* ctx, fifa_chain* ch) {
  ctx->active_scratch = ch->scratch;
  Scratch S = carve(ctx, ch->plan);
  fifa_status st;
  if (ch->overlap) {
    st = chain_iteration_overlap(ctx, ch, S);
  } else {
    st = chain_phase_draw(ctx, ch);
    if (st == FIFA_OK) st = chain_phase_sigma2(ctx, ch, S);
    if (st == FIFA_OK) st = chain_phase_hyper(ctx, ch, S);
  }
  ctx->active_scratch = nullptr;
  if (st == FIFA_ERR_CUDA && ctx->last_cuda == cudaSuccess) ctx->last_cuda = cudaGetLastError();
  return st;
}

size_t chain_bytes(const Plan* P, const fifa_opts& o) {
  auto r = [](size_t b) { return b == 0 ? (size_t)256 : (b + 255) & ~(size_t)255; };
  const int cap = o.rank_cap;
  return 5 * r(sizeof(double) * P->n) + r(sizeof(double) * CHAIN_TRACE_CAP * CHAIN_TRACE_FIELDS) +
         (o.overlap_proposal ? 2 : 1) * r(P->scratch_bytes) + r(sizeof(ChainDev)) + 2 * hmat_bytes(P, cap) +
         2 * fact_bytes(P, cap, 0) + r(sizeof(HmatDesc)) + fact_bytes(P, cap, o.prec == FIFA_MIXED ? 1 : 0);
}

static double kconst(int kind, double rho) { return kind == 0 ? 0.5 / (rho * rho) : sqrt(5.0) / rho; }

extern "C" fifa_status fifa_chain_create(fifa_ctx* ctx, const double* x_dev, const double* y_dev, int64_t n,
                                         const fifa_hyper* init, const fifa_prior* prior, uint64_t seed,
                                         uint64_t chain_id, fifa_chain** out) {
  if (!ctx || !x_dev || !y_dev || !init || !prior || !out || n < 2) return FIFA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(init->rho > 0.0) || !(init->tau2 > 0.0) || !(init->sigma2 > 0.0) || !(init->nugget >= 0.0)) return FIFA_ERR_INVALID_ARG;
  if (init->kernel != 0 && init->kernel != 1) return FIFA_ERR_INVALID_ARG;
  if (!(prior->logrho_sd > 0.0) || !(prior->prop_sd >= 0.0) || prior->a_tau2 + 0.5 * n < 1.0 ||
      prior->a_sigma2 + 0.5 * n < 1.0)
    return FIFA_ERR_INVALID_ARG;
  // validate inputs through the assembly check
  CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int), ctx->stream));
  CK(launch_check_sorted(x_dev, n, ctx->flags, ctx->stream));
  CK(cudaMemcpyAsync(ctx->host_flags, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->host_flags[0] & 2) return FIFA_ERR_INVALID_ARG;
  if (ctx->host_flags[0] & 1) return FIFA_ERR_UNSORTED;
  fifa_status st = FIFA_OK;
  Plan* P = get_plan(ctx, n, &st);
  if (!P) return st;
  fifa_chain* ch = new (std::nothrow) fifa_chain();
  if (!ch) return FIFA_ERR_OOM;
  ch->plan = P;
  auto fail = [&](fifa_status e) {
    fifa_destroy_chain(ctx, ch);
    return e;
  };
  ch->x = (double*)ctx->arena.alloc(sizeof(double) * n);
  ch->y = (double*)ctx->arena.alloc(sizeof(double) * n);
  ch->f = (double*)ctx->arena.alloc(sizeof(double) * n);
  ch->mean = (double*)ctx->arena.alloc(sizeof(double) * n);
  ch->tmp = (double*)ctx->arena.alloc(sizeof(double) * n);
  ch->trace = (double*)ctx->arena.alloc(sizeof(double) * CHAIN_TRACE_CAP * CHAIN_TRACE_FIELDS);
  ch->scratch = ctx->arena.alloc(P->scratch_bytes);
  ch->dev = (ChainDev*)ctx->arena.alloc(sizeof(ChainDev));
  if (!ch->x || !ch->y || !ch->f || !ch->mean || !ch->tmp || !ch->trace || !ch->scratch || !ch->dev)
    return fail(FIFA_ERR_OOM);
  if (ctx->opts.overlap_proposal) {
    ch->scratch_prop = ctx->arena.alloc(P->scratch_bytes);
    if (!ch->scratch_prop) return fail(FIFA_ERR_OOM);
    int dev = -1, least = 0, greatest = 0;
    CK(cudaGetDevice(&dev));
    if (dev != ctx->device) CK(cudaSetDevice(ctx->device));
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ch->draw_stream, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ch->prop_stream, cudaStreamNonBlocking, least);
    for (cudaEvent_t* ev : {&ch->ev_fork, &ch->ev_aca, &ch->ev_draw_done, &ch->ev_join_draw, &ch->ev_join_prop})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (dev != ctx->device) cudaSetDevice(dev);
    if (e != cudaSuccess) {
      ctx->last_cuda = e;
      return fail(FIFA_ERR_CUDA);
    }
    ch->overlap = true;
  }
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(ch->x, x_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(ch->y, y_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(ch->f, 0, sizeof(double) * n, s));
  CK(cudaMemsetAsync(ch->mean, 0, sizeof(double) * n, s));
  for (int k = 0; k < 2; ++k) {
    st = hmat_alloc(ctx, P, init->kernel, &ch->H[k]);
    if (st != FIFA_OK) return fail(st);
    HmatDesc& d = ch->H[k]->host;
    d.x = ch->x;
    d.rho = init->rho;
    d.kc = kconst(init->kernel, init->rho);
    d.nugget = init->nugget;
    CK(cudaMemcpyAsync(ch->H[k]->dev, &d, sizeof(HmatDesc), cudaMemcpyHostToDevice, s));
    st = fact_alloc(ctx, P, 0, &ch->F[k]);
    if (st != FIFA_OK) return fail(st);
    ch->F[k]->src = ch->H[k];
  }
  ch->Mv = new (std::nothrow) fifa_hmat();
  if (!ch->Mv) return fail(FIFA_ERR_OOM);
  ch->Mv->plan = P;
  ch->Mv->host = ch->H[0]->host;
  ch->Mv->host.shift = 1.0;
  ch->Mv->owns = false;
  ch->Mv->dev = (HmatDesc*)ctx->arena.alloc(sizeof(HmatDesc));
  if (!ch->Mv->dev) return fail(FIFA_ERR_OOM);
  st = fact_alloc(ctx, P, ctx->opts.prec == FIFA_MIXED ? 1 : 0, &ch->FM);
  if (st != FIFA_OK) return fail(st);
  ch->FM->src = ch->Mv;
  // the M~ factorization kernels read the chain's keep flag (set every iteration)
  if (ctx->opts.prec == FIFA_MIXED && (st = fact_set_skip(ctx, ch->FM, &ch->dev->fm_skip)) != FIFA_OK) return fail(st);
  ChainDev& c = ch->init;
  memset(&c, 0, sizeof(c));
  c.tau2 = init->tau2;
  c.sigma2 = init->sigma2;
  c.eta = log(init->rho);
  c.rho = init->rho;
  c.a_tau2 = prior->a_tau2;
  c.b_tau2 = prior->b_tau2;
  c.a_sigma2 = prior->a_sigma2;
  c.b_sigma2 = prior->b_sigma2;
  c.logrho_mu = prior->logrho_mu;
  c.logrho_sd = prior->logrho_sd;
  c.prop_sd = prior->prop_sd;
  c.seed = seed;
  c.chain_id = chain_id;
  c.iter = 0;
  c.n = n;
  c.kind = init->kernel;
  c.trace_cap = CHAIN_TRACE_CAP;
  c.trace = ch->trace;
  c.mixed = ctx->opts.prec == FIFA_MIXED ? 1 : 0;
  c.fm_skip = 0;
  c.s_ref = 0.0;
  CK(cudaMemcpyAsync(ch->dev, &c, sizeof(ChainDev), cudaMemcpyHostToDevice, s));
  // C~(rho_0) and its factor
  ctx->active_scratch = ch->scratch;
  st = hmat_assemble_enqueue(ctx, ch->H[0]);
  if (st == FIFA_OK) st = fact_enqueue(ctx, ch->F[0], ch->H[0]->dev);
  ctx->active_scratch = nullptr;
  if (st != FIFA_OK) return fail(st);
  int fs = 0;
  CK(cudaMemcpyAsync(ctx->host_flags, ch->F[0]->host.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  fs = ctx->host_flags[0];
  if (fs & FIFA_DEV_NOT_SPD) return fail(FIFA_ERR_NOT_SPD);
  if (fs & FIFA_DEV_TIMEOUT) return fail(FIFA_ERR_TIMEOUT);
  *out = ch;
  return FIFA_OK;
}

static fifa_status chain_build_graph(fifa_ctx* ctx, fifa_chain* ch) {
  if (ch->exec || ch->graph_failed) return FIFA_OK;
  cudaStream_t s = ctx->stream;
  if (s == nullptr) {  // the legacy default stream cannot be captured
    ch->graph_failed = true;
    return FIFA_OK;
  }
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    ch->graph_failed = true;
    return FIFA_OK;
  }
  ctx->capturing = true;
  fifa_status st = chain_iteration_enqueue(ctx, ch);
  ctx->capturing = false;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st != FIFA_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    ch->graph_failed = true;
    return FIFA_OK;
  }
  // per-node priorities: the overlapped iteration's draw stream outranks its branch
  if (cudaGraphInstantiateWithFlags(&ch->exec, g, ch->overlap ? cudaGraphInstantiateFlagUseNodePriority : 0) !=
      cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    ch->exec = nullptr;
    ch->graph_failed = true;
    return FIFA_OK;
  }
  ch->graph = g;
  return FIFA_OK;
}

extern "C" fifa_status fifa_gibbs_step(fifa_ctx* ctx, fifa_chain* ch, int iters, double* trace_host) {
  if (!ctx || !ch || iters < 0) return FIFA_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  fifa_status st = chain_build_graph(ctx, ch);
  if (st != FIFA_OK) return st;
  int done = 0;
  while (done < iters) {
    const int chunk = std::min(iters - done, CHAIN_TRACE_CAP);
    for (int k = 0; k < chunk; ++k) {
      if (ch->exec) {
        CK(cudaGraphLaunch(ch->exec, s));
      } else {
        st = chain_iteration_enqueue(ctx, ch);
        if (st != FIFA_OK) return st;
      }
    }
    if (trace_host) {
      const uint64_t first = ch->iter_host % CHAIN_TRACE_CAP;
      const uint64_t n1 = std::min<uint64_t>(chunk, CHAIN_TRACE_CAP - first);
      CK(cudaMemcpyAsync(trace_host + (size_t)done * CHAIN_TRACE_FIELDS, ch->trace + first * CHAIN_TRACE_FIELDS,
                         sizeof(double) * n1 * CHAIN_TRACE_FIELDS, cudaMemcpyDeviceToHost, s));
      if (n1 < (uint64_t)chunk)
        CK(cudaMemcpyAsync(trace_host + (size_t)(done + n1) * CHAIN_TRACE_FIELDS, ch->trace,
                           sizeof(double) * (chunk - n1) * CHAIN_TRACE_FIELDS, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    ch->iter_host += chunk;
    done += chunk;
  }
  CK(cudaMemcpyAsync(ctx->host_flags, &ch->dev->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int cs = ctx->host_flags[0];
  if (cs & FIFA_DEV_TIMEOUT) return FIFA_ERR_TIMEOUT;
  if (cs & FIFA_DEV_NOT_SPD) return FIFA_ERR_NOT_SPD;
  return FIFA_OK;
}

fifa_status chain_run_collect(fifa_ctx* ctx, fifa_chain* ch, int iters, int burn, int ndraws, double* mean_acc,
                              double* draws) {
  if (iters < 1 || burn < 0 || burn >= iters || ndraws < 0 || ndraws > iters - burn) return FIFA_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  const int64_t n = ch->plan->n;
  fifa_status st = chain_build_graph(ctx, ch);
  if (st != FIFA_OK) return st;
  CK(cudaMemsetAsync(mean_acc, 0, sizeof(double) * n, s));
  const int kept = iters - burn;
  int next_draw = 0;
  for (int t = 0; t < iters; ++t) {
    if (ch->exec) {
      CK(cudaGraphLaunch(ch->exec, s));
    } else {
      st = chain_iteration_enqueue(ctx, ch);
      if (st != FIFA_OK) return st;
    }
    if (t < burn) continue;
    CK(launch_axpy(1.0, ch->mean, mean_acc, n, s));
    // draw j is taken at iteration burn + floor((j + 1) kept / ndraws) - 1
    while (next_draw < ndraws && t == burn + (int)(((int64_t)(next_draw + 1) * kept) / ndraws) - 1) {
      CK(cudaMemcpyAsync(draws + (size_t)next_draw * n, ch->f, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      ++next_draw;
    }
  }
  ch->iter_host += iters;
  CK(cudaMemcpyAsync(ctx->host_flags, &ch->dev->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int cs = ctx->host_flags[0];
  if (cs & FIFA_DEV_TIMEOUT) return FIFA_ERR_TIMEOUT;
  if (cs & FIFA_DEV_NOT_SPD) return FIFA_ERR_NOT_SPD;
  return FIFA_OK;
}

fifa_status chain_state(fifa_ctx* ctx, const fifa_chain* ch, ChainDev* out) {
  CK(cudaMemcpyAsync(out, ch->dev, sizeof(ChainDev), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FIFA_OK;
}

extern "C" fifa_status fifa_chain_set_y(fifa_ctx* ctx, fifa_chain* ch, const double* y) {
  if (!ctx || !ch || !y || ctx->capturing) return FIFA_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(ch->y, y, sizeof(double) * ch->plan->n, cudaMemcpyDefault, ctx->stream));
  return FIFA_OK;
}

extern "C" fifa_status fifa_chain_get(fifa_ctx* ctx, const fifa_chain* ch, double* f_dev, double* mean_dev,
                                      fifa_hyper* h_host) {
  if (!ctx || !ch) return FIFA_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  const int64_t n = ch->plan->n;
  if (f_dev) CK(cudaMemcpyAsync(f_dev, ch->f, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  if (mean_dev) CK(cudaMemcpyAsync(mean_dev, ch->mean, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  ChainDev c;
  CK(cudaMemcpyAsync(&c, ch->dev, sizeof(ChainDev), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h_host) {
    h_host->kernel = c.kind;
    h_host->tau2 = c.tau2;
    h_host->rho = c.rho;
    h_host->sigma2 = c.sigma2;
    h_host->nugget = ch->H[0]->host.nugget;
  }
  return FIFA_OK;
}

extern "C" void fifa_destroy_chain(fifa_ctx* ctx, fifa_chain* ch) {
  if (!ctx || !ch) return;
  cudaStreamSynchronize(ctx->stream);
  if (ch->exec) cudaGraphExecDestroy(ch->exec);
  if (ch->graph) cudaGraphDestroy(ch->graph);
  for (int k = 0; k < 2; ++k) {
    if (ch->F[k]) fifa_destroy_fact(ctx, ch->F[k]);
    if (ch->H[k]) fifa_destroy_hmat(ctx, ch->H[k]);
  }
  if (ch->FM) fifa_destroy_fact(ctx, ch->FM);
  if (ch->Mv) fifa_destroy_hmat(ctx, ch->Mv);
  ctx->arena.release(ch->x);
  ctx->arena.release(ch->y);
  ctx->arena.release(ch->f);
  ctx->arena.release(ch->mean);
  ctx->arena.release(ch->tmp);
  ctx->arena.release(ch->trace);
  ctx->arena.release(ch->scratch);
  for (cudaStream_t t : {ch->draw_stream, ch->prop_stream})
    if (t) {
      cudaStreamSynchronize(t);
      cudaStreamDestroy(t);
    }
  for (cudaEvent_t ev : {ch->ev_fork, ch->ev_aca, ch->ev_draw_done, ch->ev_join_draw, ch->ev_join_prop})
    if (ev) cudaEventDestroy(ev);
  if (ch->scratch_prop) ctx->arena.release(ch->scratch_prop);
  ctx->arena.release(ch->dev);
  delete ch;
}

extern "C" fifa_status fifa_chain_kernel_nodes(const fifa_chain* ch, int* out_host) {
  if (!ch || !out_host) return FIFA_ERR_INVALID_ARG;
  *out_host = -1;
  if (!ch->graph) return FIFA_OK;
  size_t count = 0;
  if (cudaGraphGetNodes(ch->graph, nullptr, &count) != cudaSuccess) return FIFA_ERR_CUDA;
  std::vector<cudaGraphNode_t> nodes(count);
  if (count && cudaGraphGetNodes(ch->graph, nodes.data(), &count) != cudaSuccess) return FIFA_ERR_CUDA;
  int kernels = 0;
  for (size_t i = 0; i < count; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
  }
  *out_host = kernels;
  return FIFA_OK;
}
