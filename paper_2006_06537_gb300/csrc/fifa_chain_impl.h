// Host-side Gibbs chain object and its iteration phases (internal; shared by
// the single chain and the additive block model).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fifa.h"
#include "fifa_api_internal.h"
#include "fifa_chain.h"

#define CHAIN_TRACE_CAP 1024

struct fifa_chain {
  Plan* plan = nullptr;
  fifa_hmat* H[2] = {nullptr, nullptr};  // slot 0: current C~, slot 1: proposal (device descriptors swap)
  fifa_fact* F[2] = {nullptr, nullptr};
  fifa_fact* FM = nullptr;
  fifa_hmat* Mv = nullptr;  // view descriptor refreshed every iteration
  double *x = nullptr, *y = nullptr, *f = nullptr, *mean = nullptr, *tmp = nullptr, *trace = nullptr;
  void* scratch = nullptr;
  // overlap_proposal: the draw's stream (highest priority), the proposal
  // branch's stream (lowest) and scratch, fork / hand-over / join events
  bool overlap = false;
  void* scratch_prop = nullptr;
  cudaStream_t draw_stream = nullptr, prop_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_aca = nullptr, ev_draw_done = nullptr, ev_join_draw = nullptr,
              ev_join_prop = nullptr;
  ChainDev* dev = nullptr;
  ChainDev init{};
  uint64_t iter_host = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_failed = false;
};

// The three phases of one iteration, enqueued on ctx->stream with
// ctx->active_scratch = chain->scratch (S carved from it):
//   draw   M~ view, its factor, f | y by Algorithm 1 (data chain->y)
//   sigma2 ||y - f||^2 and sigma2 | y, f
//   hyper  q, tau2 | f, proposal C~(rho'), its factor, q', Metropolis step;
//          advances the chain's iteration counter
fifa_status chain_phase_draw(fifa_ctx* ctx, fifa_chain* ch);
fifa_status chain_phase_factor_m(fifa_ctx* ctx, fifa_chain* ch);  // first half of draw: M~ and its factor
fifa_status chain_phase_sample(fifa_ctx* ctx, fifa_chain* ch);    // second half: Algorithm 1
fifa_status chain_phase_sigma2(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S);
fifa_status chain_phase_hyper(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S);
// hyper in three parts: pre (q, tau2, proposal, assembly of C~(rho')), the
// factorization of C~(rho') into F[1], post (q' and the Metropolis step)
fifa_status chain_phase_hyper_pre(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S);
fifa_status chain_phase_hyper_post(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S);
// The parts of phases 3a / 3c after their sweep of the copy of f in tmp (the
// additive model runs the blocks' sweeps in one batched launch).
fifa_status chain_hyper_tau2_propose(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S);
fifa_status chain_hyper_tau2(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S);  // without the proposal
fifa_status chain_hyper_mh(fifa_ctx* ctx, fifa_chain* ch, const Scratch& S);
// Phase 1b without its prior part (run for several blocks at once by the additive model).
fifa_status chain_phase_sample_data(fifa_ctx* ctx, fifa_chain* ch);

// Serving helpers.  chain_run_collect runs `iters` iterations (graph replay)
// and gathers on the device: mean_acc = sum of the conditional means
// tau2 C~ r over iterations [burn, iters); draws (ndraws x n) = f at
// iterations burn + floor((j + 1)(iters - burn) / ndraws) - 1.  Synchronizes
// once at the end and returns the chain's device status.
fifa_status chain_run_collect(fifa_ctx* ctx, fifa_chain* ch, int iters, int burn, int ndraws, double* mean_acc,
                              double* draws);
fifa_status chain_state(fifa_ctx* ctx, const fifa_chain* ch, ChainDev* out);
