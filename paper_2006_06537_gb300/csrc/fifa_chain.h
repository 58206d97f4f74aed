// Device-resident Gibbs chain state (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fifa_common.cuh"

#define CHAIN_TRACE_FIELDS 13

// Mixed precision: the FP64 factor of M~ is kept from one iteration to the
// next and refreshed (refactored) only when the Metropolis step accepted a new
// length-scale (C~ changed), when s = tau2 / sigma2 moved by more than
// CHAIN_REFRESH_REL from the s it was factored at, or when the last solve took
// more than CHAIN_REFRESH_ITERS conjugate-gradient iterations; in between, the
// conjugate gradients on the current M~ absorb the change of s.
#define CHAIN_REFRESH_REL 0.05
#define CHAIN_REFRESH_ITERS 6

struct ChainDev {
  double tau2, sigma2;  // adjacent: read as scal[0], scal[1] by the Algorithm 1 kernels
  double eta, rho, eta_prop, rho_prop;
  double rss, q, q_prop, log_alpha, refine_res;
  double a_tau2, b_tau2, a_sigma2, b_sigma2, logrho_mu, logrho_sd, prop_sd;
  double red_num, red_den;
  uint64_t seed, chain_id, iter;
  int64_t n;
  int kind, accept, status, trace_cap;
  double* trace;
  uint64_t n_accept;  // accepted Metropolis proposals since creation
  // M~ factor management (mixed precision; an FP64 chain refactors every iteration)
  int mixed;          // 1: keep the M~ factor while it serves as a preconditioner
  int fm_skip;        // read by the factorization kernels of M~: 1 = keep the factor
  int force_refresh;  // set by an accepted proposal (C~ changed)
  int refreshed;      // this iteration refactored M~
  int pcg_iters;      // conjugate-gradient iterations of the last M~ solve
  double s_ref;       // s of the M~ the kept factor belongs to (0: none yet)
  uint64_t n_refresh; // M~ factorizations since creation
};

cudaError_t launch_chain_make_view(const HmatDesc* Hc, HmatDesc* Mv, ChainDev* c, cudaStream_t st);
cudaError_t launch_chain_sigma2(ChainDev* c, cudaStream_t st);
cudaError_t launch_chain_tau2(ChainDev* c, cudaStream_t st);
cudaError_t launch_chain_propose(ChainDev* c, HmatDesc* Hp, cudaStream_t st);
cudaError_t launch_chain_mh(ChainDev* c, HmatDesc* Hc, HmatDesc* Hp, FactDesc* Fc, FactDesc* Fp, const FactDesc* Fm,
                            cudaStream_t st);

cudaError_t launch_add_gather(const double* y, const double* F, const int64_t* perm, int64_t n, int d, int k,
                              double* out, cudaStream_t st);
cudaError_t launch_add_scatter(const double* fs, const int64_t* perm, int64_t n, double* Fk, cudaStream_t st);
cudaError_t launch_add_residual(const double* y, const double* F, int64_t n, int d, double* out, cudaStream_t st);
cudaError_t launch_add_sigma2(ChainDev* g, ChainDev* const* blocks, int d, cudaStream_t st);
