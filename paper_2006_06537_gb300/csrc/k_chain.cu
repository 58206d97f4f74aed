// Scalar Gibbs updates on the device (one thread), so a whole iteration runs
// without returning to the host (Sec. 4.1, Eqs. posterior_gibs2-4):
//   sigma2 ~ IG(a_s + n/2, b_s + ||y - f||^2 / 2)
//   tau2   ~ IG(a_t + n/2, b_t + q / 2),   q = ||W_C^-1 f||^2
//   eta'   = eta + prop_sd z,  rho' = exp(eta')  (random-walk Metropolis on log rho)
//   log alpha = -(logdet C~' - logdet C~)/2 - (q' - q)/(2 tau2) + log p(eta') - log p(eta)
// On acceptance the current and proposed H-matrix / factor descriptors are
// swapped in device memory, so the captured graph keeps reading "current"
// from the same address.
#include <algorithm>

#include "fifa_chain.h"
#include "fifa_common.cuh"
#include "fifa_rng.cuh"

// M~ = s C~ + I with s = tau2 / sigma2, and whether its factor is refreshed
// this iteration (always for an FP64 chain; see CHAIN_REFRESH_* for mixed).
__global__ void k_chain_make_view(const HmatDesc* __restrict__ Hc, HmatDesc* __restrict__ Mv, ChainDev* __restrict__ c) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    HmatDesc d = *Hc;
    const double sv = c->tau2 / c->sigma2;
    d.scale = sv;
    d.shift = 1.0;
    *Mv = d;
    int refresh = 1;
    if (c->mixed)
      refresh = c->force_refresh || !(c->s_ref > 0.0) || !(fabs(sv / c->s_ref - 1.0) <= CHAIN_REFRESH_REL) ||
                c->pcg_iters > CHAIN_REFRESH_ITERS;
    if (refresh) {
      c->s_ref = sv;
      c->force_refresh = 0;
      c->n_refresh += 1;
    }
    c->fm_skip = refresh ? 0 : 1;
    c->refreshed = refresh;
  }
}

__global__ void k_chain_sigma2(ChainDev* __restrict__ c) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double shape = c->a_sigma2 + 0.5 * (double)c->n;
  const double scale = c->b_sigma2 + 0.5 * c->rss;
  const double g = gamma_mt(shape, c->seed, 2u, c->iter, c->chain_id);
  c->sigma2 = scale / g;
}

__global__ void k_chain_tau2(ChainDev* __restrict__ c) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double shape = c->a_tau2 + 0.5 * (double)c->n;
  const double scale = c->b_tau2 + 0.5 * c->q;
  const double g = gamma_mt(shape, c->seed, 3u, c->iter, c->chain_id);
  c->tau2 = scale / g;
}

__global__ void k_chain_propose(ChainDev* __restrict__ c, HmatDesc* __restrict__ Hp) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double z = philox_normal(c->seed, 0u, 4u, c->iter, c->chain_id);
  const double eta = c->eta + c->prop_sd * z;
  const double rho = exp(eta);
  c->eta_prop = eta;
  c->rho_prop = rho;
  Hp->rho = rho;
  Hp->kc = (c->kind == 0) ? __ddiv_rn(0.5, __dmul_rn(rho, rho)) : __ddiv_rn(sqrt(5.0), rho);
}

__device__ __forceinline__ double log_prior_eta(const ChainDev* c, double eta) {
  const double z = (eta - c->logrho_mu) / c->logrho_sd;
  return -0.5 * z * z;
}

template <typename D>
__device__ __forceinline__ void swap_desc(D* a, D* b) {
  D t = *a;
  *a = *b;
  *b = t;
}

__global__ void k_chain_mh(ChainDev* __restrict__ c, HmatDesc* __restrict__ Hc, HmatDesc* __restrict__ Hp,
                           FactDesc* __restrict__ Fc, FactDesc* __restrict__ Fp, const FactDesc* __restrict__ Fm) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double ld_cur = *Fc->logdet, ld_prop = *Fp->logdet;
  const int pst = *Fp->status | (*Hp->status & ~FIFA_DEV_RANK_CAP);
  double la = -0.5 * (ld_prop - ld_cur) - (c->q_prop - c->q) / (2.0 * c->tau2) + log_prior_eta(c, c->eta_prop) -
              log_prior_eta(c, c->eta);
  if (pst != 0 || !isfinite(la)) la = -INFINITY;
  const double u = philox_uniform(c->seed, 0u, 5u, c->iter, c->chain_id);
  const int acc = (log(u) < la) ? 1 : 0;
  c->status |= *Fm->status | (*Fc->status & ~FIFA_DEV_RANK_CAP);
  c->accept = acc;
  c->n_accept += (uint64_t)acc;
  c->log_alpha = la;
  if (acc) {
    if (c->eta_prop != c->eta) c->force_refresh = 1;  // C~ changed: the kept M~ factor no longer fits
    swap_desc(Hc, Hp);
    swap_desc(Fc, Fp);
    c->eta = c->eta_prop;
    c->rho = c->rho_prop;
  }
  if (c->trace && c->trace_cap > 0) {
    double* row = c->trace + (size_t)(c->iter % (uint64_t)c->trace_cap) * CHAIN_TRACE_FIELDS;
    row[0] = (double)c->iter;
    row[1] = c->sigma2;
    row[2] = c->tau2;
    row[3] = c->rho;
    row[4] = (double)acc;
    row[5] = la;
    row[6] = acc ? ld_prop : ld_cur;
    row[7] = c->q;
    row[8] = c->rss;
    row[9] = c->refine_res;
    row[10] = (double)c->status;
    row[11] = (double)c->refreshed;
    row[12] = (double)c->pcg_iters;
  }
  c->iter += 1;
}


cudaError_t launch_chain_make_view(const HmatDesc* Hc, HmatDesc* Mv, ChainDev* c, cudaStream_t st) {
  k_chain_make_view<<<1, 32, 0, st>>>(Hc, Mv, c);
  return cudaGetLastError();
}
cudaError_t launch_chain_sigma2(ChainDev* c, cudaStream_t st) {
  k_chain_sigma2<<<1, 32, 0, st>>>(c);
  return cudaGetLastError();
}
cudaError_t launch_chain_tau2(ChainDev* c, cudaStream_t st) {
  k_chain_tau2<<<1, 32, 0, st>>>(c);
  return cudaGetLastError();
}
cudaError_t launch_chain_propose(ChainDev* c, HmatDesc* Hp, cudaStream_t st) {
  k_chain_propose<<<1, 32, 0, st>>>(c, Hp);
  return cudaGetLastError();
}
cudaError_t launch_chain_mh(ChainDev* c, HmatDesc* Hc, HmatDesc* Hp, FactDesc* Fc, FactDesc* Fp, const FactDesc* Fm,
                            cudaStream_t st) {
  k_chain_mh<<<1, 32, 0, st>>>(c, Hc, Hp, Fc, Fp, Fm);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Additive model of d one-dimensional blocks (Sec. 4.2): F is n x d in the
// original point order, column k at F + k n; perm_k sorts x_k (stable).
// ---------------------------------------------------------------------------

// Partial residual of block k in x_k-sorted order:
//   out[i] = y[p] - F[p, j0] - F[p, j1] - ...  (j != k, ascending), p = perm_k[i]
__global__ void k_add_gather(const double* __restrict__ y, const double* __restrict__ F,
                             const int64_t* __restrict__ perm, int64_t n, int d, int k, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = perm[i];
    double r = y[p];
    for (int j = 0; j < d; ++j)
      if (j != k) r = __dsub_rn(r, F[(int64_t)j * n + p]);
    out[i] = r;
  }
}

// F[perm_k[i], k] = f_sorted[i]
__global__ void k_add_scatter(const double* __restrict__ fs, const int64_t* __restrict__ perm, int64_t n,
                              double* __restrict__ Fk) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Fk[perm[i]] = fs[i];
}

// Full residual minus the last block: out = y - F[:, 0] - ... - F[:, d-2], so
// that ||out - F[:, d-1]||^2 is the model's residual sum of squares.
__global__ void k_add_residual(const double* __restrict__ y, const double* __restrict__ F, int64_t n, int d,
                               double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double r = y[i];
    for (int j = 0; j + 1 < d; ++j) r = __dsub_rn(r, F[(int64_t)j * n + i]);
    out[i] = r;
  }
}

// Shared sigma2 | y, F_1..F_d, drawn from the stream of g (chain id d), copied
// into every block's state; appends (iteration, sigma2, rss) to g's trace.
__global__ void k_add_sigma2(ChainDev* __restrict__ g, ChainDev* const* __restrict__ blocks, int d) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double shape = g->a_sigma2 + 0.5 * (double)g->n;
  const double scale = g->b_sigma2 + 0.5 * g->rss;
  const double gm = gamma_mt(shape, g->seed, 2u, g->iter, g->chain_id);
  const double s2 = scale / gm;
  g->sigma2 = s2;
  for (int k = 0; k < d; ++k) blocks[k]->sigma2 = s2;
  if (g->trace && g->trace_cap > 0) {
    double* row = g->trace + (size_t)(g->iter % (uint64_t)g->trace_cap) * 3;
    row[0] = (double)g->iter;
    row[1] = s2;
    row[2] = g->rss;
  }
  g->iter += 1;
}

static inline int add_grid(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 8); }

cudaError_t launch_add_gather(const double* y, const double* F, const int64_t* perm, int64_t n, int d, int k,
                              double* out, cudaStream_t st) {
  k_add_gather<<<add_grid(n), 256, 0, st>>>(y, F, perm, n, d, k, out);
  return cudaGetLastError();
}
cudaError_t launch_add_scatter(const double* fs, const int64_t* perm, int64_t n, double* Fk, cudaStream_t st) {
  k_add_scatter<<<add_grid(n), 256, 0, st>>>(fs, perm, n, Fk);
  return cudaGetLastError();
}
cudaError_t launch_add_residual(const double* y, const double* F, int64_t n, int d, double* out, cudaStream_t st) {
  k_add_residual<<<add_grid(n), 256, 0, st>>>(y, F, n, d, out);
  return cudaGetLastError();
}
cudaError_t launch_add_sigma2(ChainDev* g, ChainDev* const* blocks, int d, cudaStream_t st) {
  k_add_sigma2<<<1, 32, 0, st>>>(g, blocks, d);
  return cudaGetLastError();
}
