// Mixed-precision solves with M~ (the precision pattern of the sampler):
//
//  k_demote    FP32 copy of an FP64 factor W of M~: the leaf factors (both
//              triangles), their reciprocal pivots and the used columns of
//              every level's orthonormal bases, each rounded to nearest.  The
//              node matrices Zf, Zi stay FP64 and are shared with the FP64
//              factor.  W32 W32^T is then a symmetric positive definite
//              preconditioner whose relative distance to the factored matrix is
//              about sqrt(kappa) u32 (W is only as ill-conditioned as the square
//              root of M~), applied by the FP32 sweeps of k_apply.cu.
//  k_pcg_*     conjugate gradients preconditioned by W32 W32^T on the FP64
//              operator M~ (the current one; the factor may belong to an
//              earlier M~ of the chain), for up to two right-hand sides, with
//              every scalar on the device.  Each reduction is a fixed grid of
//              block partial sums (PCG_NB per right-hand side) that the
//              consuming kernel adds in a fixed order, so results are bitwise
//              reproducible; converged systems stop updating, and once every
//              system has converged the products and preconditioner launches of
//              the remaining captured iterations return at once.
#include <cuda_runtime.h>
#include <math.h>

#include "fifa_common.cuh"
#include "fifa_mixed.h"

__global__ void __launch_bounds__(256) k_demote(const FactDesc* __restrict__ F64, const FactDesc* __restrict__ F32) {
  F64 += blockIdx.y;  // problem of a batched launch
  F32 += blockIdx.y;
  if (F64->skip && *F64->skip) return;  // the FP64 factor was kept, so is its copy
  const int L = F64->L, Bm = F64->Bm, cap = F64->cap, nleaf = F64->nleaf;
  const int64_t n = F64->n;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
  const double* l64 = (const double*)F64->Lleaf;
  float* l32 = (float*)F32->Lleaf;
  for (int64_t i = tid; i < (int64_t)nleaf * Bm * Bm; i += nt) l32[i] = (float)l64[i];
  const double* d64 = (const double*)F64->Ldinv;
  float* d32 = (float*)F32->Ldinv;
  for (int64_t i = tid; i < (int64_t)nleaf * Bm; i += nt) d32[i] = (float)d64[i];
  // bases: row p lies in one node per level; descend the tree from the root
  const double* q64 = (const double*)F64->Q;
  float* q32 = (float*)F32->Q;
  const int* bnd = F64->bnd;
  for (int64_t p = tid; p < n; p += nt) {
    int node = 0;
    for (int l = 0; l < L; ++l) {
      int s, h, e;
      node_range(bnd, l, node, s, h, e);
      const int r = F64->rank[node_id(l, node)];
      for (int k = 0; k < r; ++k) {
        const size_t at = ((size_t)l * cap + k) * n + p;
        q32[at] = (float)q64[at];
      }
      node = 2 * node + (p >= h ? 1 : 0);
    }
  }
}

cudaError_t launch_demote(const FactDesc* F64, const FactDesc* F32, int64_t n, cudaStream_t st, int nprob) {
  const int64_t want = (n + 255) / 256;
  const int grid = (int)(want < 4096 ? (want < 1 ? 1 : want) : 4096);
  k_demote<<<dim3(grid, nprob), 256, 0, st>>>(F64, F32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conjugate gradients.  State per parity slot q and right-hand side j at
// st[(2 q + j) * PCG_SLOT + k]: k = 0 rho = r^T z, 1 b^T b, 2 done (1: converged
// or stopped), 3 r^T r.  act[q] = 1 while some system of slot q iterates;
// iteration t reads slot t & 1 and writes slot (t + 1) & 1, so no kernel reads
// what it writes.  Partial sums: part + PCG_PART(which, j) for which in
// {0: r^T r, 1: b^T b / p^T q, 2: r^T z}.
// ---------------------------------------------------------------------------
#define PCG_PART(w, j) (((w) * 2 + (j)) * PCG_NB)

__device__ __forceinline__ double pcg_sum(const double* __restrict__ part, int w, int j) {
  // every block adds the same partials in the same order
  double v = 0.0;
  for (int b = 0; b < PCG_NB; ++b) v += __ldcg(part + PCG_PART(w, j) + b);
  return v;
}

// r = b - r (r holds M~ x on entry), z = r; partials of r^T r and b^T b.
__global__ void __launch_bounds__(256) k_pcg_residual0(const double* __restrict__ b, double* __restrict__ r,
                                                      double* __restrict__ z, int64_t n, double* __restrict__ part) {
  const int j = blockIdx.y;
  const double* bj = b + (size_t)j * n;
  double* rj = r + (size_t)j * n;
  double* zj = z + (size_t)j * n;
  double rr = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bv = bj[i], rv = bv - rj[i];
    rj[i] = rv;
    zj[i] = rv;
    rr += rv * rv;
    bb += bv * bv;
  }
  __shared__ double red[40];
  rr = block_sum(rr, red);
  bb = block_sum(bb, red);
  if (threadIdx.x == 0) {
    __stcg(part + PCG_PART(0, j) + blockIdx.x, rr);
    __stcg(part + PCG_PART(1, j) + blockIdx.x, bb);
  }
}

// p = z; partials of r^T z.
__global__ void __launch_bounds__(256) k_pcg_start(const double* __restrict__ r, const double* __restrict__ z,
                                                  double* __restrict__ p, int64_t n, double* __restrict__ part) {
  const int j = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double zv = z[(size_t)j * n + i];
    p[(size_t)j * n + i] = zv;
    acc += r[(size_t)j * n + i] * zv;
  }
  __shared__ double red[40];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) __stcg(part + PCG_PART(2, j) + blockIdx.x, acc);
}

// Slot 0 from the first residual (one block).
__global__ void k_pcg_init(double* __restrict__ st, int* __restrict__ act, int* __restrict__ iters,
                           const double* __restrict__ part, int nrhs, double tol2) {
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int j = 0; j < PCG_RHS_MAX; ++j) {
    double* s = st + j * PCG_SLOT;
    if (j >= nrhs) {
      s[0] = 0.0; s[1] = 0.0; s[2] = 1.0; s[3] = 0.0;
      continue;
    }
    const double rr = pcg_sum(part, 0, j), bb = pcg_sum(part, 1, j), rz = pcg_sum(part, 2, j);
    const bool done = !(rr > tol2 * bb) || !(rz > 0.0) || !isfinite(rz);
    s[0] = rz;
    s[1] = bb;
    s[2] = done ? 1.0 : 0.0;
    s[3] = rr;
    any |= done ? 0 : 1;
  }
  act[0] = any;
  *iters = 0;
}

// Partials of p^T q (after q = M~ p).
__global__ void __launch_bounds__(256) k_pcg_pq(const double* __restrict__ p, const double* __restrict__ q, int64_t n,
                                               double* __restrict__ part, const int* __restrict__ active) {
  if (*active == 0) return;
  const int j = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += p[(size_t)j * n + i] * q[(size_t)j * n + i];
  __shared__ double red[40];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) __stcg(part + PCG_PART(1, j) + blockIdx.x, acc);
}

__device__ __forceinline__ double pcg_alpha(const double* __restrict__ s, const double* __restrict__ part, int j) {
  if (s[2] != 0.0) return 0.0;
  const double pq = pcg_sum(part, 1, j);
  const double a = s[0] / pq;
  return (pq > 0.0 && isfinite(a)) ? a : 0.0;
}

// alpha = rho / p^T q; x += alpha p; r -= alpha q; z = r; partials of r^T r.
__global__ void __launch_bounds__(256) k_pcg_xr(double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                                               const double* __restrict__ p, const double* __restrict__ q, int64_t n,
                                               const double* __restrict__ st, double* __restrict__ part,
                                               const int* __restrict__ active) {
  if (*active == 0) return;
  const int j = blockIdx.y;
  const double a = pcg_alpha(st + j * PCG_SLOT, part, j);
  double rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const size_t at = (size_t)j * n + i;
    double rv = r[at];
    if (a != 0.0) {
      x[at] += a * p[at];
      rv -= a * q[at];
      r[at] = rv;
    }
    z[at] = rv;
    rr += rv * rv;
  }
  __shared__ double red[40];
  rr = block_sum(rr, red);
  if (threadIdx.x == 0) __stcg(part + PCG_PART(0, j) + blockIdx.x, rr);
}

// Whether the preconditioner must run this step: some system still iterating
// whose updated residual is above the tolerance.  A system that has just met it
// is marked done by k_pcg_dir from the same r^T r, so its z is never used and
// the sweep is skipped when no other system needs it (one block).
__global__ void k_pcg_gate(const double* __restrict__ st, const double* __restrict__ part,
                           const int* __restrict__ active, int* __restrict__ act_sweep, int nrhs, double tol2) {
  if (threadIdx.x != 0) return;
  int any = 0;
  if (*active != 0)
    for (int j = 0; j < nrhs; ++j) {
      const double* s = st + j * PCG_SLOT;
      if (s[2] != 0.0) continue;
      const double rr = pcg_sum(part, 0, j);
      if (pcg_alpha(s, part, j) != 0.0 && rr > tol2 * s[1]) any = 1;
    }
  *act_sweep = any;
}

// Partials of r^T z (after z = P^-1 r).
__global__ void __launch_bounds__(256) k_pcg_rz(const double* __restrict__ r, const double* __restrict__ z, int64_t n,
                                               double* __restrict__ part, const int* __restrict__ active) {
  if (*active == 0) return;
  const int j = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += r[(size_t)j * n + i] * z[(size_t)j * n + i];
  __shared__ double red[40];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) __stcg(part + PCG_PART(2, j) + blockIdx.x, acc);
}

// beta = rho' / rho; p = z + beta p; convergence test on the recursive
// residual; block (0, 0) writes the next slot (also when nothing iterates, so
// the next iteration reads a valid slot).
__global__ void __launch_bounds__(256) k_pcg_dir(double* __restrict__ p, const double* __restrict__ z, int64_t n,
                                                const double* __restrict__ st_cur, double* __restrict__ st_nxt,
                                                const int* __restrict__ act_cur, int* __restrict__ act_nxt,
                                                int* __restrict__ iters, const double* __restrict__ part, int nrhs,
                                                double tol2) {
  const int j = blockIdx.y;
  const bool on = *act_cur != 0;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    int any = 0;
    for (int k = 0; k < PCG_RHS_MAX; ++k) {
      const double* s = st_cur + k * PCG_SLOT;
      double* t = st_nxt + k * PCG_SLOT;
      t[0] = s[0]; t[1] = s[1]; t[2] = s[2]; t[3] = s[3];
      if (!on || k >= nrhs || s[2] != 0.0) continue;
      const double a = pcg_alpha(s, part, k);
      const double rr = pcg_sum(part, 0, k), rz = pcg_sum(part, 2, k);
      const bool done = a == 0.0 || !(rr > tol2 * s[1]) || !(rz > 0.0) || !isfinite(rz);
      t[0] = rz;
      t[2] = done ? 1.0 : 0.0;
      t[3] = rr;
      any |= done ? 0 : 1;
    }
    *act_nxt = any;
    if (on) *iters += 1;
  }
  if (!on || j >= nrhs) return;
  const double* s = st_cur + j * PCG_SLOT;
  if (s[2] != 0.0) return;
  const double beta = pcg_sum(part, 2, j) / s[0];
  if (!isfinite(beta)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const size_t at = (size_t)j * n + i;
    p[at] = z[at] + beta * p[at];
  }
}

// True residual after the iteration: partials of ||b - q||^2 (q = M~ x), then
// res = max_j sqrt(||b_j - q_j||^2 / ||b_j||^2).
__global__ void __launch_bounds__(256) k_pcg_true(const double* __restrict__ b, const double* __restrict__ q, int64_t n,
                                                 double* __restrict__ part) {
  const int j = blockIdx.y;
  double acc = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bv = b[(size_t)j * n + i], d = bv - q[(size_t)j * n + i];
    acc += d * d;
    bb += bv * bv;
  }
  __shared__ double red[40];
  acc = block_sum(acc, red);
  bb = block_sum(bb, red);
  if (threadIdx.x == 0) {
    __stcg(part + PCG_PART(0, j) + blockIdx.x, acc);
    __stcg(part + PCG_PART(1, j) + blockIdx.x, bb);
  }
}

__global__ void k_pcg_res(const double* __restrict__ part, int nrhs, double* __restrict__ res,
                          const int* __restrict__ iters, int* __restrict__ iters_out) {
  if (threadIdx.x != 0) return;
  double m = 0.0;
  for (int j = 0; j < nrhs; ++j) {
    const double d = pcg_sum(part, 0, j), bb = pcg_sum(part, 1, j);
    const double v = bb > 0.0 ? sqrt(d / bb) : sqrt(d);
    m = fmax(m, v);
  }
  if (res) *res = m;
  if (iters_out) *iters_out = *iters;
}

// The same report from the recursive residual of the final state slot:
// res = max_j sqrt(r_j^T r_j / b_j^T b_j) (no extra product with A).
__global__ void k_pcg_res_recursive(const double* __restrict__ st, int nrhs, double* __restrict__ res,
                                    const int* __restrict__ iters, int* __restrict__ iters_out) {
  if (threadIdx.x != 0) return;
  double m = 0.0;
  for (int j = 0; j < nrhs; ++j) {
    const double* s = st + j * PCG_SLOT;
    const double v = s[1] > 0.0 ? sqrt(fmax(s[3], 0.0) / s[1]) : sqrt(fmax(s[3], 0.0));
    m = fmax(m, v);
  }
  if (res) *res = m;
  if (iters_out) *iters_out = *iters;
}

cudaError_t launch_pcg_residual0(const double* b, double* r, double* z, int64_t n, int nrhs, double* part,
                                 cudaStream_t st) {
  k_pcg_residual0<<<dim3(PCG_NB, nrhs), 256, 0, st>>>(b, r, z, n, part);
  return cudaGetLastError();
}
cudaError_t launch_pcg_start(const double* r, const double* z, double* p, int64_t n, int nrhs, double* part,
                             double* stt, int* act, int* iters, double tol2, cudaStream_t st) {
  k_pcg_start<<<dim3(PCG_NB, nrhs), 256, 0, st>>>(r, z, p, n, part);
  k_pcg_init<<<1, 32, 0, st>>>(stt, act, iters, part, nrhs, tol2);
  return cudaGetLastError();
}
cudaError_t launch_pcg_pq(const double* p, const double* q, int64_t n, int nrhs, double* part, const int* active,
                          cudaStream_t st) {
  k_pcg_pq<<<dim3(PCG_NB, nrhs), 256, 0, st>>>(p, q, n, part, active);
  return cudaGetLastError();
}
cudaError_t launch_pcg_update(double* x, double* r, double* z, const double* p, const double* q, int64_t n, int nrhs,
                              const double* stt, double* part, const int* active, int* act_sweep, double tol2,
                              cudaStream_t st) {
  k_pcg_xr<<<dim3(PCG_NB, nrhs), 256, 0, st>>>(x, r, z, p, q, n, stt, part, active);
  k_pcg_gate<<<1, 32, 0, st>>>(stt, part, active, act_sweep, nrhs, tol2);
  return cudaGetLastError();
}
cudaError_t launch_pcg_direction(const double* r, double* p, const double* z, int64_t n, int nrhs,
                                 const double* st_cur, double* st_nxt, const int* act_cur, int* act_nxt, int* iters,
                                 double* part, double tol2, cudaStream_t st) {
  k_pcg_rz<<<dim3(PCG_NB, nrhs), 256, 0, st>>>(r, z, n, part, act_cur);
  k_pcg_dir<<<dim3(PCG_NB, nrhs), 256, 0, st>>>(p, z, n, st_cur, st_nxt, act_cur, act_nxt, iters, part, nrhs, tol2);
  return cudaGetLastError();
}
cudaError_t launch_pcg_true_residual(const double* b, const double* q, int64_t n, int nrhs, double* part,
                                     double* res, const int* iters, int* iters_out, cudaStream_t st) {
  k_pcg_true<<<dim3(PCG_NB, nrhs), 256, 0, st>>>(b, q, n, part);
  k_pcg_res<<<1, 32, 0, st>>>(part, nrhs, res, iters, iters_out);
  return cudaGetLastError();
}
cudaError_t launch_pcg_recursive_residual(const double* st_final, int nrhs, double* res, const int* iters,
                                          int* iters_out, cudaStream_t st) {
  k_pcg_res_recursive<<<1, 32, 0, st>>>(st_final, nrhs, res, iters, iters_out);
  return cudaGetLastError();
}
