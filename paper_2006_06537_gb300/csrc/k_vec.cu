// Vector, random-number and check kernels.
//
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
//   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key advanced by the Weyl increments W0 = floor(2^32 (phi - 1)),
// W1 = floor(2^32 (sqrt 3 - 1)) between rounds.  Counter = (pair or attempt
// index, stream tag, iteration, stream id), key = seed.  Uniforms are
// (52-bit integer + 0.5) * 2^-52; normals by Box-Muller, two per call.
#include "fifa_common.cuh"
#include "fifa_launch.h"
#include "fifa_rng.cuh"

__global__ void k_det_exp(const double* __restrict__ in, double* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = det_exp(in[i]);
}

__global__ void k_normals(uint64_t seed, uint32_t tag, const uint64_t* __restrict__ iter_dev, uint64_t iter_host,
                          uint64_t stream_id, double* __restrict__ out, int64_t n) {
  const uint64_t it = iter_dev ? *iter_dev : iter_host;
  const int64_t nq = (n + 1) / 2;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
    double z0, z1;
    philox_normal_pair(seed, (uint32_t)q, tag, it, stream_id, z0, z1);
    out[2 * q] = z0;
    if (2 * q + 1 < n) out[2 * q + 1] = z1;
  }
}

__global__ void k_check_sorted(const double* __restrict__ x, int64_t n, int* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i + 1 < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = x[i], b = x[i + 1];
    if (!(a <= b)) atomicOr(flag, 1);
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicOr(flag, 2);
}

__global__ void k_philox(uint64_t seed, const uint32_t* __restrict__ ctr, uint32_t* __restrict__ out, int64_t cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    uint4 w = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    out[4 * i] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
  }
}

static int grid_for(int64_t n, int per = 256) {
  int64_t g = (n + per - 1) / per;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_det_exp(const double* in, double* out, int64_t n, cudaStream_t st) {
  k_det_exp<<<grid_for(n), 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_normals(uint64_t seed, uint32_t tag, const uint64_t* iter_dev, uint64_t iter_host, uint64_t stream_id,
                           double* out, int64_t n, cudaStream_t st) {
  k_normals<<<grid_for((n + 1) / 2), 256, 0, st>>>(seed, tag, iter_dev, iter_host, stream_id, out, n);
  return cudaGetLastError();
}

cudaError_t launch_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t cnt, cudaStream_t st) {
  k_philox<<<grid_for(cnt), 256, 0, st>>>(seed, ctr, out, cnt);
  return cudaGetLastError();
}

cudaError_t launch_check_sorted(const double* x, int64_t n, int* flag, cudaStream_t st) {
  k_check_sorted<<<grid_for(n), 256, 0, st>>>(x, n, flag);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Elementwise pieces of Algorithm 1 and of iterative refinement.
// ---------------------------------------------------------------------------
#include "fifa_api_internal.h"

__global__ void k_axpy(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}


// The two halves of the right-hand sides of Algorithm 1: rhs[0..n) =
// (tau2 / sigma) Ca + tau Wb (part 0), rhs[n..2n) = y / sigma2 (part 1).
__global__ void k_alg1_rhs_part(const double* __restrict__ Ca, const double* __restrict__ Wb,
                                const double* __restrict__ y, double* __restrict__ rhs, int64_t n, double tau2,
                                double sigma2, const double* scal, int part) {
  if (scal) {
    tau2 = scal[0];
    sigma2 = scal[1];
  }
  const double tau = sqrt(tau2), sig = sqrt(sigma2), a = tau2 / sig;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (part == 0) rhs[i] = a * Ca[i] + tau * Wb[i];
    else rhs[n + i] = y[i] / sigma2;
  }
}

// The data-independent start of Algorithm 1 for several blocks at once
// (blockIdx.y): normals a (tag 0) and b (tag 1) of each block's Philox stream,
// and after its products rhs0 = (tau2 / sigma) C a + tau W_C b.
__global__ void k_alg1_prior_normals(uint64_t seed, const Alg1Prior* __restrict__ P, int64_t n) {
  const Alg1Prior& q = P[blockIdx.y >> 1];
  const uint32_t tag = blockIdx.y & 1;
  double* out = tag ? q.b : q.a;
  const uint64_t it = *q.iter;
  const int64_t nq = (n + 1) / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
    double z0, z1;
    philox_normal_pair(seed, (uint32_t)i, tag, it, q.sid, z0, z1);
    out[2 * i] = z0;
    if (2 * i + 1 < n) out[2 * i + 1] = z1;
  }
}
__global__ void k_alg1_prior_rhs(const Alg1Prior* __restrict__ P, int64_t n) {
  const Alg1Prior& q = P[blockIdx.y];
  const double tau2 = q.scal[0], sigma2 = q.scal[1];
  const double tau = sqrt(tau2), sig = sqrt(sigma2), a = tau2 / sig;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    q.rhs[i] = a * q.Ca[i] + tau * q.b[i];
}

// f = w + tau2 C r ; mean = tau2 C r
__global__ void k_alg1_finish(const double* __restrict__ wr, const double* __restrict__ Cr, double* __restrict__ f,
                              double* __restrict__ mean, int64_t n, double tau2, const double* scal) {
  if (scal) tau2 = scal[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double mu = tau2 * Cr[i];
    f[i] = wr[i] + mu;
    if (mean) mean[i] = mu;
  }
}

cudaError_t launch_axpy(double a, const double* x, double* y, int64_t n, cudaStream_t st) {
  k_axpy<<<grid_for(n), 256, 0, st>>>(a, x, y, n);
  return cudaGetLastError();
}
cudaError_t launch_alg1_rhs_part(const double* Ca, const double* Wb, const double* y, double* rhs, int64_t n,
                                 double tau2, double sigma2, const double* scal_dev, int part, cudaStream_t st) {
  k_alg1_rhs_part<<<grid_for(n), 256, 0, st>>>(Ca, Wb, y, rhs, n, tau2, sigma2, scal_dev, part);
  return cudaGetLastError();
}
cudaError_t launch_alg1_prior_normals(uint64_t seed, const Alg1Prior* P, int nprob, int64_t n, cudaStream_t st) {
  k_alg1_prior_normals<<<dim3(grid_for((n + 1) / 2), 2 * nprob), 256, 0, st>>>(seed, P, n);
  return cudaGetLastError();
}
cudaError_t launch_alg1_prior_rhs(const Alg1Prior* P, int nprob, int64_t n, cudaStream_t st) {
  k_alg1_prior_rhs<<<dim3(grid_for(n), nprob), 256, 0, st>>>(P, n);
  return cudaGetLastError();
}
cudaError_t launch_alg1_finish(const double* wr, const double* Cr, double* f, double* mean, int64_t n, double tau2,
                               const double* scal_dev, cudaStream_t st) {
  k_alg1_finish<<<grid_for(n), 256, 0, st>>>(wr, Cr, f, mean, n, tau2, scal_dev);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Object preparation through device descriptors (so a captured graph follows
// descriptor swaps): zero an H-matrix's status and ranks; copy ranks into a
// factor and zero its status.
// ---------------------------------------------------------------------------
__global__ void k_prep_hmat(HmatDesc* __restrict__ H, int nnodes) {
  H += blockIdx.y;  // problem of a batched launch (descriptor arrays)
  int* rk = H->rank;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnodes; i += gridDim.x * blockDim.x) rk[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *H->status = 0;
}

__global__ void k_prep_fact(FactDesc* __restrict__ F, const HmatDesc* __restrict__ H, int nnodes) {
  F += blockIdx.y;  // problem of a batched launch (descriptor arrays)
  H += blockIdx.y;
  if (F->skip && *F->skip) return;  // the factor is kept: its ranks and status stay
  int* dst = F->rank;
  const int* src = H->rank;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnodes; i += gridDim.x * blockDim.x) dst[i] = src[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) *F->status = 0;
}

cudaError_t launch_prep_hmat(HmatDesc* H, int nnodes, cudaStream_t st, int nprob) {
  k_prep_hmat<<<dim3(grid_for(nnodes > 0 ? nnodes : 1), nprob), 256, 0, st>>>(H, nnodes);
  return cudaGetLastError();
}
cudaError_t launch_prep_fact(FactDesc* F, const HmatDesc* H, int nnodes, cudaStream_t st, int nprob) {
  k_prep_fact<<<dim3(grid_for(nnodes > 0 ? nnodes : 1), nprob), 256, 0, st>>>(F, H, nnodes);
  return cudaGetLastError();
}

// Deterministic sum of squares: fixed grid of partial sums, then one block in order.
__global__ void k_sumsq_part(const double* __restrict__ a, const double* __restrict__ b, int64_t n, double* __restrict__ part) {
  __shared__ double red[40];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = b ? a[i] - b[i] : a[i];
    acc += d * d;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}
__global__ void k_sumsq_final(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double red[40];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) *out = acc;
}
#define SUMSQ_BLOCKS 256
cudaError_t launch_sumsq(const double* a, const double* b, int64_t n, double* part, double* out, cudaStream_t st) {
  k_sumsq_part<<<SUMSQ_BLOCKS, 256, 0, st>>>(a, b, n, part);
  k_sumsq_final<<<1, 256, 0, st>>>(part, SUMSQ_BLOCKS, out);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// FP64 FMA throughput probe (the roofline denominator of the FP64-issue-bound
// kernels): every thread advances 8 independent chains x <- x a + b of fused
// multiply-adds in registers, no memory traffic; the grid fills every SM.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dfma_probe(double* __restrict__ out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == -1.0) out[0] = s;  // never true (the chains stay near b / (1 - a) > 0); keeps the work
}

cudaError_t launch_dfma_probe(double* out, int iters, int blocks, cudaStream_t st) {
  k_dfma_probe<<<blocks, 256, 0, st>>>(out, iters, 0.999999, 1e-6);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Algorithm 1.h (heteroskedastic noise, precisions d_i): a = sqrt(d) a0;
// rhs = [tau2 C~ a + tau W_C b, y]; after the solves with P~ = tau2 C~ + D^-1:
// R = tau2 C~ P~^-1 y and f = R + D^-1 P~^-1 Z.
// ---------------------------------------------------------------------------
__global__ void k_alg1h_scale(const double* __restrict__ d, double* __restrict__ a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] *= sqrt(d[i]);
}
__global__ void k_alg1h_rhs(const double* __restrict__ Ca, const double* __restrict__ Wb, const double* __restrict__ y,
                            double* __restrict__ rhs, int64_t n, double tau2) {
  const double tau = sqrt(tau2);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    rhs[i] = tau2 * Ca[i] + tau * Wb[i];
    rhs[n + i] = y[i];
  }
}
__global__ void k_alg1h_finish(const double* __restrict__ Zs, const double* __restrict__ Cr, const double* __restrict__ d,
                               double* __restrict__ f, double* __restrict__ R, int64_t n, double tau2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double r = tau2 * Cr[i];
    f[i] = r + Zs[i] / d[i];
    if (R) R[i] = r;
  }
}
cudaError_t launch_alg1h_scale(const double* d, double* a, int64_t n, cudaStream_t st) {
  k_alg1h_scale<<<grid_for(n), 256, 0, st>>>(d, a, n);
  return cudaGetLastError();
}
cudaError_t launch_alg1h_rhs(const double* Ca, const double* Wb, const double* y, double* rhs, int64_t n, double tau2,
                             cudaStream_t st) {
  k_alg1h_rhs<<<grid_for(n), 256, 0, st>>>(Ca, Wb, y, rhs, n, tau2);
  return cudaGetLastError();
}
cudaError_t launch_alg1h_finish(const double* Zs, const double* Cr, const double* d, double* f, double* R, int64_t n,
                                double tau2, cudaStream_t st) {
  k_alg1h_finish<<<grid_for(n), 256, 0, st>>>(Zs, Cr, d, f, R, n, tau2);
  return cudaGetLastError();
}
