// Mixed-precision solves with M~ (k_mixed.cu): the FP32 copy of an FP64
// factor and the device-side conjugate-gradient steps around it.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fifa_common.cuh"

#define PCG_NB 120      // partial-sum blocks per right-hand side
#define PCG_SLOT 8      // doubles of state per right-hand side and parity slot
#define PCG_RHS_MAX 2
// Scratch of one solve (doubles): partials [0, 6 PCG_NB), state [768, 800),
// then ints: act[2], iters, act_sweep, at double offset 800.
#define PCG_SCRATCH_DOUBLES 1024
#define PCG_OFF_STATE 768
#define PCG_OFF_INTS 800

// F32 (prec 1) <- F64 rounded to FP32 (leaf factors, reciprocal pivots, used
// basis columns); nothing when F64's skip flag is set.  nprob descriptor pairs.
cudaError_t launch_demote(const FactDesc* F64, const FactDesc* F32, int64_t n, cudaStream_t st, int nprob = 1);

cudaError_t launch_pcg_residual0(const double* b, double* r, double* z, int64_t n, int nrhs, double* part,
                                 cudaStream_t st);
cudaError_t launch_pcg_start(const double* r, const double* z, double* p, int64_t n, int nrhs, double* part,
                             double* stt, int* act, int* iters, double tol2, cudaStream_t st);
cudaError_t launch_pcg_pq(const double* p, const double* q, int64_t n, int nrhs, double* part, const int* active,
                          cudaStream_t st);
// x, r (and z = r) updated, then act_sweep = whether any system still needs the
// preconditioner this step (its updated residual above the tolerance).
cudaError_t launch_pcg_update(double* x, double* r, double* z, const double* p, const double* q, int64_t n, int nrhs,
                              const double* stt, double* part, const int* active, int* act_sweep, double tol2,
                              cudaStream_t st);
cudaError_t launch_pcg_direction(const double* r, double* p, const double* z, int64_t n, int nrhs,
                                 const double* st_cur, double* st_nxt, const int* act_cur, int* act_nxt, int* iters,
                                 double* part, double tol2, cudaStream_t st);
cudaError_t launch_pcg_true_residual(const double* b, const double* q, int64_t n, int nrhs, double* part,
                                     double* res, const int* iters, int* iters_out, cudaStream_t st);
// res = max_j ||r_j|| / ||b_j|| from the recursive residuals of the final state slot.
cudaError_t launch_pcg_recursive_residual(const double* st_final, int nrhs, double* res, const int* iters,
                                          int* iters_out, cudaStream_t st);
