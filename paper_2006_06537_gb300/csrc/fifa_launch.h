// Host-side launchers of the device kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include "fifa_common.cuh"

// Assembly launchers take nprob problems of one plan (descriptor arrays,
// blockIdx.y); the grouped ACA's partials / barriers / abort flags of problem q
// sit q * pstride bytes after problem 0's.
cudaError_t launch_leaf_assemble(const HmatDesc* Hd, int nleaf, cudaStream_t st, int nprob = 1);
#define ACA_WARP_MAX 128  // largest side of a block that the warp-per-block ACA takes
cudaError_t launch_aca_warp(const HmatDesc* Hd, const int4* work, int nwork, cudaStream_t st, int nprob = 1);
cudaError_t launch_aca(const HmatDesc* Hd, const int4* work, int ncta, bool cooperative, ArgMax* part,
                       unsigned int* bar, int* abort_flag, cudaStream_t st, int nprob = 1, size_t pstride = 0);
int aca_max_coresident_ctas();

size_t leaf_factor_smem(int Bm, int L, int cap, int prec);
size_t level_smem(int ldm, int cap);
// Doubles per CTA slot of the level kernel's partial sums: a cap x cap Gram
// matrix or a 2cap x 8 projection block.
__host__ __device__ inline size_t level_part_stride(int cap) {
  // the larger of the packed Gram entries of both sides, r (r + 1) <= cap (cap + 1),
  // and a 2 cap x 8 projection chunk
  return (size_t)(cap * (cap + 1) > 2 * cap * 8 ? cap * (cap + 1) : 2 * cap * 8);
}
cudaError_t launch_leaf_factor(const HmatDesc* Hd, const FactDesc* Fd, int prec, int nleaf, int Bm, int L, int cap,
                               cudaStream_t st, int nprob = 1);
#define LEVEL_BUCKETS 3
// Level kernels: rank buckets (.., 4], (4, 16], (16, cap] with groups of G[b]
// CTAs; bucket b uses the barriers at bar + b * bar_stride.
// nprob problems in one launch (grid.y): descriptor arrays, scratch sstride bytes apart.
cudaError_t launch_level(const FactDesc* Fd, int prec, int lvl, int nodes, const int* G, int cap, double* part,
                         unsigned int* bar, int bar_stride, int* abort_flag, int side_max, cudaStream_t st,
                         int nprob = 1, size_t sstride = 0);
// Co-resident CTAs of the level kernel of rank bucket b (0: <= 4, 1: 5..16, 2: > 16).
int level_bucket_coresident(int prec, int b, int cap);
cudaError_t launch_logdet_reduce(const FactDesc* Fd, cudaStream_t st, int nprob = 1);

#define SWEEP_RHS_MAX 2
// active (nullable): when *active == 0 the application / product kernels return at
// once (iterations of a solve that has converged).
cudaError_t launch_sweep_level(const FactDesc* Fd, int prec, int lvl, int nodes, int G, double* v, int nrhs, double* part,
                               int zsel, int ztrans, cudaStream_t st, const int* active = nullptr);
// Fused sweep (one cooperative launch of 2^ls CTAs; rows >= the longest
// level-ls node).  part: 2 * 2^ls * FS_PART_STRIDE doubles; bar zeroed before.
#define FS_PART_STRIDE (2 * FIFA_CAP_MAX * SWEEP_RHS_MAX)
#define FS_CTAS_MAX 1024
int sweep_fused_coresident(int prec, int rows, int cap);
// mode 0: W v, 1: W^-1 v, 2: W^T v, 3: W^-T v, 4: W^-T W^-1 v (both inverse sweeps
// in one launch); mode 1 in two launches with the same arithmetic: 5 = its
// leaves and levels >= ls (CTAs independent, launched non-cooperatively; reads
// only those levels of the factor), then 6 = its levels < ls.  Arithmetic in
// the factor's storage precision (prec 1: FP32).
cudaError_t launch_sweep_fused(const FactDesc* Fd, int prec, int ls, int rows, int cap, double* v, int nrhs,
                               int mode, double* part, unsigned int* bar, int* abort_flag, cudaStream_t st,
                               const int* active = nullptr);
// nprob FP64 factors of one plan in one launch (one right-hand side each at
// vlist[q]; per-problem partials / barrier / abort flag pstride bytes apart)
cudaError_t launch_sweep_fused_batched(const FactDesc* Fd, int ls, int rows, double* const* vlist, int nprob,
                                       int mode, double* part, unsigned int* bar, int* abort_flag, size_t pstride,
                                       cudaStream_t st);
// Fused H-matrix product (one cooperative launch of 2^ls CTAs, rows <= 4096).
// part: 2^ls * ls * MV_PART_STRIDE doubles; bar zeroed before.
#define MV_FUSED_ROWS_MAX 4096
int mv_fused_coresident(int rows);
cudaError_t launch_mv_fused(const HmatDesc* Hd, int ls, int rows, const double* x, int nrhs, double* y, double* part,
                            unsigned int* bar, int* abort_flag, cudaStream_t st, const int* active = nullptr);
// nprob H-matrices of one plan in one launch (one right-hand side each:
// xlist[q] -> ylist[q]; per-problem partials / barrier / abort flag pstride
// bytes apart)
cudaError_t launch_mv_fused_batched(const HmatDesc* Hd, int ls, int rows, const double* const* xlist,
                                    double* const* ylist, int nprob, double* part, unsigned int* bar, int* abort_flag,
                                    size_t pstride, cudaStream_t st);
cudaError_t launch_sweep_leaf(const FactDesc* Fd, int prec, int nleaf, double* v, int nrhs, int mode, cudaStream_t st,
                              const int* active = nullptr);
cudaError_t launch_matvec(const HmatDesc* Hd, int nleaf, int L, const double* x, int nrhs, double* part, double* proj,
                          double* y, cudaStream_t st, const int* active = nullptr);

// vector / random / scalar kernels (k_gibbs.cu)
cudaError_t launch_det_exp(const double* in, double* out, int64_t n, cudaStream_t st);
cudaError_t launch_normals(uint64_t seed, uint32_t tag, const uint64_t* iter_dev, uint64_t iter_host, uint64_t stream_id,
                           double* out, int64_t n, cudaStream_t st);
cudaError_t launch_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t cnt, cudaStream_t st);
cudaError_t launch_check_sorted(const double* x, int64_t n, int* flag, cudaStream_t st);
// FP64 FMA throughput probe: 16 iters flops per thread, 256 threads per block.
cudaError_t launch_dfma_probe(double* out, int iters, int blocks, cudaStream_t st);
