// Host-side object definitions behind the opaque handles of fifa.h.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <utility>
#include <vector>

#include "../../include/fifa.h"
#include "fifa_common.cuh"

struct Arena {
  char* base = nullptr;
  size_t size = 0, in_use = 0, peak = 0;
  std::map<size_t, size_t> free_;  // offset -> size
  std::map<size_t, size_t> used_;
  void* alloc(size_t bytes);
  void release(void* p);
};

struct Plan {
  int64_t n = 0;
  int B = 0, L = 0, nleaf = 0, nnodes = 0, Bm = 0;
  std::vector<int> bnd_host;
  int* bnd_dev = nullptr;
  int4* aca_work = nullptr;  // coop entries first, then solo entries
  int aca_ncoop = 0, aca_nsolo = 0, aca_nwarp = 0;
  std::vector<int4> work_host;
  size_t work_off = 0, dev_bytes = 0;  // device block: bounds, then the work list at work_off
  std::vector<int> lvl_G[3], sweep_G;  // lvl_G[b]: group size of the level kernel of rank bucket b
  int lvl_ctas_max = 1;
  int fs_ls = -1, fs_rows = 0;  // fused sweep: 2^fs_ls CTAs of fs_rows rows (-1: per-level sweeps)
  int mv_ls = -1, mv_rows = 0;  // fused H-matvec: 2^mv_ls CTAs of mv_rows rows (-1: three-pass product)
  size_t scratch_bytes = 0;
};

struct Scratch {
  ArgMax* aca_part;
  unsigned int* aca_bar;
  double* lvl_part;
  unsigned int* lvl_bar;
  double* sweep_part;
  double* mv_part;
  double* mv_proj;
  double* vec;  // 16 n doubles
  double* red;  // 512 doubles of reduction partials
  int* flags;
  double* fs_part;        // fused sweep partials
  unsigned int* fs_bar;   // fused sweep grid barrier
  double* mv_fpart;       // fused H-matvec partials
  unsigned int* mv_bar;   // fused H-matvec grid barrier
  double* pcg;            // PCG_SCRATCH_DOUBLES: partial sums and state of a mixed-precision solve
};

struct fifa_ctx {
  fifa_opts opts{};
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  Arena arena;
  bool own_arena = false;
  std::map<std::pair<int64_t, int>, Plan*> plans;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  int aca_coresident = 0;
  int level_coresident[3] = {0, 0, 0};  // per rank bucket, least over the two precisions
  int* flags = nullptr;       // device
  int* host_flags = nullptr;  // pinned
  bool capturing = false;
  void* active_scratch = nullptr;  // a chain's own scratch while it enqueues work
  cudaError_t last_cuda = cudaSuccess;
};

struct fifa_hmat {
  Plan* plan = nullptr;
  HmatDesc host{};
  HmatDesc* dev = nullptr;
  bool owns = false;
  const fifa_hmat* base = nullptr;
};

struct fifa_fact {
  Plan* plan = nullptr;
  FactDesc host{};
  FactDesc* dev = nullptr;
  const fifa_hmat* src = nullptr;  // the factored operator (the one a mixed solve iterates on)
  // Mixed precision: an FP32 copy of this FP64 factor (prec 1; Zf, Zi, ranks,
  // log-determinant and status shared), refreshed after every factorization
  // and applied as the preconditioner of the FP64-residual iteration.
  bool has32 = false;
  FactDesc host32{};
  FactDesc* dev32 = nullptr;
};

Plan* get_plan(fifa_ctx* ctx, int64_t n, fifa_status* st);
// The divisor of every co-resident CTA budget of a context (fifa_opts.coresident_share).
inline int coresident_share(const fifa_opts& o) { return o.coresident_share > 1 ? o.coresident_share : 1; }
// Point a context (created on a caller-provided arena) at another device
// range: drops its plans and every object in the old arena (synchronizes).
fifa_status ctx_rebind_arena(fifa_ctx* ctx, void* base, size_t bytes);
// Arena bytes of one hmat / fact / chain (every allocation rounded as the arena does).
size_t hmat_bytes(const Plan* P, int cap);
size_t fact_bytes(const Plan* P, int cap, int with32);
size_t chain_bytes(const Plan* P, const fifa_opts& o);
Scratch carve(fifa_ctx* ctx, Plan* P);
fifa_status ensure_scratch(fifa_ctx* ctx, Plan* P);
fifa_status hmat_alloc(fifa_ctx* ctx, Plan* P, int kind, fifa_hmat** out);
fifa_status hmat_assemble_enqueue(fifa_ctx* ctx, fifa_hmat* H);
// The assembly in two parts: descriptor reset + grouped ACA (CTAs that wait on
// each other), then leaves + one-CTA / one-warp ACA (independent CTAs).
fifa_status hmat_assemble_grouped_enqueue(fifa_ctx* ctx, fifa_hmat* H);
fifa_status hmat_assemble_rest_enqueue(fifa_ctx* ctx, fifa_hmat* H);
// Assemble nprob H-matrices of plan P (descriptor array H0) in shared launches;
// problem q's scratch at scratch0 + q * sstride bytes.
fifa_status hmat_assemble_batched(fifa_ctx* ctx, Plan* P, HmatDesc* H0, int nprob, void* scratch0, size_t sstride);
// Grid of a fused sweep of nprob factors of plan P in one launch: 2^ls CTAs per
// problem of rows rows each; false if the plan has no fused sweep or nprob
// problems' CTAs cannot all be co-resident.
bool sweep_batch_config(fifa_ctx* ctx, const Plan* P, int nprob, int* ls, int* rows);
// FP64 sweeps (mode as launch_sweep_fused) of nprob factors of plan P
// (descriptor array F0) on one vector each (device array vlist), in one launch
// configured by sweep_batch_config; scratch as hmat_assemble_batched.
fifa_status sweep_enqueue_batched(fifa_ctx* ctx, Plan* P, const FactDesc* F0, double* const* vlist, int nprob,
                                  int mode, int ls, int rows, void* scratch0, size_t sstride);
// with32: also allocate the FP32 copy (a mixed-precision factor of M~).
fifa_status fact_alloc(fifa_ctx* ctx, Plan* P, int with32, fifa_fact** out);
// Point the factor's skip flag at a device int (nullable) and upload its descriptor.
fifa_status fact_set_skip(fifa_ctx* ctx, fifa_fact* F, const int* skip_dev);
fifa_status fact_enqueue(fifa_ctx* ctx, fifa_fact* F, const HmatDesc* Hdev);
// The factorization in two parts: 0 = reset, leaves and the levels without CTA
// groups (independent CTAs only); 1 = the grouped top levels, log-determinant
// and FP32 copy.  fact_ungrouped_from: the first level of part 0's range.
fifa_status fact_enqueue_part(fifa_ctx* ctx, fifa_fact* F, const HmatDesc* Hdev, int part);
int fact_ungrouped_from(const Plan* P);
// W^-1 v (one vector, FP64 factor) in two launches: part 0 = leaves and the
// fused sweep's CTA-local levels (independent CTAs), part 1 = the levels above
// (one cooperative launch); the same arithmetic as the one-launch sweep.
bool sweep_inverse_split_ok(const Plan* P);
fifa_status sweep_inverse_part_enqueue(fifa_ctx* ctx, const fifa_fact* F, double* v, int part);
// F32_0 (nullable): the problems' FP32 copies, refreshed after the factorization.
fifa_status fact_enqueue_batched(fifa_ctx* ctx, Plan* P, FactDesc* F0, const HmatDesc* H0, int nprob,
                                 void* scratch0, size_t sstride, const FactDesc* F32_0 = nullptr);
fifa_status sweep_enqueue(fifa_ctx* ctx, const fifa_fact* F, int trans, int inverse, double* v, int nrhs);
// Sweep with a factor descriptor of either precision; mode as launch_sweep_fused
// (4: W^-T W^-1); active (nullable) as there.
fifa_status sweep_enqueue_desc(fifa_ctx* ctx, Plan* P, const FactDesc* Fdev, int prec, int mode, double* v, int nrhs,
                               const int* active = nullptr);
fifa_status matvec_enqueue(fifa_ctx* ctx, const fifa_hmat* A, const double* in, double* out, int nrhs,
                           const int* active = nullptr);
// x = A^-1 b.  FP64 factor: W^-T W^-1 b.  Mixed factor: conjugate gradients on
// the FP64 operator op (default F->src) preconditioned by the FP32 copy.
// res_dev (nullable): the final relative residual, the true ||b - A x|| / ||b||
// (one more FP64 product) if true_res, else the iteration's recursive one;
// iters_dev (nullable): conjugate-gradient iterations taken.
fifa_status solve_enqueue(fifa_ctx* ctx, const fifa_fact* F, const double* b, double* x, int nrhs, double* work,
                          double* res_dev = nullptr, int* iters_dev = nullptr, const fifa_hmat* op = nullptr,
                          bool true_res = true);
fifa_status sample_enqueue(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, const fifa_fact* WM, const double* y,
                           double tau2, double sigma2, uint64_t seed, uint64_t sid, const uint64_t* iter_dev,
                           uint64_t iter_host, double* f, double* mean, const double* scal_dev, double* res_dev = nullptr,
                           int* iters_dev = nullptr, const fifa_hmat* op = nullptr);
// Algorithm 1's two parts (sample_enqueue runs both): the prior part (normals
// a, b; C~ a; W_C b; rhs0 = (tau2 / sigma) C~ a + tau W_C b) reads no data; the
// data part (rhs1 = y / sigma2, the solves with M~, C~ r, f) does.  Both use
// the plan scratch vectors a, b, Ca, rhs of the active scratch.
fifa_status sample_prior_enqueue(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, double tau2, double sigma2,
                                 uint64_t seed, uint64_t sid, const uint64_t* iter_dev, uint64_t iter_host,
                                 const double* scal_dev);
fifa_status sample_data_enqueue(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WM, const double* y, double tau2,
                                double sigma2, double* f, double* mean, const double* scal_dev, double* res_dev,
                                int* iters_dev, const fifa_hmat* op);
// One block's vectors and state for the prior part of Algorithm 1 run for
// several blocks at once.
struct Alg1Prior {
  const uint64_t* iter;  // the block's iteration counter (device)
  uint64_t sid;          // its Philox stream id
  double* a;             // n: normals of tag 0
  double* b;             // n: normals of tag 1, then W_C b in place
  double* Ca;            // n
  double* rhs;           // rhs0 at rhs[0..n)
  const double* scal;    // tau2, sigma2 (device)
};
// The prior part for nprob blocks of plan P at once: descriptor arrays C0 (C~)
// and WC0 (W_C); P_dev the blocks' Alg1Prior (device); a_list / b_list /
// Ca_list device arrays of their a, b, Ca; the shared launches' grids (ls < 0:
// one product / sweep per block, C_each / WC_each); scratch as
// hmat_assemble_batched.
fifa_status sample_prior_batched(fifa_ctx* ctx, Plan* P, const HmatDesc* C0, const FactDesc* WC0, const Alg1Prior* P_dev,
                                 const double* const* a_list, double* const* b_list, double* const* Ca_list, int nprob,
                                 uint64_t seed, int sweep_ls, int sweep_rows, int mv_ls, int mv_rows, void* scratch0,
                                 size_t sstride, const fifa_hmat* const* C_each, const fifa_fact* const* WC_each);
// Grid of a fused H-matrix product of nprob problems of plan P in one launch
// (as sweep_batch_config).
bool mv_batch_config(fifa_ctx* ctx, const Plan* P, int nprob, int* ls, int* rows);

// vector kernels (k_vec.cu)
cudaError_t launch_prep_hmat(HmatDesc* H, int nnodes, cudaStream_t st, int nprob = 1);
cudaError_t launch_prep_fact(FactDesc* F, const HmatDesc* H, int nnodes, cudaStream_t st, int nprob = 1);
cudaError_t launch_sumsq(const double* a, const double* b, int64_t n, double* part, double* out, cudaStream_t st);
cudaError_t launch_axpy(double a, const double* x, double* y, int64_t n, cudaStream_t st);
cudaError_t launch_alg1_finish(const double* wr, const double* Cr, double* f, double* mean, int64_t n, double tau2,
                               const double* scal_dev, cudaStream_t st);
cudaError_t launch_alg1_rhs_part(const double* Ca, const double* Wb, const double* y, double* rhs, int64_t n,
                                 double tau2, double sigma2, const double* scal_dev, int part, cudaStream_t st);
cudaError_t launch_alg1_prior_normals(uint64_t seed, const Alg1Prior* P, int nprob, int64_t n, cudaStream_t st);
cudaError_t launch_alg1_prior_rhs(const Alg1Prior* P, int nprob, int64_t n, cudaStream_t st);
cudaError_t launch_alg1h_scale(const double* d, double* a, int64_t n, cudaStream_t st);
cudaError_t launch_alg1h_rhs(const double* Ca, const double* Wb, const double* y, double* rhs, int64_t n, double tau2,
                             cudaStream_t st);
cudaError_t launch_alg1h_finish(const double* Zs, const double* Cr, const double* d, double* f, double* R, int64_t n,
                                double tau2, cudaStream_t st);
fifa_status sample_hetero_enqueue(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, const fifa_fact* WP,
                                  const double* y, double tau2, const double* d, uint64_t seed, uint64_t sid,
                                  const uint64_t* iter_dev, uint64_t iter_host, double* f, double* R,
                                  double* res_dev = nullptr, int* iters_dev = nullptr);
