/*
 * fifa.h -- C ABI of the GB300 FIFA-GP Gibbs-step library.
 *
 * Method: Moran & Wheeler, "Fast increased fidelity approximate Gibbs samplers
 * for Bayesian Gaussian process regression" (arXiv 2006.06537).  The library
 * computes, on one GPU, every step of one Gibbs iteration for 1-D inputs:
 * HODLR assembly of the kernel matrix (Sec. 3.2), its symmetric factorization
 * and log-determinant (SI, "HODLR decomposition and factorization",
 * "Determinant computation speedup"), the solves, matrix-vector products and
 * factor applications of Algorithm 1 (Sec. 4.1.1), and the conditional draws
 * of Eqs. (posterior_gibs1)-(posterior_gibs4).
 *
 * Model and notation used by every call:
 *   y = f + e,  e ~ N(0, sigma2 I);   f ~ N(0, tau2 * C(rho))
 *   C(rho)[a][b] = k(x_a, x_b) + nugget * [a == b]   (unit-variance kernel)
 *   SE:         k = exp(-(x_a - x_b)^2 / (2 rho^2))
 *   Matern-5/2: k = (1 + t + t^2/3) exp(-t),  t = sqrt(5) |x_a - x_b| / rho
 *   C~ is the HODLR approximation of C; M~ = s C~ + I with s = tau2 / sigma2
 *   (the paper's M = tau K + I with precision tau = 1/sigma2 and K = tau2 C).
 *
 * Conventions for all calls:
 *   - Device pointers ("_dev") are CUDA global-memory addresses on the
 *     context's device; host pointers ("_host") are ordinary memory.
 *   - The caller owns every buffer it passes; the library owns the opaque
 *     objects, which live inside the context's device arena.
 *   - Calls are asynchronous on the context's stream unless they return a
 *     value through a _host pointer, in which case they synchronize it.
 *   - Inputs x must be sorted non-decreasing (Sec. 3.2 sorts 1-D inputs);
 *     otherwise FIFA_ERR_UNSORTED.  Any n >= 1 is accepted.
 *   - Device-side failures (a non-positive pivot, a timed-out wait) set a
 *     status word in the object; the next synchronizing call on it returns it.
 *   - No C++ exception crosses this boundary.
 */
#ifndef FIFA_H
#define FIFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FIFA_OK = 0,
  FIFA_ERR_INVALID_ARG = 1,
  FIFA_ERR_UNSORTED = 2,
  FIFA_ERR_NOT_SPD = 3,     /* a Cholesky pivot was not positive (PSD loss, SI "Practical considerations") */
  FIFA_ERR_RANK_CAP = 4,    /* an ACA block reached the rank cap before the tolerance */
  FIFA_ERR_OOM = 5,         /* the context arena has no room for the object */
  FIFA_ERR_CUDA = 6,        /* a CUDA runtime call failed */
  FIFA_ERR_TIMEOUT = 7,     /* a bounded device-side wait gave up */
  FIFA_ERR_UNSUPPORTED = 8  /* a size outside what the kernels handle (leaf size, rank cap) */
} fifa_status;

typedef enum { FIFA_KERNEL_SE = 0, FIFA_KERNEL_MATERN52 = 1 } fifa_kernel;
typedef enum { FIFA_FP64 = 0, FIFA_MIXED = 1 } fifa_precision;

/* Hyperparameters Theta of Sec. 4.1 in the length-scale form above. */
typedef struct {
  int kernel;     /* fifa_kernel */
  double tau2;    /* signal variance (the paper's sigma_f^2) */
  double rho;     /* length-scale */
  double sigma2;  /* noise variance (1 / the paper's precision tau) */
  double nugget;  /* added to the diagonal of C before construction (Sec. 4.1.4) */
} fifa_hyper;

/* H-matrix options: Algorithm 1 inputs B (maximum block size) and epsilon. */
typedef struct {
  int leaf_size;      /* B: leaves hold at most B points; 1..128 */
  double aca_tol;     /* absolute max-norm tolerance of every ACA block of C */
  int rank_cap;       /* maximum ACA rank per block; 1..64 */
  int prec;           /* fifa_precision: FP64, or MIXED (see below) */
  double refine_tol;  /* MIXED: stop iterating when ||b - M~ x|| <= refine_tol ||b|| */
  int refine_max;     /* MIXED: conjugate-gradient steps captured per solve (fixed; once every system
                         has converged the remaining steps' launches return at once) */
  int independent_ctas; /* 1: no kernel splits a tree node over a group of CTAs that wait on each
                           other (every CTA runs independently).  0: groups fill the GPU (or the
                           context's coresident_share of it) for the top levels.  Several
                           contexts that launch work concurrently on one GPU need 1, or 0 with
                           coresident_share >= the number of such contexts. */
  int wait_polls;     /* a CTA waiting for the rest of its group gives up after this many polls
                         (each followed by a 64 ns sleep), sets FIFA_ERR_TIMEOUT in the object's
                         status and makes the whole launch return; 0: the default 2^26 polls
                         (seconds).  Objects take the value of the context that created them. */
  int coresident_share; /* 0 or 1: a launch whose CTAs wait on each other may use every CTA the
                           GPU holds at once.  k > 1: at most 1/k of them, so that k contexts
                           with independent_ctas = 0 may launch such work side by side (their
                           waiting launches then fit on the GPU together).  1..64 */
  int overlap_proposal; /* 1: a chain of this context runs the assembly and factorization of its
                           proposal C~(rho') on a second stream of its own, concurrently with
                           Algorithm 1's draw and the sigma2 / tau2 updates (they do not depend
                           on each other: rho' comes from the previous iteration's state).  Only
                           kernels whose CTAs never wait on each other run beside the draw; the
                           grouped top-level ACA runs before it and the grouped top-level
                           factorization after it, so launch sizes and every result are the same
                           as with 0.  Costs a second scratch area per chain (fifa_chain_bytes
                           counts it).  Applies to chains stepped whole (fifa_gibbs_step,
                           serving); the additive and tensor-product models step their blocks
                           phase by phase and do not use it.  0 or 1 */
} fifa_opts;

/* Priors: inverse-gamma IG(shape, scale) on tau2 and sigma2 (the conjugate
 * forms of Eqs. posterior_gibs2-3), normal prior on log rho with a random-walk
 * Metropolis step of standard deviation prop_sd (Sec. 4.1, the Metropolis
 * alternative to the discrete rho grid). */
typedef struct {
  double a_tau2, b_tau2, a_sigma2, b_sigma2;
  double logrho_mu, logrho_sd, prop_sd;
} fifa_prior;

typedef struct fifa_ctx fifa_ctx;     /* device arena, stream, plans, scratch */
typedef struct fifa_hmat fifa_hmat;   /* C~ (assembled) or M~ = s C~ + I (a view of a C~) */
typedef struct fifa_fact fifa_fact;   /* W with W W^T = A, and log det A */
typedef struct fifa_chain fifa_chain; /* Gibbs chain state resident on the device */

/* Create a context on the current CUDA device.
 *   cuda_stream: cudaStream_t to launch on (NULL = legacy default stream).
 *   arena_dev / arena_bytes: device memory the library sub-allocates all its
 *     objects and scratch from (e.g. a torch uint8 tensor); the caller keeps it
 *     alive until fifa_destroy_ctx.  arena_dev == NULL: the library allocates
 *     arena_bytes itself and frees them in fifa_destroy_ctx.
 * Errors: FIFA_ERR_INVALID_ARG (bad opts), FIFA_ERR_UNSUPPORTED, FIFA_ERR_CUDA. */
fifa_status fifa_create(fifa_ctx** out, const fifa_opts* opts, void* cuda_stream,
                        void* arena_dev, size_t arena_bytes);
void fifa_destroy_ctx(fifa_ctx* ctx);

/* Assemble C~(rho) (Sec. 3.2; Algorithm 1 "Construct"): dense leaves
 * C(I_i, I_i) + nugget I and, for every non-leaf node, a partial-pivoted ACA
 * factorization U V^T of its upper off-diagonal block (proof of Lemma 1).
 * x_dev: n sorted doubles (read during this call's kernels only).
 * hyper->tau2 and ->sigma2 are not used here.  Errors: INVALID_ARG, UNSORTED,
 * OOM, CUDA; a block that hits the rank cap sets FIFA_ERR_RANK_CAP as the
 * object's status (results remain usable, the tolerance is not met there). */
fifa_status fifa_assemble(fifa_ctx* ctx, const double* x_dev, int64_t n, const fifa_hyper* hyper,
                          fifa_hmat** out);

/* M~ = s C~ + I (proof of Theorem 4.1: M~ built from K~), as a view that
 * shares C's storage: leaves s D_i + I, U scaled by s, V shared.  C must
 * outlive M.  Errors: INVALID_ARG, OOM. */
fifa_status fifa_shift_scale(fifa_ctx* ctx, const fifa_hmat* C, double s, fifa_hmat** M);

/* P~ = s C~ + diag(diag_dev) (Appendix "Heteroskedastic noise derivation":
 * P~ = K~ + D^-1 with K~ = tau2 C~, s = tau2 and diag_dev = 1/d, the inverse
 * noise precisions), as a view sharing C's storage: leaves s D_i + diag, U
 * scaled by s, V shared.  diag_dev: n device doubles, read by the kernels that
 * use the view (the caller keeps them alive and unchanged meanwhile); C must
 * outlive P.  fifa_factor, fifa_matvec and fifa_solve accept the view.
 * Errors: INVALID_ARG (C itself a view), OOM. */
fifa_status fifa_add_diagonal(fifa_ctx* ctx, const fifa_hmat* C, double s, const double* diag_dev, fifa_hmat** P);

/* The same product as fifa_matvec, for callers that cannot allocate device
 * memory themselves: a plug-in whose host framework owns all device memory,
 * a process whose memory is fully reserved by a pooling allocator, or a
 * latency-critical loop that must not enter the allocator (cudaMalloc can
 * synchronize the device).  The paper has no counterpart; this is a property
 * of the library, not of the method.
 *   Scratch: a file-scope static device array of 2^20 doubles (8 MiB) that every
 *   GPU loading the library holds until exit; no allocation routine is called.
 *   The first call on each device looks up the array's address with
 *   cudaGetSymbolAddress while that device is current and caches it together
 *   with the id of the device's context; make that first call before any
 *   stream capture begins.  After a device reset (a new context) the next call
 *   looks the address up again, so make it outside stream capture as well.
 *   All calls share the array: calls that overlap on the GPU race on it and must
 *   be ordered by the caller.  Each call writes every scratch entry it reads.
 *   Limit: nleaf * levels * rank_cap * 2 + (2^levels - 1) * 4 * rank_cap doubles
 *   must fit in 2^20, else FIFA_ERR_UNSUPPORTED (e.g. rank_cap 32 allows up to
 *   10 levels).  The calling thread's current device must be the context's
 *   (else FIFA_ERR_INVALID_ARG).  in_dev and out_dev must not alias. */
fifa_status fifa_matvec_static(fifa_ctx* ctx, const fifa_hmat* A, const double* in_dev, double* out_dev, int nrhs);

/* Symmetric factorization A = W W^T, W = A_L ... A_0 (SI, Ambikasaran Thm 3.1)
 * and log det A, computed in FP64.  When the context is MIXED and A is a
 * shift_scale view (the M~ of Algorithm 1), the factor also carries an FP32
 * copy of W (leaf factors, reciprocal pivots and bases rounded to FP32) that
 * fifa_solve applies in FP32 arithmetic as the preconditioner of conjugate
 * gradients on the FP64 operator.
 * Errors: OOM, CUDA; NOT_SPD is reported through fifa_fact_status/logdet. */
fifa_status fifa_factor(fifa_ctx* ctx, const fifa_hmat* A, fifa_fact** out);

/* log det A (SI "Determinant computation speedup"); synchronizes.
 * Returns the factor's device status (FIFA_ERR_NOT_SPD if a pivot failed). */
fifa_status fifa_logdet(fifa_ctx* ctx, const fifa_fact* F, double* out_host);

/* x = A^-1 b = W^-T W^-1 b for nrhs column-major vectors of length n.
 * b_dev and x_dev may alias.  For a MIXED factor: conjugate gradients on the
 * FP64 operator A preconditioned by the factor's FP32 copy (applied in FP32
 * arithmetic), x0 = that preconditioner applied to b, at most refine_max steps
 * to ||b - A x|| <= refine_tol ||b|| (fifa_opts).  Errors: INVALID_ARG. */
fifa_status fifa_solve(fifa_ctx* ctx, const fifa_fact* F, const double* b_dev, double* x_dev, int nrhs);

/* out = W32^-T W32^-1 in for a MIXED factor F of M~ (fifa_factor on a
 * shift_scale view in a MIXED context): the preconditioner of its solves, the
 * FP32 copy of W applied in FP32 arithmetic (in and out stay FP64).  Agrees
 * with A^-1 in to about sqrt(kappa(A)) u32.  in_dev and out_dev may alias.
 * Errors: INVALID_ARG (also for a factor without an FP32 copy). */
fifa_status fifa_apply_precond(fifa_ctx* ctx, const fifa_fact* F, const double* in_dev, double* out_dev, int nrhs);

/* out = op(W) in, op = W, W^T, W^-1 or W^-T (trans, inverse in {0,1});
 * in_dev and out_dev may alias.  Errors: INVALID_ARG. */
fifa_status fifa_apply_W(fifa_ctx* ctx, const fifa_fact* F, int trans, int inverse,
                         const double* in_dev, double* out_dev, int nrhs);

/* out = A in (H-matrix product: leaf products plus low-rank blocks).
 * in_dev and out_dev must not alias.  Errors: INVALID_ARG. */
fifa_status fifa_matvec(fifa_ctx* ctx, const fifa_hmat* A, const double* in_dev, double* out_dev, int nrhs);

/* Algorithm 1: a, b ~ N(0, I) from Philox4x32-10 (key = seed, counter =
 * (pair index, stream tag 0/1, iter, stream_id)); Z = (tau2/sigma) C~ a +
 * tau W_C b; solve M~ w = Z; solve M~ r = y / sigma2; f = w + tau2 C~ r.
 * C: C~; WC: factor of C~; WM: factor of M~ = (tau2/sigma2) C~ + I.
 * mean_dev (nullable) receives tau2 C~ r, the posterior mean.  Errors: INVALID_ARG. */
fifa_status fifa_sample(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, const fifa_fact* WM,
                        const double* y_dev, double tau2, double sigma2, uint64_t seed,
                        uint64_t stream_id, uint64_t iter, double* f_dev, double* mean_dev);

/* Algorithm 1.h (Appendix "Heteroskedastic noise derivation"): the draw of
 * f | y for y = f + e, e_i ~ N(0, 1/d_i), f ~ N(0, tau2 C~).  a0, b ~ N(0, I)
 * from Philox4x32-10 (streams as fifa_sample: tags 0 / 1, iter, stream_id);
 * a = sqrt(d) a0; Z = tau2 C~ a + tau W_C b; Z* = P~^-1 Z; R = tau2 C~ P~^-1 y;
 * f = R + D^-1 Z*, with P~ = tau2 C~ + D^-1 (fifa_add_diagonal with diag 1/d).
 * C: C~; WC: factor of C~; WP: factor of P~ (MIXED: solved by conjugate
 * gradients as fifa_solve).  d_dev: n precisions > 0.  R_dev (nullable)
 * receives R, the posterior mean.  Errors: INVALID_ARG. */
fifa_status fifa_sample_hetero(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, const fifa_fact* WP,
                               const double* y_dev, double tau2, const double* d_dev, uint64_t seed,
                               uint64_t stream_id, uint64_t iter, double* f_dev, double* R_dev);

/* Function posterior at new inputs (Sec. "Function posterior at new inputs",
 * Eq. gp_posterior_newx), given f at the training inputs: with K~ = tau2 C~,
 *   mu*_j      = c(x*_j, x)^T C~^-1 f,
 *   sigma*^2_j = tau2 (1 - c(x*_j, x)^T C~^-1 c(x, x*_j)),
 * c the unit-variance kernel of C (its kind and length-scale; no nugget on the
 * cross entries; k(x*, x*) = tau2).  C: an assembled C~ (not a view) of the
 * sorted training inputs x_dev (n doubles); WC: its factor; f_dev: n values;
 * xstar_dev: nstar new inputs in any order.  mu_dev, var_dev (nstar doubles
 * each, either nullable) receive the two results.  Costs one W_C^-T W_C^-1
 * solve and nstar n kernel entries for the means, and one W_C^-1 sweep per two
 * new inputs for the variances.  Errors: INVALID_ARG, UNSUPPORTED. */
fifa_status fifa_predict(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, const double* x_dev,
                         const double* f_dev, const double* xstar_dev, int64_t nstar, double tau2, double* mu_dev,
                         double* var_dev);

/* Length-scale on a discrete grid (Eq. posterior_gibs4, the sampler the paper
 * times, with its factorizations computed once): C~(s_h) assembled and
 * factored in FP64 for every grid value s_h = rho_host[h] (h < G) of the
 * sorted inputs x_dev (copied), kernel and nugget as fifa_hyper.
 * log_prior_host (nullable, G values): log prior weight of each grid value
 * (uniform when null).  Holds G H-matrices and factors in the arena.
 * Errors: INVALID_ARG, UNSORTED, OOM, NOT_SPD (a grid matrix that does not
 * factor), those of fifa_assemble. */
typedef struct fifa_grid fifa_grid;
fifa_status fifa_grid_create(fifa_ctx* ctx, const double* x_dev, int64_t n, int kernel, double nugget,
                             const double* rho_host, int G, const double* log_prior_host, fifa_grid** out);

/* Draw the grid index of rho | f, tau2: log w_h = log prior_h - logdet C~_h / 2
 * - ||W_h^-1 f||^2 / (2 tau2); probabilities normalised after subtracting the
 * largest log weight; index = the first h whose cumulative probability
 * exceeds u, u the Philox uniform of (seed, tag 5, iter, stream_id) (the last
 * index if rounding leaves the total below u).  Synchronizes.  probs_host
 * (nullable) receives the G probabilities.  Errors: INVALID_ARG. */
fifa_status fifa_grid_draw(fifa_ctx* ctx, fifa_grid* grid, const double* f_dev, double tau2, uint64_t seed,
                           uint64_t stream_id, uint64_t iter, int* index_host, double* probs_host);

/* The H-matrix C~(s_h) and its factor (owned by the grid; usable with
 * fifa_sample, fifa_shift_scale, fifa_matvec ...).  Errors: INVALID_ARG. */
fifa_status fifa_grid_get(const fifa_grid* grid, int h, const fifa_hmat** C, const fifa_fact** W);
void fifa_destroy_grid(fifa_ctx* ctx, fifa_grid* grid);

/* A Gibbs chain: copies x, y to the device arena, assembles and factors
 * C~(init->rho); state sigma2 = init->sigma2, tau2 = init->tau2, f = 0.
 * init->nugget and ->kernel fix those settings for the chain.  Errors as
 * fifa_assemble / fifa_factor. */
fifa_status fifa_chain_create(fifa_ctx* ctx, const double* x_dev, const double* y_dev, int64_t n,
                              const fifa_hyper* init, const fifa_prior* prior, uint64_t seed,
                              uint64_t chain_id, fifa_chain** out);

/* Run `iters` Gibbs iterations (Eqs. posterior_gibs1-4 in order: f by
 * Algorithm 1, sigma2, tau2, then the Metropolis step on log rho).  The
 * whole iteration is captured once in a CUDA graph and replayed; nothing
 * returns to the host in between.
 * Precision: an FP64 chain factors M~ = (tau2/sigma2) C~ + I every iteration
 * and solves with it directly.  A MIXED chain keeps its FP64 factor of M~
 * between iterations and refactors only when the Metropolis step accepted a
 * new rho, when tau2/sigma2 moved by more than 5% from the value it was
 * factored at, or when the last solve needed more than 6 conjugate-gradient
 * steps; its M~ solves are conjugate gradients on the current FP64 M~
 * preconditioned by the FP32 copy of the kept factor.  C~ factors, log
 * determinants and W_C products stay FP64 in both.
 * trace_host (nullable): iters rows of FIFA_TRACE_FIELDS doubles (written after
 * the last iteration, synchronizes): iteration, sigma2, tau2, rho, accepted,
 * log alpha, logdet C~(rho), q = f^T C~^-1 f, ||y - f||^2, relative residual of
 * the M~ solves (MIXED: the conjugate gradients' recursive residual, the larger
 * of the two systems; 0 for FP64), status, M~ refactored this iteration (1/0),
 * conjugate-gradient steps of the M~ solves.  Errors: the chain's device status. */
#define FIFA_TRACE_FIELDS 13
fifa_status fifa_gibbs_step(fifa_ctx* ctx, fifa_chain* chain, int iters, double* trace_host);

/* Kernel launches of one Gibbs iteration: the kernel nodes of the captured
 * iteration graph (built by the first fifa_gibbs_step), or -1 if the chain
 * runs without a graph.  Synchronizes nothing. */
fifa_status fifa_chain_kernel_nodes(const fifa_chain* chain, int* out_host);

/* Replace the chain's observations y (n doubles, same inputs x) before its
 * next iteration: y may be host memory (pinned for an asynchronous copy) or
 * device memory; the copy is enqueued on the context's stream (no
 * synchronization), so the caller keeps y unchanged until the stream reaches
 * it.  For data streamed into a resident chain (the model of Sec. 2.1 with
 * fixed inputs).  Errors: INVALID_ARG (also during stream capture), CUDA. */
fifa_status fifa_chain_set_y(fifa_ctx* ctx, fifa_chain* chain, const double* y);

/* Current state: f (and the last posterior mean tau2 C~ r) to device buffers
 * (nullable), hyperparameters to h_host (nullable); synchronizes. */
fifa_status fifa_chain_get(fifa_ctx* ctx, const fifa_chain* chain, double* f_dev, double* mean_dev,
                           fifa_hyper* h_host);

/* Device bytes a context needs for one Gibbs chain of n points with these
 * options (its plan, scratch, H-matrices, factors, vectors and trace): an
 * arena of this size holds exactly fifa_chain_create's allocations.
 * Synchronizes nothing.  Errors: INVALID_ARG, UNSUPPORTED (as fifa_create). */
fifa_status fifa_chain_bytes(const fifa_opts* opts, int64_t n, size_t* bytes_out);

/* Additive model of d one-dimensional GP blocks (Sec. 4.2 allows an additive
 * model instead of the tensor-product kernel for d-dimensional inputs):
 *   y = sum_k f_k(x_k) + e,  e ~ N(0, sigma2 I),  f_k ~ GP(0, tau2_k C(rho_k)).
 * X_dev: d columns of n doubles, coordinate k of point i at X_dev[k n + i],
 * points in any order; y_dev: n doubles.  Each block stably sorts its
 * coordinate at creation (ties keep the lower point index first) and keeps a
 * chain on the sorted coordinate.  init gives the kernel, nugget, and the
 * starting rho and tau2 of every block and the shared sigma2.  Block k draws
 * from Philox stream id k, the shared sigma2 from stream id d.  The caller's
 * buffers are copied; they may be freed after the call (synchronizes).
 * Errors: INVALID_ARG (d outside 1..FIFA_ADDITIVE_MAX_D, non-finite x),
 * OOM, and those of fifa_chain_create. */
typedef struct fifa_additive fifa_additive;
#define FIFA_ADDITIVE_MAX_D 16
fifa_status fifa_additive_create(fifa_ctx* ctx, const double* X_dev, const double* y_dev, int64_t n, int d,
                                 const fifa_hyper* init, const fifa_prior* prior, uint64_t seed,
                                 fifa_additive** out);

/* Run `sweeps` block-Gibbs sweeps: for k = 0..d-1, f_k by Algorithm 1 on the
 * partial residual y - sum_{j != k} f_j (subtracted in ascending j, sorted by
 * x_k); then sigma2 | y, f_1..f_d; then for each k, tau2_k | f_k and the
 * Metropolis step on log rho_k.  One sweep is captured in a CUDA graph.
 * trace_host (nullable): sweeps rows of FIFA_ADDITIVE_TRACE_FIELDS(d) doubles:
 * sweep, sigma2, ||y - sum_k f_k||^2, status, largest refinement residual of the
 * blocks' M~ solves, tau2[d], rho[d], accepted[d].
 * Errors: the blocks' device status (NOT_SPD, TIMEOUT). */
#define FIFA_ADDITIVE_TRACE_FIELDS(d) (5 + 3 * (d))
fifa_status fifa_additive_sweep(fifa_ctx* ctx, fifa_additive* model, int sweeps, double* trace_host);

/* Current state (synchronizes): F_dev (nullable) receives f_1..f_d as d
 * columns of n doubles in the original point order; sigma2_host (nullable);
 * blocks_host (nullable) d entries with each block's tau2 and rho (sigma2
 * the shared value). */
fifa_status fifa_additive_get(fifa_ctx* ctx, const fifa_additive* model, double* F_dev, double* sigma2_host,
                              fifa_hyper* blocks_host);

/* Kernel nodes of the captured sweep graph, or -1 without a graph. */
fifa_status fifa_additive_kernel_nodes(const fifa_additive* model, int* out_host);

void fifa_destroy_additive(fifa_ctx* ctx, fifa_additive* model);

/* Tensor product of d one-dimensional GPs (Sec. 4.2, Eq. tensor_prod):
 *   y_i = beta f_1(x_{1,i}) ... f_d(x_{d,i}) + e_i,  e_i ~ N(0, sigma2),
 *   f_h ~ GP(1, C(rho_h)) (unit variance, prior mean 1), beta ~ N(beta_mu, beta_sd^2).
 * X_dev: d columns of n doubles (coordinate h of point i at X_dev[h n + i]),
 * any order; y_dev: n doubles (copied; both may be freed after the call).
 * init: kernel, nugget, starting rho of every block and sigma2 (init->tau2 is
 * not used: the blocks have unit variance); prior: IG on sigma2, normal prior
 * and random-walk step on every log rho_h.  Every f_h starts at 1, beta at
 * beta0.  Block h draws from Philox stream id h, sigma2 from d, beta from d + 1.
 * Errors: INVALID_ARG (d outside 1..FIFA_ADDITIVE_MAX_D, non-finite x, beta_sd
 * <= 0), OOM, those of fifa_chain_create. */
typedef struct fifa_tensor fifa_tensor;
fifa_status fifa_tensor_create(fifa_ctx* ctx, const double* X_dev, const double* y_dev, int64_t n, int d,
                               const fifa_hyper* init, const fifa_prior* prior, double beta0, double beta_mu,
                               double beta_sd, uint64_t seed, fifa_tensor** out);

/* Run `sweeps` sweeps: for h = 0..d-1, f_h - 1 by Algorithm 1.h on the sorted
 * x_h with data y / g - 1 and precisions g^2 / sigma2, g = beta prod_{k != h} f_k
 * (the block's P~ = C~ + D^-1 refactored each sweep); beta | y, F (its normal
 * conditional); sigma2 | y, F, beta; then the Metropolis step on every log
 * rho_h with tau2 = 1.  One sweep is captured in a CUDA graph.  trace_host
 * (nullable): sweeps rows of FIFA_TENSOR_TRACE_FIELDS(d) doubles: sweep, beta,
 * sigma2, ||y - beta prod_h f_h||^2, status, rho[d], accepted[d].
 * Errors: INVALID_ARG (a zero product g_i: no information on f_h), the blocks'
 * device status (NOT_SPD, TIMEOUT). */
#define FIFA_TENSOR_TRACE_FIELDS(d) (5 + 2 * (d))
fifa_status fifa_tensor_sweep(fifa_ctx* ctx, fifa_tensor* model, int sweeps, double* trace_host);

/* Current state (synchronizes): F_dev (nullable) receives f_1..f_d as d columns
 * of n doubles in the original point order; beta_host, sigma2_host (nullable);
 * blocks_host (nullable): d entries with each block's rho. */
fifa_status fifa_tensor_get(fifa_ctx* ctx, const fifa_tensor* model, double* F_dev, double* beta_host,
                            double* sigma2_host, fifa_hyper* blocks_host);
void fifa_destroy_tensor(fifa_ctx* ctx, fifa_tensor* model);

/* Serving: independent 1-D GP regression requests (each a Gibbs chain on its
 * own sorted inputs) with continuous batching on the current GPU.  The server
 * allocates hbm_budget device bytes once and runs `slots` workers, each a host
 * thread with its own CUDA stream.  A queued request is admitted, oldest first
 * among those a worker may run, when that worker is idle and the budget can
 * hold its chain (fifa_chain_bytes plus its input and result buffers);
 * admitted requests run concurrently and their kernels overlap on the GPU.
 * Narrow workers use independent CTAs (opts.independent_ctas forced to 1).
 * With wide_min_n > 0, the wide workers run the requests with n >= wide_min_n,
 * with CTA groups and fused sweeps (the only streams whose kernels' CTAs wait
 * on each other), each sized to 1 / wide_workers of the CTAs the GPU holds at
 * once, so the wide workers' waiting launches always fit on the GPU together.
 * A request's worker type depends only on its n, and every wide worker uses
 * the same sizes, so its result does not depend on what else is in flight.
 * The workers' streams overlap only as far as the process's hardware work
 * queues allow: CUDA_DEVICE_MAX_CONNECTIONS (default 8, read when the process
 * creates its CUDA context) should be at least `slots`.  This API has no
 * counterpart in the paper; it serves its sampler to many users. */
typedef struct fifa_server fifa_server;
typedef struct {
  fifa_opts opts;     /* leaf size, ACA tolerance, rank cap, precision of every request */
  size_t hbm_budget;  /* device bytes reserved once for all requests in flight */
  int slots;          /* requests in flight at once, 1..256 */
  int64_t wide_min_n; /* 0: all workers narrow; > 0: the first wide_workers workers are wide */
  int wide_workers;   /* wide workers when wide_min_n > 0 (0 means 1; < slots): each sizes its
                         grouped launches to 1 / wide_workers of the GPU (coresident_share) */
} fifa_server_opts;

typedef struct {
  const double* x_host;  /* n inputs, sorted ascending (copied at submit) */
  const double* y_host;  /* n observations (copied at submit) */
  int64_t n;
  fifa_hyper init;       /* kernel, nugget, starting tau2, rho, sigma2 */
  fifa_prior prior;
  uint64_t seed, chain_id;  /* Philox key and stream id of the chain */
  int iters;             /* Gibbs iterations (Eqs. posterior_gibs1-4 and the Metropolis step) */
  int burn;              /* iterations left out of the returned estimates, 0 <= burn < iters */
  int ndraws;            /* draws of f returned, 0 <= ndraws <= iters - burn */
} fifa_request;

typedef struct {
  int status;                         /* fifa_status of the request */
  double t_submit, t_start, t_done;   /* seconds on the server's monotonic clock */
  fifa_hyper last;                    /* hyperparameters after the last iteration */
  double accept_rate;                 /* accepted Metropolis proposals / iters */
  size_t bytes;                       /* device bytes the request held while running */
} fifa_result;

typedef struct {
  double now;               /* seconds on the server's clock */
  int queued, in_flight, peak_in_flight;
  size_t bytes_in_use, peak_bytes;
  uint64_t completed, iterations_done;
} fifa_server_counters;

/* Errors: INVALID_ARG (slots outside 1..256, budget below 16 MiB, bad opts),
 * UNSUPPORTED, OOM (the budget cannot be allocated). */
fifa_status fifa_server_create(const fifa_server_opts* opts, fifa_server** out);

/* Queue a request; returns at once with its id.  The result (posterior mean =
 * average over iterations [burn, iters) of the conditional means tau2 C~ r,
 * and f at iterations burn + floor((j + 1)(iters - burn) / ndraws) - 1) is
 * kept until fifa_server_wait collects it.  Errors: INVALID_ARG (sizes,
 * non-finite data), UNSORTED, OOM (one request larger than the budget). */
fifa_status fifa_server_submit(fifa_server* server, const fifa_request* req, uint64_t* id_out);

/* Block until request `id` is done; copy its posterior mean (n doubles) and
 * draws (ndraws x n) to host buffers (nullable) and its timing to res
 * (nullable); then forget the request.  Returns the request's status
 * (INVALID_ARG for an unknown id). */
fifa_status fifa_server_wait(fifa_server* server, uint64_t id, double* mean_host, double* draws_host,
                             fifa_result* res);

/* Non-blocking: *done_out = 1 if request `id` has finished (fifa_server_wait
 * then returns at once), else 0.  INVALID_ARG for an unknown or collected id. */
fifa_status fifa_server_poll(fifa_server* server, uint64_t id, int* done_out);

fifa_status fifa_server_stats(fifa_server* server, fifa_server_counters* out);

/* Finish the requests in flight, drop the queued ones, free the budget.  Call
 * it after every fifa_server_wait has returned. */
void fifa_server_destroy(fifa_server* server);

/* Introspection for tests and tools (synchronize).  Layouts:
 *   ranks[node], node = 2^l - 1 + i for node i of level l (2^L - 1 nodes);
 *   row_piv / col_piv [node * rank_cap + k] (block-local indices, -1 unused);
 *   bases[(l * rank_cap + k) * n + p]: column k of the level-l basis at global
 *     row p (U of the node for rows in its left child, V for its right child);
 *   leaves[(leaf * Bm + b) * Bm + a] = C~ leaf entry (a, b), Bm = max leaf size. */
fifa_status fifa_hmat_dims(const fifa_hmat* H, int64_t* n, int* levels, int* nleaf, int* leaf_max,
                           int* rank_cap);
/* The plan the library builds for n points (host only: no GPU needed), given
 * the co-resident CTA budgets it queries on a GPU: aca_cores for the ACA
 * kernel, lvl_cores[3] for the level kernel's rank buckets (<= 4, 5..16,
 * > 16).  Optional outputs: bounds_out, the tree bounds with level l at offset
 * 2^l - 1 + l (2^(L+1) + L ints; node i of level l spans
 * [b[l][i], b[l][i + 1]) with its split at b[l + 1][2 i + 1]); aca_work_out,
 * 4 ints per entry {level, node, g, G}: the grouped entries (G CTAs per
 * block), then one CTA per block, then one warp per block; lvl_groups_out,
 * the CTA group size per rank bucket and level (3 x L ints, bucket-major).
 * Call with null outputs first to size them.  Errors: INVALID_ARG,
 * UNSUPPORTED (more levels than the library supports), OOM. */
typedef struct {
  int levels, nleaf, leaf_max;
  int aca_grouped_ctas, aca_solo_blocks, aca_warp_blocks;
  int64_t scratch_bytes;
} fifa_plan_info;
fifa_status fifa_plan_describe(const fifa_opts* opts, int64_t n, int aca_cores, const int* lvl_cores,
                               fifa_plan_info* info, int* bounds_out, int* aca_work_out, int* lvl_groups_out);

/* Rows [row0, row0 + nrows) of the level-l bases only (for sampled checks of
 * large problems): out_host[k * nrows + (p - row0)] = bases[(l * rank_cap + k)
 * * n + p], k < rank_cap.  Errors: INVALID_ARG (level or row range outside
 * the H-matrix). */
fifa_status fifa_hmat_level_rows(fifa_ctx* ctx, const fifa_hmat* H, int level, int64_t row0, int64_t nrows,
                                 double* out_host);
fifa_status fifa_hmat_export(fifa_ctx* ctx, const fifa_hmat* H, int* ranks_host, int* row_piv_host,
                             int* col_piv_host, double* bases_host, double* leaves_host);
/* Factor pieces in the same layouts: bases are the orthonormal Q_U / Q_V,
 * leaves the lower Cholesky factors (as double even for FP32 factors),
 * Zf / Zi [node * (2 cap)^2 + a * 2cap + b] = (L_S - I) and (L_S^-1 - I). */
fifa_status fifa_fact_export(fifa_ctx* ctx, const fifa_fact* F, double* bases_host, double* leaves_host,
                             double* Zf_host, double* Zi_host);

void fifa_destroy_hmat(fifa_ctx* ctx, fifa_hmat* H);
void fifa_destroy_fact(fifa_ctx* ctx, fifa_fact* F);
void fifa_destroy_chain(fifa_ctx* ctx, fifa_chain* chain);

const char* fifa_status_str(fifa_status s);

/* Text of the last CUDA runtime error a call on this context met (for
 * FIFA_ERR_CUDA), or "no error". */
const char* fifa_last_cuda_error(const fifa_ctx* ctx);

/* Deterministic exponential used for every kernel entry (same operation
 * sequence as the CPU reference, so ACA pivots agree bit for bit):
 * out[i] = det_exp(in[i]) for n device doubles.  Exposed for parity tests. */
fifa_status fifa_det_exp(fifa_ctx* ctx, const double* in_dev, double* out_dev, int64_t n);

/* Philox4x32-10 normals of stream (seed, tag, iter, stream_id), n values. */
fifa_status fifa_normals(fifa_ctx* ctx, uint64_t seed, uint32_t tag, uint64_t iter, uint64_t stream_id,
                         double* out_dev, int64_t n);

/* Raw Philox4x32-10 words: out[4i..4i+3] = Philox(ctr[4i..4i+3], key = seed),
 * for `count` counters (device uint32 arrays).  Exposed for parity tests. */
fifa_status fifa_philox(fifa_ctx* ctx, uint64_t seed, const uint32_t* ctr_dev, uint32_t* out_dev, int64_t count);

/* Measurement only (not part of the method): FP64 fused multiply-add
 * throughput of this GPU, the roofline denominator of the FP64-issue-bound
 * kernels.  Runs 8 independent FMA chains of `iters` steps in every thread of
 * 8 CTAs x 256 threads per SM, timed with CUDA events on the context's stream
 * (synchronizes): tflops_host = 16 iters threads / time; ms_host (nullable) the
 * kernel time.  Errors: INVALID_ARG, CUDA. */
fifa_status fifa_probe_fp64_fma(fifa_ctx* ctx, int iters, double* tflops_host, double* ms_host);

#ifdef __cplusplus
}
#endif
#endif /* FIFA_H */
