// Shared device definitions of the FIFA-GP GB300 library.
//
// Data layout in HBM (one HODLR matrix C~ for n sorted points, leaf size B,
// L levels, rank cap R):
//   bnd      int32   tree bounds; level l occupies bnd[2^l - 1 + l .. 2^(l+1) - 1 + l],
//                    node i of level l is [bnd[off(l)+i], bnd[off(l)+i+1])
//   leaves   f64     nleaf x Bm x Bm, column-major per leaf (Bm = max leaf size)
//   bases    f64     L x R x n: column k of level l at bases[(l*R + k)*n + p]; row p
//                    holds U of the level-l node containing p when p lies in the
//                    node's left child and V when it lies in the right child, so a
//                    level's bases tile all n rows and every access is a
//                    contiguous, coalesced column segment.
//   rank     int32   per node (heap order: node i of level l is 2^l - 1 + i)
// A factor stores the same shapes (leaves -> lower Cholesky factors, bases ->
// orthonormal Q_U / Q_V) in f64 or f32, plus per node the (2R)^2 matrices
// Zf = L_S - I and Zi = L_S^-1 - I in f64.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define FIFA_CAP_MAX 64
#define FIFA_LEAF_MAX 128
#define FIFA_LEVELS_MAX 26
#define FIFA_SPIN_LIMIT (1u << 26)

// Status bits written by device code (OR-ed into a status word).
#define FIFA_DEV_NOT_SPD 1
#define FIFA_DEV_RANK_CAP 2
#define FIFA_DEV_TIMEOUT 4

struct HmatDesc {
  int64_t n;
  int L, nleaf, Bm, cap, kind;
  const int* bnd;
  const double* x;
  double* leaves;
  double* bases;
  int* rank;
  int* row_piv;
  int* col_piv;
  int* status;
  double kc;      // kernel constant (0.5/rho^2 or sqrt(5)/rho)
  double rho;
  double nugget;
  double eps;
  double scale;   // view: A = scale * C~ + shift * I (U scaled by `scale`)
  double shift;
  const double* diag;  // nullable: per-row diagonal, A = scale * C~ + diag(diag) (replaces shift)
  unsigned int spin;   // polls before a group wait gives up (0: FIFA_SPIN_LIMIT)
};

struct FactDesc {
  int64_t n;
  int L, nleaf, Bm, cap, prec;  // prec: 0 = f64 storage, 1 = f32 storage (a rounded copy of an FP64
                                // factor, applied in FP32 arithmetic; Zf, Zi and the rest shared with it)
  const int* bnd;
  void* Lleaf;                  // nleaf x Bm x Bm Cholesky factors L, L^T mirrored into the upper triangle
  void* Ldinv;                  // nleaf x Bm reciprocals of their diagonals (storage precision)
  void* Q;                      // L x cap x n orthonormal bases
  double* Zf;                   // nnodes x (2cap)^2 : L_S - I
  double* Zi;                   // nnodes x (2cap)^2 : L_S^-1 - I
  double* Rw;                   // nnodes x 2 x cap^2 workspace (upper R of each side)
  int* rank;                    // nnodes
  double* ld_parts;             // nleaf + nnodes partial log-determinants
  double* logdet;               // [1]
  int* status;                  // [1]
  const int* skip;              // nullable: while *skip != 0 the factorization kernels leave this
                                // factor as it is (a factor kept from an earlier iteration)
  unsigned int spin;            // polls before a group wait gives up (0: FIFA_SPIN_LIMIT)
};

__host__ __device__ inline int bnd_off(int l) { return (1 << l) - 1 + l; }
__host__ __device__ inline int node_id(int l, int i) { return (1 << l) - 1 + i; }

__device__ __forceinline__ void node_range(const int* bnd, int l, int i, int& s, int& h, int& e) {
  s = bnd[bnd_off(l) + i];
  e = bnd[bnd_off(l) + i + 1];
  h = s + (e - s) / 2;
}

// Index of the level-l node that contains row p (binary search over bounds).
__device__ __forceinline__ int node_of_row(const int* bnd, int l, int p) {
  const int* b = bnd + bnd_off(l);
  int lo = 0, hi = 1 << l;  // b[lo] <= p < b[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (b[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Deterministic exponential (Cody-Waite reduction + degree-13 Taylor/Horner,
// plain IEEE binary64 products and sums, never fused), the same operation
// sequence as the CPU reference so kernel entries agree bit for bit.
//   LN2_HI: ln 2 rounded to binary64 then truncated to 32 significand bits
//   LN2_LO: (ln 2 - LN2_HI) rounded to binary64;  INV_LN2: 1/ln 2 rounded.
// ---------------------------------------------------------------------------
// 2^(j/32), j = 0..31, correctly rounded (Tang's table-driven exponential).
static __device__ const double kExp2Tab[32] = {
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0,
    0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, 0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0,
    0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0,
    0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, 0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0,
    0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0,
    0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, 0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0};

// Deterministic e^x: x = (32 m + j) ln2/32 + r, k = rint(32 x / ln2) (ln2/32
// split as HI + LO), r = fma(-k, LO, fma(-k, HI, x)), e^x = 2^m 2^(j/32) (1 + q)
// with p = 1 + r/2 + ... + r^5/6! by Horner's rule (one fused multiply-add
// per step) and q = p r, returned as fma(t, q, t) with t = 2^(j/32) 2^m built
// exactly.  Every operation is an explicitly rounded IEEE product or fused
// multiply-add (none left to the compiler to contract), the same sequence as
// the CPU reference; x < -708 -> 0.  11 FP64 operations.
__device__ __forceinline__ double det_exp(double x) {
  if (!(x >= -708.0)) return x != x ? x : 0.0;
  const double INV_LN2N = 0x1.71547652b82fep+5;
  const double LN2N_HI = 0x1.62e42fee00000p-6;
  const double LN2N_LO = 0x1.a39ef35793c76p-38;
  const double k = rint(__dmul_rn(x, INV_LN2N));
  const double r = __fma_rn(-k, LN2N_LO, __fma_rn(-k, LN2N_HI, x));
  double p = 1.0 / 720.0;
  p = __fma_rn(p, r, 1.0 / 120.0);
  p = __fma_rn(p, r, 1.0 / 24.0);
  p = __fma_rn(p, r, 1.0 / 6.0);
  p = __fma_rn(p, r, 0.5);
  p = __fma_rn(p, r, 1.0);
  const double q = __dmul_rn(p, r);
  const long long ki = (long long)k;
  const unsigned long long tb = (unsigned long long)__double_as_longlong(__ldg(&kExp2Tab[ki & 31])) +
                                ((unsigned long long)(ki >> 5) << 52);
  const double t = __longlong_as_double((long long)tb);
  return __fma_rn(t, q, t);
}

// Unit-variance kernel entry k(xa, xb), bit-identical to the CPU reference:
// SE det_exp(-((d d) c)); Matern-5/2 fma(t t, 1/3, 1 + t) det_exp(-t), t = |d| c.
__device__ __forceinline__ double kern_entry(int kind, double kc, double xa, double xb) {
  double d = __dsub_rn(xa, xb);
  if (kind == 0) return det_exp(-__dmul_rn(__dmul_rn(d, d), kc));
  double t = __dmul_rn(fabs(d), kc);
  double poly = __fma_rn(__dmul_rn(t, t), 1.0 / 3.0, __dadd_rn(1.0, t));
  return __dmul_rn(poly, det_exp(-t));
}

// ---------------------------------------------------------------------------
// Block-wide helpers (blockDim.x a multiple of 32, <= 1024).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum: result valid in every thread. `sh` >= 32 doubles.
__device__ inline double block_sum(double v, double* sh) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  double r = sh[32];
  __syncthreads();
  return r;
}

// (value, index) argmax with ties to the lowest index; value -1 = none.
// Values are absolute values (>= 0, never NaN) or exactly -1, so their IEEE
// bit patterns read as signed 64-bit integers order the same way: the
// comparisons run on the integer pipe, not the FP64 one.
struct ArgMax {
  double v;
  int i;
  double sv;  // signed value carried along
};
__device__ __forceinline__ bool am_wins(const ArgMax& a, const ArgMax& b) {  // b beats a
  const long long av = __double_as_longlong(a.v), bv = __double_as_longlong(b.v);
  return bv > av || (bv == av && b.i < a.i);
}
__device__ __forceinline__ ArgMax am_better(ArgMax a, ArgMax b) { return am_wins(a, b) ? b : a; }
// max of two values >= 0 or -1 (same ordering argument)
__device__ __forceinline__ double nn_max(double a, double b) {
  return __double_as_longlong(b) > __double_as_longlong(a) ? b : a;
}
__device__ __forceinline__ ArgMax warp_argmax(ArgMax a) {
  for (int o = 16; o > 0; o >>= 1) {
    ArgMax b;
    b.v = __shfl_down_sync(0xffffffffu, a.v, o);
    b.i = __shfl_down_sync(0xffffffffu, a.i, o);
    b.sv = __shfl_down_sync(0xffffffffu, a.sv, o);
    a = am_better(a, b);
  }
  return a;
}
// Block argmax; result valid in every thread. `sh` >= 33 ArgMax slots.
__device__ inline ArgMax block_argmax(ArgMax a, ArgMax* sh) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_argmax(a);
  __syncthreads();
  if (lane == 0) sh[w] = a;
  __syncthreads();
  if (w == 0) {
    ArgMax t = lane < nw ? sh[lane] : ArgMax{-1.0, 0x7fffffff, 0.0};
    t = warp_argmax(t);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  ArgMax r = sh[32];
  __syncthreads();
  return r;
}
// Block max of values >= 0 (or -1); result valid in every thread.
__device__ __forceinline__ double block_max(double v, double* sh) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = nn_max(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? sh[lane] : -1.0;
    for (int o = 16; o > 0; o >>= 1) t = nn_max(t, __shfl_down_sync(0xffffffffu, t, o));
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  double r = sh[32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Small dense routines run by a whole block on row-major matrices with
// leading dimension ld (shared or global memory).
// ---------------------------------------------------------------------------
// In place: A (r x r, symmetric, upper triangle read) -> upper R with A = R^T R.
// Lower triangle is zeroed.  Returns false (in every thread) on a non-positive
// pivot.  clamp > 0: a pivot below clamp * (largest diagonal entry) is raised to
// that value instead (modified Cholesky: the result factors a nearby SPD
// matrix; used for factors that only precondition an FP64 iteration).
// Reciprocal pivots of the last blk_chol_upper call in this CTA (r <= 2 FIFA_CAP_MAX).
__device__ inline double* blk_chol_rinv() {
  __shared__ double rinv[2 * FIFA_CAP_MAX];
  return rinv;
}

__device__ inline bool blk_chol_upper(double* A, int ld, int r, int* flag, double clamp = 0.0) {
  __shared__ double chol_floor;
  double* rinv = blk_chol_rinv();
  if (threadIdx.x == 0) {
    *flag = 0;
    double dmax = 0.0;
    for (int k = 0; k < r; ++k) dmax = fmax(dmax, A[k * ld + k]);
    chol_floor = clamp * dmax;
  }
  __syncthreads();
  const double floor_v = chol_floor;
  for (int k = 0; k < r; ++k) {
    if (threadIdx.x == 0) {
      double d = A[k * ld + k];
      if (clamp > 0.0 && !(d > floor_v)) d = floor_v > 0.0 ? floor_v : 1.0;
      if (!(d > 0.0)) { *flag = 1; d = 1.0; }
      const double rs = rsqrt(d);  // one reciprocal square root gives the pivot and its reciprocal
      A[k * ld + k] = d * rs;
      rinv[k] = rs;
    }
    __syncthreads();
    const double dinv = rinv[k];
    for (int j = k + 1 + threadIdx.x; j < r; j += blockDim.x) A[k * ld + j] *= dinv;
    __syncthreads();
    int m = r - k - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      int i = k + 1 + t / m, j = k + 1 + t % m;
      if (j >= i) A[i * ld + j] -= A[k * ld + i] * A[k * ld + j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
    int i = t / r, j = t % r;
    if (j < i) A[i * ld + j] = 0.0;
  }
  __syncthreads();
  return *flag == 0;
}

// Rinv = R^-1 for upper-triangular R (r x r); one thread per column.  R must
// be the factor of the CTA's last blk_chol_upper call (its reciprocal pivots
// replace the divisions).
__device__ inline void blk_triinv_upper(const double* R, int ldr, double* Ri, int ldi, int r) {
  const double* rinv = blk_chol_rinv();
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    for (int i = r - 1; i >= 0; --i) {
      double acc = (i == j) ? 1.0 : 0.0;
      for (int k = i + 1; k <= j; ++k) acc -= R[i * ldr + k] * Ri[k * ldi + j];
      Ri[i * ldi + j] = (i <= j) ? acc * rinv[i] : 0.0;
    }
  }
  __syncthreads();
}

// Li = L^-1 for lower-triangular L (r x r); one thread per column.
__device__ inline void blk_triinv_lower(const double* Lm, int ldl, double* Li, int ldi, int r) {
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    for (int i = 0; i < r; ++i) {
      double acc = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) acc -= Lm[i * ldl + k] * Li[k * ldi + j];
      Li[i * ldi + j] = (i >= j) ? acc / Lm[i * ldl + i] : 0.0;
    }
  }
  __syncthreads();
}

template <typename T> __device__ __forceinline__ double to_d(T v) { return (double)v; }

// Bounded spin barrier among the G blocks of one group (counter monotone).
// Returns false (in every thread) if the wait gave up; *err then has the
// TIMEOUT bit set.
__device__ inline bool group_barrier(unsigned int* counter, unsigned int target, int* err,
                                     volatile int* abort_flag, unsigned int limit) {
  if (limit == 0) limit = FIFA_SPIN_LIMIT;
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1u);
    unsigned int spins = 0;
    ok = 1;
    while (true) {
      unsigned int v = *((volatile unsigned int*)counter);
      if (v >= target) break;
      if (*abort_flag) { ok = 0; break; }
      if (++spins > limit) {
        atomicOr(err, FIFA_DEV_TIMEOUT);
        *abort_flag = 1;
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}
