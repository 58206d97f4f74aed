// Symmetric factorization A = W W^T, W = A_L A_{L-1} ... A_0, of a HODLR matrix
// (SI "HODLR decomposition and factorization", after Ambikasaran et al. 2014,
// Theorem 3.1) and its log-determinant (SI "Determinant computation speedup").
//
//  k_leaf_factor : per leaf, L_i = chol(scale * D_i + shift * I) in FP64 shared
//                  memory, log-det partial, and L_i^-1 applied to the rows of
//                  every ancestor basis lying in the leaf (the first transform),
//                  the first chunk of those columns inside the Cholesky steps.
//  k_level       : per node of one level (bottom-up), the orthonormal bases
//                  Q_U, Q_V of the transformed U~, V~ by CholeskyQR2 (two Gram
//                  passes; stable here because the column-scaled bases are
//                  well conditioned), R = R2 R1, L_S = chol(I + R X R^T),
//                  Zf = L_S - I, Zi = L_S^-1 - I, and the inverse node factor
//                  I + Q Zi Q^T applied to every ancestor basis on the node's rows.
//                  Large nodes: G CTAs split the rows and exchange partial sums
//                  through bounded-spin group barriers.
//  k_level_multi : the same for the deepest levels (sides of <= 128 rows,
//                  rank <= 4), several nodes per CTA staged in shared memory;
//  k_level_small : rank 5..8 nodes of those levels, one CTA each.
#include <algorithm>
#include <atomic>
#include "fifa_common.cuh"
#include "fifa_launch.h"

// Ancestor columns per right-hand-side chunk of the leaf TRSM: the first chunk
// is eliminated together with the Cholesky steps, later chunks (more ancestor
// columns than this) by a separate triangular solve.
__host__ __device__ inline int lf_nch(int Bm) { return Bm <= 64 ? 64 : 32; }

template <typename T>
__global__ void __launch_bounds__(256, 7) k_leaf_factor(const HmatDesc* __restrict__ Hd, const FactDesc* __restrict__ Fd) {
  extern __shared__ double sm[];
  Hd += blockIdx.y;  // problem of a batched launch (descriptor arrays)
  Fd += blockIdx.y;
  if (Fd->skip && *Fd->skip) return;  // this factor is kept as it is
  const int leaf = blockIdx.x;
  const int L = Fd->L, Bm = Fd->Bm, cap = Fd->cap;
  const int64_t n = Fd->n;
  const double sc = Hd->scale, shf = Hd->shift;
  const int* bnd = Fd->bnd;
  const int s = bnd[bnd_off(L) + leaf], e = bnd[bnd_off(L) + leaf + 1], m = e - s;
  const int ld = Bm + 1, NCH = lf_nch(Bm);
  double* A = sm;                          // FP64 Cholesky, column-major A[j*ld + i]
  T* La = sizeof(T) == sizeof(double) ? (T*)A : (T*)(A + (size_t)Bm * ld);  // L in the TRSM precision
  T* X = (T*)(A + (size_t)Bm * ld + (sizeof(T) == sizeof(double) ? 0 : ((size_t)Bm * ld + 1) / 2));
  double* red = (double*)(X + (size_t)NCH * ld) + 1;  // 40 doubles (8-byte aligned past X)
  red = (double*)(((uintptr_t)red) & ~(uintptr_t)7);
  int* flag = (int*)(red + 40);
  int* clist = flag + 4;                   // L * cap entries: (level << 8) | col
  const double* D = Hd->leaves + (size_t)leaf * Bm * Bm;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t % m, j = t / m;
    double v = __dmul_rn(sc, D[(size_t)j * Bm + i]);
    if (i == j) v = __dadd_rn(v, Hd->diag ? Hd->diag[s + i] : shf);
    A[j * ld + i] = v;
  }
  // column list of all ancestor bases restricted to this leaf: the level-l
  // ancestor of leaf i is node i >> (L - l); the leaf lies in its left child
  // (U rows, scaled in a view) when bit L - l - 1 of i is clear
  __shared__ int ncols;
  __shared__ int rkl[FIFA_LEVELS_MAX];
  __shared__ double lscale[FIFA_LEVELS_MAX];
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    rkl[l] = Hd->rank[node_id(l, leaf >> (L - l))];
    lscale[l] = ((leaf >> (L - l - 1)) & 1) ? 1.0 : sc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    for (int l = 0; l < L; ++l)
      for (int q = 0; q < rkl[l]; ++q) clist[c++] = (l << 8) | q;
    ncols = c;
  }
  __syncthreads();
  const int nc = ncols;
  T* Q = (T*)Fd->Q;
  auto load_chunk = [&](int c0, int w) {
    for (int t = threadIdx.x; t < w * m; t += blockDim.x) {
      int cc = t / m, i = t % m;
      int code = clist[c0 + cc], l = code >> 8, q = code & 255;
      const double scl = lscale[l];
      double v = Hd->bases[((size_t)l * cap + q) * n + s + i];
      X[cc * ld + i] = (T)((scl == 1.0) ? v : __dmul_rn(scl, v));
    }
  };
  auto store_chunk = [&](int c0, int w) {
    for (int t = threadIdx.x; t < w * m; t += blockDim.x) {
      int cc = t / m, i = t % m;
      int code = clist[c0 + cc], l = code >> 8, q = code & 255;
      Q[((size_t)l * cap + q) * n + s + i] = X[cc * ld + i];
    }
  };
  const int w0 = min(NCH, nc);
  load_chunk(0, w0);
  // reciprocals of the pivots: one reciprocal square root per column, products elsewhere
  __shared__ double rinv[FIFA_LEAF_MAX];
  auto pivot = [&](int k) {  // by one thread
    double d = A[k * ld + k];
    if (!(d > 0.0)) { flag[0] = 1; d = 1.0; }
    const double rs = rsqrt(d);
    A[k * ld + k] = d * rs;
    rinv[k] = rs;
  };
  if (threadIdx.x == 0) flag[0] = 0;
  // column k ready for its step: pivot, column k of L and row k of X scaled
  // (warp 0 alone)
  auto prep_column = [&](int k) {
    const int lane = threadIdx.x;
    if (lane == 0) pivot(k);
    __syncwarp();
    const double dinv = rinv[k];
    for (int i = k + 1 + lane; i < m; i += 32) A[k * ld + i] *= dinv;
    for (int cc = lane; cc < w0; cc += 32) X[cc * ld + k] *= (T)dinv;
  };
  __syncthreads();  // the first chunk of X is loaded
  if (threadIdx.x < 32 && m > 0) prep_column(0);
  __syncthreads();
  // right-looking Cholesky with the first chunk of right-hand sides eliminated
  // in the same steps (L^-1 X), one barrier per column: in step k warp 0
  // updates column k + 1 and row k + 1 of X first and prepares column k + 1
  // (pivot and scaling) for the next step, while the other warps update the
  // rest of the trailing triangle and of X
  for (int k = 0; k < m; ++k) {
    const int w = m - k - 1;
    if (threadIdx.x < 32) {
      if (w > 0) {
        const int lane = threadIdx.x;
        const double lk1 = A[k * ld + k + 1];  // L[k+1][k]
        for (int i = k + 1 + lane; i < m; i += 32) A[(k + 1) * ld + i] -= A[k * ld + i] * lk1;
        for (int cc = lane; cc < w0; cc += 32) X[cc * ld + k + 1] -= (T)lk1 * X[cc * ld + k];
        __syncwarp();
        prep_column(k + 1);
      }
    } else {
      const int t0 = threadIdx.x - 32, nt2 = blockDim.x - 32, w1 = w - 1;
      // trailing triangle beyond column k + 1: t -> (a, b), b <= a, t = a(a+1)/2 + b
      for (int t = t0; t < w1 * (w1 + 1) / 2; t += nt2) {
        int a = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        if ((a + 1) * (a + 2) / 2 <= t) ++a;
        if (a * (a + 1) / 2 > t) --a;
        const int b = t - a * (a + 1) / 2;
        const int i = k + 2 + a, j = k + 2 + b;
        A[j * ld + i] -= A[k * ld + i] * A[k * ld + j];
      }
      for (int t = t0; t < w1 * w0; t += nt2) {
        const int cc = t / w1, i = k + 2 + t % w1;
        X[cc * ld + i] -= (T)A[k * ld + i] * X[cc * ld + k];
      }
    }
    __syncthreads();
  }
  double lsum = 0.0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) lsum += log(A[k * ld + k]);
  lsum = block_sum(lsum, red);
  if (threadIdx.x == 0) {
    Fd->ld_parts[leaf] = lsum;
    if (flag[0]) atomicOr(Fd->status, FIFA_DEV_NOT_SPD);
  }
  for (int k = threadIdx.x; k < m; k += blockDim.x) ((double*)Fd->Ldinv)[(size_t)leaf * Bm + k] = rinv[k];
  T* Lout = (T*)Fd->Lleaf + (size_t)leaf * Bm * Bm;
  for (int t = threadIdx.x; t < Bm * Bm; t += blockDim.x) {
    int i = t % Bm, j = t / Bm;
    // L in the lower triangle, L^T mirrored into the upper one (transposed
    // solves then read contiguous columns as well)
    double v = (i < m && j < m) ? (i >= j ? A[j * ld + i] : A[i * ld + j]) : 0.0;
    Lout[t] = (T)v;
  }
  store_chunk(0, w0);
  if (nc <= w0) return;
  if (sizeof(T) != sizeof(double)) {
    for (int t = threadIdx.x; t < m * ld; t += blockDim.x) La[t] = (T)A[t];
  }
  __syncthreads();
  // further chunks: forward substitution with the finished factor
  for (int c0 = w0; c0 < nc; c0 += NCH) {
    const int w = min(NCH, nc - c0);
    load_chunk(c0, w);
    __syncthreads();
    for (int k = 0; k < m; ++k) {
      for (int cc = threadIdx.x; cc < w; cc += blockDim.x) X[cc * ld + k] *= (T)rinv[k];
      __syncthreads();
      const int rem = m - k - 1;
      for (int t = threadIdx.x; t < rem * w; t += blockDim.x) {
        int cc = t / rem, i = k + 1 + t % rem;
        X[cc * ld + i] -= La[k * ld + i] * X[cc * ld + k];
      }
      __syncthreads();
    }
    store_chunk(c0, w);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// General level kernel (large nodes, ranks above the small-node buckets).  Row
// transforms and updates are row-parallel with coalesced column accesses;
// reductions over rows use the tiled output-major helpers below; small dense
// algebra (r <= cap) runs in shared memory.
// ---------------------------------------------------------------------------
// Ancestor columns per update chunk (the same for every rank bucket: 16 for the
// rank <= 4 kernel measured slower, its accumulators spill).
#define LEVEL_W(RB) 8
#define LV_RED 64

// Serial upper Cholesky of A (r x r, ld) in place by one thread, pivots from
// one rsqrt each (as blk_chol_upper); rinv receives the reciprocal pivots.
__device__ inline bool thr_chol_upper(double* A, int ld, int r, double* rinv, double clamp) {
  double dmax = 0.0;
  for (int k = 0; k < r; ++k) dmax = fmax(dmax, A[k * ld + k]);
  const double floor_v = clamp * dmax;
  bool ok = true;
  for (int k = 0; k < r; ++k) {
    double d = A[k * ld + k];
    if (clamp > 0.0 && !(d > floor_v)) d = floor_v > 0.0 ? floor_v : 1.0;
    if (!(d > 0.0)) {
      ok = false;
      d = 1.0;
    }
    const double rs = rsqrt(d);
    A[k * ld + k] = d * rs;
    rinv[k] = rs;
    for (int j = k + 1; j < r; ++j) A[k * ld + j] *= rs;
    for (int i = k + 1; i < r; ++i)
      for (int j = i; j < r; ++j) A[i * ld + j] -= A[k * ld + i] * A[k * ld + j];
  }
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < i; ++j) A[i * ld + j] = 0.0;
  return ok;
}

// Ri = R^-1 (upper, r x r) by one thread, with the reciprocal pivots rinv.
__device__ inline void thr_triinv_upper(const double* R, int ldr, const double* rinv, double* Ri, int ldi, int r) {
  for (int j = 0; j < r; ++j)
    for (int i = r - 1; i >= 0; --i) {
      double acc = (i == j) ? 1.0 : 0.0;
      for (int k = i + 1; k <= j; ++k) acc -= R[i * ldr + k] * Ri[k * ldi + j];
      Ri[i * ldi + j] = (i <= j) ? acc * rinv[i] : 0.0;
    }
}

template <typename T, int RB>
__device__ __forceinline__ void rowmul_row(T* __restrict__ Xb, int64_t n, int r, int p, const double* Ri, int ldr) {
  double x[RB];
#pragma unroll
  for (int c = 0; c < RB; ++c) x[c] = c < r ? to_d(Xb[(size_t)c * n + p]) : 0.0;
#pragma unroll
  for (int c = 0; c < RB; ++c) {
    if (c < r) {
      double v = 0.0;
#pragma unroll
      for (int a = 0; a <= c; ++a) v += x[a] * Ri[a * ldr + c];
      Xb[(size_t)c * n + p] = (T)v;
    }
  }
}

// Rows [a0, a1): X[:, p] <- X[:, p] Ri (r x r upper triangular, shared, ld ldr).
template <typename T>
__device__ void rowmul_pass(T* __restrict__ Xb, int64_t n, int r, int a0, int a1, const double* Ri, int ldr) {
  for (int p = a0 + threadIdx.x; p < a1; p += blockDim.x) {
    if (r <= 4) rowmul_row<T, 4>(Xb, n, r, p, Ri, ldr);
    else if (r <= 8) rowmul_row<T, 8>(Xb, n, r, p, Ri, ldr);
    else if (r <= 16) rowmul_row<T, 16>(Xb, n, r, p, Ri, ldr);
    else {
      for (int c = r - 1; c >= 0; --c) {  // right to left: column c reads only columns <= c
        double v = 0.0;
        for (int a = 0; a <= c; ++a) v += to_d(Xb[(size_t)a * n + p]) * Ri[a * ldr + c];
        Xb[(size_t)c * n + p] = (T)v;
      }
    }
  }
  __syncthreads();
}

// Rows [a0, a1): B_j[p] += sum_a Q[a][p] Tm[a * W + j] for the WN columns of
// a chunk (Tm rows W apart).
template <typename T, int W, int WN>
__device__ void update_pass_n(const T* __restrict__ Qb, T* const* Bp, int64_t n, int r, int a0, int a1, const T* Tm) {
  for (int p = a0 + threadIdx.x; p < a1; p += blockDim.x) {
    T acc[WN];
#pragma unroll
    for (int j = 0; j < WN; ++j) acc[j] = Bp[j][p];
    for (int a = 0; a < r; ++a) {
      const T q = Qb[(size_t)a * n + p];
#pragma unroll
      for (int j = 0; j < WN; ++j) acc[j] += q * Tm[a * W + j];
    }
#pragma unroll
    for (int j = 0; j < WN; ++j) Bp[j][p] = acc[j];
  }
}

// The same for w <= W columns: a full chunk, or the last one with exactly its
// w columns (no products for the missing ones).
template <typename T, int W>
__device__ void update_pass(const T* __restrict__ Qb, T* const* Bp, int w, int64_t n, int r, int a0, int a1,
                            const T* Tm) {
  static_assert(W == 8, "chunks of 8 ancestor columns");
  switch (w) {
    case 8: update_pass_n<T, W, 8>(Qb, Bp, n, r, a0, a1, Tm); break;
    case 7: update_pass_n<T, W, 7>(Qb, Bp, n, r, a0, a1, Tm); break;
    case 6: update_pass_n<T, W, 6>(Qb, Bp, n, r, a0, a1, Tm); break;
    case 5: update_pass_n<T, W, 5>(Qb, Bp, n, r, a0, a1, Tm); break;
    case 4: update_pass_n<T, W, 4>(Qb, Bp, n, r, a0, a1, Tm); break;
    case 3: update_pass_n<T, W, 3>(Qb, Bp, n, r, a0, a1, Tm); break;
    case 2: update_pass_n<T, W, 2>(Qb, Bp, n, r, a0, a1, Tm); break;
    default: update_pass_n<T, W, 1>(Qb, Bp, n, r, a0, a1, Tm); break;
  }
}

// Pivot floors of the modified Cholesky used by FP32-stored factors, which only
// precondition an FP64 iteration (0: plain Cholesky, failures are reported).
template <typename T> __device__ __forceinline__ double clamp_gram() { return sizeof(T) == 4 ? 1e-12 : 0.0; }
template <typename T> __device__ __forceinline__ double clamp_cap() { return sizeof(T) == 4 ? 1e-6 : 0.0; }

// Reduce `count` doubles of the G partials of this group (slot order fixed)
// into dst; if G == 1 the partial already sits in dst.  The G partials of each
// output are split over the CTA's threads in chunks and the chunk sums
// combined by a pairwise tree in `red` (>= blockDim.x doubles of shared
// memory), so a large group costs a few loads per thread, not G serial ones.
__device__ inline bool group_reduce(double* dst, const double* src_local, int count, int G, int g, int base,
                                    double* part, size_t pstride, unsigned int* bar, unsigned int& phase,
                                    int* status, int* abort_flag, double* red, unsigned int spin) {
  if (G == 1) return true;
  // two slot sets alternate with the barrier count: a slot is rewritten only
  // after a later barrier that every reader of its previous contents has passed
  const size_t set = (size_t)(phase & 1u) * gridDim.x;
  double* mine = part + (set + base + g) * pstride;
  for (int t = threadIdx.x; t < count; t += blockDim.x) mine[t] = src_local[t];
  ++phase;
  if (!group_barrier(bar + base, (unsigned)G * phase, status, abort_flag, spin)) return false;
  const double* slots = part + (set + base) * pstride;
  if (count >= (int)blockDim.x) {
    for (int t = threadIdx.x; t < count; t += blockDim.x) {
      double v = 0.0;
      for (int q = 0; q < G; ++q) v += __ldcg(slots + (size_t)q * pstride + t);
      dst[t] = v;
    }
    __syncthreads();
    return true;
  }
  const int nch = min(G, (int)blockDim.x / count);
  const int t = threadIdx.x;
  if (t < nch * count) {
    const int o = t % count, ch = t / count;
    double v = 0.0;
    for (int q = ch; q < G; q += nch) v += __ldcg(slots + (size_t)q * pstride + o);
    red[ch * count + o] = v;
  }
  __syncthreads();
  for (int w = nch; w > 1;) {
    const int hw = (w + 1) / 2;
    for (int i = t; i < (w - hw) * count; i += blockDim.x) red[i] += red[i + hw * count];
    w = hw;
    __syncthreads();
  }
  for (int o = t; o < count; o += blockDim.x) dst[o] = red[o];
  __syncthreads();
  return true;
}


// ---------------------------------------------------------------------------
// Tiled, output-major reductions for the general level kernel: tiles of rows
// are staged in shared memory (coalesced loads, two buffers: the next tile's
// asynchronous copies are in flight while the current one is reduced), each
// output entry is owned by a group of threads that walk disjoint rows of the
// tile, and the groups' partial sums are combined by a short pairwise tree.
// FP64 instructions go to products of nonzero entries only.
// ---------------------------------------------------------------------------
#define LV_TR 128  // rows per staged tile
#define LV_TRP (LV_TR + 1)

__device__ __forceinline__ void pair_decode(int o, int r, int& a, int& b) {
  int rem = o;
  a = 0;
  while (rem >= r - a) {
    rem -= r - a;
    ++a;
  }
  b = a + rem;
}

// 8-byte asynchronous global -> shared copy (cp.async), its group commit and wait.
__device__ __forceinline__ void cp_async8(double* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Stage rows [p0, p0 + tr) of ncol columns (column c at col(c)) into a tile
// (column c at c * LV_TRP): asynchronous copies for FP64 storage, converting
// loads for FP32 storage.
template <typename T, typename ColF>
__device__ __forceinline__ void stage_tile(double* tile, int ncol, int p0, int tr, ColF col) {
  for (int i = threadIdx.x; i < ncol * tr; i += blockDim.x) {
    const int c = i / tr, p = i - c * tr;
    const T* src = col(c) + p0 + p;
    if constexpr (sizeof(T) == sizeof(double)) cp_async8(tile + c * LV_TRP + p, src);
    else tile[c * LV_TRP + p] = to_d(*src);
  }
}

// Walk the tiles of rows [a0, a1) with double buffering: body(tile, tr) runs on
// each staged tile by every thread (tbuf: doubles per buffer).
template <typename T, typename ColF, typename BodyF>
__device__ __forceinline__ void tile_walk(double* tile, int tbuf, int ncol, int a0, int a1, ColF col, BodyF body) {
  const int nt = a1 > a0 ? (a1 - a0 + LV_TR - 1) / LV_TR : 0;
  if (nt > 0) stage_tile<T>(tile, ncol, a0, min(LV_TR, a1 - a0), col);
  cp_async_commit();
  for (int k = 0; k < nt; ++k) {
    const int pn = a0 + (k + 1) * LV_TR;
    if (k + 1 < nt) stage_tile<T>(tile + ((k + 1) & 1) * tbuf, ncol, pn, min(LV_TR, a1 - pn), col);
    cp_async_commit();
    cp_async_wait_prev();  // this thread's copies of tile k have landed
    __syncthreads();       // ... and every thread's
    body(tile + (k & 1) * tbuf, min(LV_TR, a1 - (a0 + k * LV_TR)));
    __syncthreads();       // the buffer is free for tile k + 2
  }
}

// Packed Gram matrix: Gp[q] = sum over rows [a0, a1) of X[a][p] X[b][p] for the
// pair (a, b), a <= b < r, q = pair index (row-major upper triangle).  More
// pairs than threads are taken in chunks of blockDim.x pairs.
template <typename T>
__device__ void gram_tiled(const T* __restrict__ Xb, int64_t n, int r, int a0, int a1, double* tile, int tbuf,
                           double* part, double* Gp) {
  const int np_all = r * (r + 1) / 2;
  const int t = threadIdx.x;
  for (int q0 = 0; q0 < np_all; q0 += blockDim.x) {
    const int np = min((int)blockDim.x, np_all - q0);
    const int ng = max(1, (int)blockDim.x / np);
    const bool active = t < np * ng;
    const int o = active ? t % np : 0, gidx = active ? t / np : 0;
    int a = 0, b = 0;
    pair_decode(q0 + o, r, a, b);
    double acc = 0.0;
    tile_walk<T>(tile, tbuf, r, a0, a1, [&](int c) { return Xb + (size_t)c * n; },
                 [&](const double* tl, int tr) {
                   if (active)
                     for (int p = gidx; p < tr; p += ng) acc += tl[a * LV_TRP + p] * tl[b * LV_TRP + p];
                 });
    if (active) part[gidx * np + o] = acc;
    __syncthreads();
    // pairwise tree over the ng group partials, all outputs at once (few FP64
    // instructions per output instead of ng serial adds)
    for (int w = ng; w > 1;) {
      const int hw = (w + 1) / 2;
      for (int i = t; i < (w - hw) * np; i += blockDim.x) {
        const int g = i / np, q = i % np;
        part[g * np + q] += part[(g + hw) * np + q];
      }
      w = hw;
      __syncthreads();
    }
    for (int q = t; q < np; q += blockDim.x) Gp[q0 + q] = part[q];
    __syncthreads();
  }
}

// Unpack a packed Gram matrix into G (r x r, both triangles, ld ldg).
__device__ void gram_unpack(const double* Gp, int r, double* G, int ldg) {
  for (int q = threadIdx.x; q < r * (r + 1) / 2; q += blockDim.x) {
    int a, b;
    pair_decode(q, r, a, b);
    G[a * ldg + b] = Gp[q];
    G[b * ldg + a] = Gp[q];
  }
  __syncthreads();
}

// Pm[a * W + j] = sum over rows [a0, a1) of Q[a][p] B_j[p], products in the storage precision.
template <typename T, int W>
__device__ void proj_tiled(const T* __restrict__ Qb, T* const* Bp, int w, int64_t n, int r, int a0, int a1,
                           double* tile, int tbuf, double* part, double* Pm) {
  const int np = r * w;
  const int ng = max(1, (int)blockDim.x / np);
  const int t = threadIdx.x;
  const bool active = t < np * ng;
  const int o = active ? t % np : 0, gidx = active ? t / np : 0;
  const int a = o / w, j = o % w;
  T acc = (T)0;
  tile_walk<T>(tile, tbuf, r + w, a0, a1, [&](int c) { return c < r ? Qb + (size_t)c * n : (const T*)Bp[c - r]; },
               [&](const double* tl, int tr) {
                 if (active)
                   for (int p = gidx; p < tr; p += ng) acc += (T)tl[a * LV_TRP + p] * (T)tl[(r + j) * LV_TRP + p];
               });
  if (active) part[gidx * np + o] = (double)acc;
  __syncthreads();
  for (int gw = ng; gw > 1;) {  // pairwise tree over the group partials
    const int hw = (gw + 1) / 2;
    for (int i = t; i < (gw - hw) * np; i += blockDim.x) {
      const int g = i / np, q = i % np;
      part[g * np + q] += part[(g + hw) * np + q];
    }
    gw = hw;
    __syncthreads();
  }
  for (int q = t; q < np; q += blockDim.x) Pm[(q / w) * W + q % w] = part[q];
  __syncthreads();
}

// RB > 0: a rank bucket, nodes with RLO < r <= RB, small matrices with leading
// dimension RB (less shared memory and registers, more CTAs per SM); RB == 0:
// nodes with r > RLO, leading dimension cap.
template <typename T, int RB, int RLO>
__global__ void __launch_bounds__(256, RB == 4 ? 4 : (RB == 16 ? 3 : 2))
    k_level(const FactDesc* __restrict__ Fd, int lvl, int G, double* __restrict__ gpart,
            unsigned int* __restrict__ bar, int* __restrict__ abort_flag, int skip_le, size_t sstride) {
  extern __shared__ double sm[];
  // problem of a batched launch: its descriptor, and its scratch sstride bytes on
  Fd += blockIdx.y;
  if (Fd->skip && *Fd->skip) return;  // the same for every CTA: no group waits on a missing one
  gpart = (double*)((char*)gpart + blockIdx.y * sstride);
  bar = (unsigned int*)((char*)bar + blockIdx.y * sstride);
  abort_flag = (int*)((char*)abort_flag + blockIdx.y * sstride);
  const int bi = blockIdx.x / G, g = blockIdx.x % G, base = blockIdx.x - g;
  const int nid = node_id(lvl, bi);
  const int cap = Fd->cap, nleaf = Fd->nleaf;
  const int64_t n = Fd->n;
  const int* bnd = Fd->bnd;
  int s, h, e;
  node_range(bnd, lvl, bi, s, h, e);
  const int r = Fd->rank[nid];
  if (r <= skip_le || r <= RLO || (RB > 0 && r > RB)) return;  // another launch takes this node
  if (r == 0) {
    if (g == 0 && threadIdx.x == 0) Fd->ld_parts[nleaf + nid] = 0.0;
    return;
  }
  int* status = Fd->status;
  T* Qall = (T*)Fd->Q;
  T* Qb = Qall + (size_t)lvl * cap * n;
  const int len = e - s, rc = (len + G - 1) / G;
  const int r0 = s + min(len, g * rc), r1 = s + min(len, g * rc + rc);
  const int ldm = RB > 0 ? RB : cap;  // leading dimension of the small matrices
  constexpr int W = LEVEL_W(RB);      // ancestor columns per update chunk
  const int cc2 = ldm * ldm;
  double* Gm = sm;                        // Gram / factor of the left side
  double* Gm2 = Gm + cc2;                 // ... of the right side
  double* Ri = Gm2 + cc2;                 // inverse factors of both sides (Ri2 follows Ri:
  double* Ri2 = Ri + cc2;                 // the packed Gram entries of both sides span them)
  double* RU = Ri2 + cc2;                 // R1, then R = R2 R1 of the left side
  double* RV = RU + cc2;                  // ... of the right side
  double* rvs = RV + cc2;                 // 2 x 8 reciprocal pivots (serial small factorizations)
  const int tbuf = (ldm + W) * LV_TRP;    // doubles per row tile
  double* tile = rvs + 16;                // two (ldm + W) x LV_TRP row tiles
  double* part = tile + 2 * tbuf;         // 256 group partial sums
  double* tmp = part + 256;               // LV_RED
  double* Pm = tmp + LV_RED;              // 2ldm x W
  T* Tm = (T*)(Pm + 2 * ldm * W);      // 2ldm x W, storage precision
  T** Bp = (T**)(Pm + 4 * ldm * W);    // W column pointers
  int* iflag = (int*)(Bp + W);
  int* alist = iflag + 4;                 // ancestor columns (level << 8 | col)
  const size_t pstride = level_part_stride(cap);
  unsigned int phase = 0;
  bool ok = true;

  // CholeskyQR2 of both sides at once (Gram, R1, Q1 = X R1^-1, Gram, R2,
  // Q = Q1 R2^-1, R = R2 R1): one group reduction per pass carries the packed
  // Gram entries of both sides, so CTAs whose rows lie in one side never idle
  // while the other side is factored
  const int npk = r * (r + 1) / 2;
  const int sa0 = max(r0, s), sa1 = min(r1, h), sb0 = max(r0, h), sb1 = min(r1, e);
  if (threadIdx.x == 0) iflag[2] = 0;
  for (int pass = 0; pass < 2; ++pass) {
    gram_tiled<T>(Qb, n, r, sa0, sa1, tile, tbuf, part, Ri);
    gram_tiled<T>(Qb, n, r, sb0, sb1, tile, tbuf, part, Ri + npk);
    if (!group_reduce(Ri, Ri, 2 * npk, G, g, base, gpart, pstride, bar, phase, status, abort_flag, part, Fd->spin))
      return;
    gram_unpack(Ri, r, Gm, ldm);
    gram_unpack(Ri + npk, r, Gm2, ldm);
    if (r <= 8) {
      // small ranks: each side's factorization by one thread (two warps side by side)
      if (threadIdx.x == 0 || threadIdx.x == 32) {
        const int sd = threadIdx.x >> 5;
        double* Gs = sd ? Gm2 : Gm;
        double* Rs = sd ? RV : RU;
        double* rv = rvs + 8 * sd;
        if (!thr_chol_upper(Gs, ldm, r, rv, clamp_gram<T>())) iflag[2] = 1;
        thr_triinv_upper(Gs, ldm, rv, sd ? Ri2 : Ri, ldm, r);
        for (int i = 0; i < r; ++i)
          for (int j = 0; j < r; ++j) {
            if (pass == 0) {
              Rs[i * ldm + j] = Gs[i * ldm + j];
            } else if (i <= j) {  // R = R2 R1 in place, rows top-down: row i reads rows >= i of R1
              double v = 0.0;
              for (int k = i; k <= j; ++k) v += Gs[i * ldm + k] * Rs[k * ldm + j];
              Rs[i * ldm + j] = v;
            }
          }
      }
      __syncthreads();
    } else {
      for (int sd = 0; sd < 2; ++sd) {
        double* Gs = sd ? Gm2 : Gm;
        double* Rs = sd ? RV : RU;
        ok = blk_chol_upper(Gs, ldm, r, iflag, clamp_gram<T>()) && ok;
        blk_triinv_upper(Gs, ldm, sd ? Ri2 : Ri, ldm, r);
        if (pass == 0) {
          for (int t = threadIdx.x; t < cc2; t += blockDim.x) Rs[t] = Gs[t];
        } else {
          // R = R2 R1 in place, one thread per column, rows top-down
          for (int j = threadIdx.x; j < r; j += blockDim.x)
            for (int i = 0; i <= j; ++i) {
              double v = 0.0;
              for (int k = i; k <= j; ++k) v += Gs[i * ldm + k] * Rs[k * ldm + j];
              Rs[i * ldm + j] = v;
            }
        }
        __syncthreads();
      }
    }
    rowmul_pass<T>(Qb, n, r, sa0, sa1, Ri, ldm);
    rowmul_pass<T>(Qb, n, r, sb0, sb1, Ri2, ldm);
  }
  ok = ok && iflag[2] == 0;
  if (!ok && g == 0 && threadIdx.x == 0) atomicOr(status, FIFA_DEV_NOT_SPD);

  // capacitance: S = I + R X R^T, L_S = chol(S) (computed by the group's first CTA)
  const int r2 = 2 * r, ld2 = 2 * cap;
  double* Zf = Fd->Zf + (size_t)nid * ld2 * ld2;
  double* Zi = Fd->Zi + (size_t)nid * ld2 * ld2;
  if (g == 0 && 8 * ldm * ldm <= 2 * tbuf) {
    // S and its inverse factor in shared memory (the row tile is free here),
    // so the serial pivot chain never waits on global memory
    double* Sm = tile;
    double* Sim = tile + 4 * ldm * ldm;
    for (int t = threadIdx.x; t < r2 * r2; t += blockDim.x) {
      const int a = t / r2, b = t % r2;
      double v = (a == b) ? 1.0 : 0.0;
      if (a < r && b >= r) {
        for (int k = 0; k < r; ++k) v += RU[a * ldm + k] * RV[(b - r) * ldm + k];
      } else if (a >= r && b < r) {
        for (int k = 0; k < r; ++k) v += RV[(a - r) * ldm + k] * RU[b * ldm + k];
      }
      Sm[a * r2 + b] = v;
    }
    __syncthreads();
    const bool ok2 = blk_chol_upper(Sm, r2, r2, iflag, clamp_cap<T>());  // R_S (upper), L_S = R_S^T
    double ls = 0.0;
    for (int k = threadIdx.x; k < r2; k += blockDim.x) ls += log(Sm[k * r2 + k]);
    ls = block_sum(ls, tmp);
    blk_triinv_upper(Sm, r2, Sim, r2, r2);  // R_S^-1 (upper) = (L_S^-1)^T
    for (int t = threadIdx.x; t < r2 * r2; t += blockDim.x) {
      const int a = t / r2, b = t % r2;
      const double dd = (a == b) ? 1.0 : 0.0;
      Zf[a * ld2 + b] = (a >= b ? Sm[b * r2 + a] : 0.0) - dd;
      Zi[a * ld2 + b] = (a >= b ? Sim[b * r2 + a] : 0.0) - dd;
    }
    if (threadIdx.x == 0) {
      Fd->ld_parts[nleaf + nid] = ls;
      if (!ok2) atomicOr(status, FIFA_DEV_NOT_SPD);
    }
    __syncthreads();
  } else if (g == 0) {
    for (int t = threadIdx.x; t < r2 * r2; t += blockDim.x) {
      const int a = t / r2, b = t % r2;
      double v = (a == b) ? 1.0 : 0.0;
      if (a < r && b >= r) {
        const int bb = b - r;
        for (int k = 0; k < r; ++k) v += RU[a * ldm + k] * RV[bb * ldm + k];
      } else if (a >= r && b < r) {
        const int aa = a - r;
        for (int k = 0; k < r; ++k) v += RV[aa * ldm + k] * RU[b * ldm + k];
      }
      Zf[a * ld2 + b] = v;
    }
    __syncthreads();
    const bool ok2 = blk_chol_upper(Zf, ld2, r2, iflag, clamp_cap<T>());  // Zf <- R_S (upper), S = R_S^T R_S, L_S = R_S^T
    double ls = 0.0;
    for (int k = threadIdx.x; k < r2; k += blockDim.x) ls += log(Zf[k * ld2 + k]);
    ls = block_sum(ls, tmp);
    blk_triinv_upper(Zf, ld2, Zi, ld2, r2);  // Zi <- R_S^-1 (upper) = (L_S^-1)^T
    for (int t = threadIdx.x; t < r2 * r2; t += blockDim.x) {  // transpose in place, then subtract I
      const int a = t / r2, b = t % r2;
      if (a < b) {
        double u = Zf[a * ld2 + b], l = Zf[b * ld2 + a];
        Zf[a * ld2 + b] = l;
        Zf[b * ld2 + a] = u;
        u = Zi[a * ld2 + b];
        l = Zi[b * ld2 + a];
        Zi[a * ld2 + b] = l;
        Zi[b * ld2 + a] = u;
      }
    }
    __syncthreads();
    for (int a = threadIdx.x; a < r2; a += blockDim.x) {
      Zf[a * ld2 + a] -= 1.0;
      Zi[a * ld2 + a] -= 1.0;
    }
    if (threadIdx.x == 0) {
      Fd->ld_parts[nleaf + nid] = ls;
      if (!ok2) atomicOr(status, FIFA_DEV_NOT_SPD);
    }
    __syncthreads();
  }
  if (G > 1) {
    ++phase;
    if (!group_barrier(bar + base, (unsigned)G * phase, status, abort_flag, Fd->spin)) return;
  }
  if (lvl == 0) return;

  // the inverse node factor I + Q Zi Q^T applied to every ancestor basis on these rows
  __shared__ int nanc;
  __shared__ int rka[FIFA_LEVELS_MAX];
  for (int j = threadIdx.x; j < lvl; j += blockDim.x) rka[j] = Fd->rank[node_id(j, bi >> (lvl - j))];
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    for (int j = 0; j < lvl; ++j)
      for (int q = 0; q < rka[j]; ++q) alist[c++] = (j << 8) | q;
    nanc = c;
  }
  __syncthreads();
  const int na = nanc;
  for (int c0 = 0; c0 < na; c0 += W) {
    const int w = min(W, na - c0);
    if (threadIdx.x < W) {
      const int code = alist[c0 + min((int)threadIdx.x, w - 1)];
      Bp[threadIdx.x] = Qall + ((size_t)(code >> 8) * cap + (code & 255)) * n;
    }
    for (int t = threadIdx.x; t < 2 * ldm * W; t += blockDim.x) Pm[t] = 0.0;
    __syncthreads();
    proj_tiled<T, W>(Qb, Bp, w, n, r, max(r0, s), min(r1, h), tile, tbuf, part, Pm);
    proj_tiled<T, W>(Qb, Bp, w, n, r, max(r0, h), min(r1, e), tile, tbuf, part, Pm + r * W);
    if (!group_reduce(Pm, Pm, r2 * W, G, g, base, gpart, pstride, bar, phase, status, abort_flag, part, Fd->spin))
      return;
    for (int t = threadIdx.x; t < r2 * W; t += blockDim.x) {
      const int a = t / W, j = t % W;
      double acc = 0.0;
      if (j < w)
        for (int b = 0; b < r2; ++b) acc += Zi[a * ld2 + b] * Pm[b * W + j];
      Tm[a * W + j] = (T)acc;
    }
    __syncthreads();
    update_pass<T, W>(Qb, Bp, w, n, r, max(r0, s), min(r1, h), Tm);
    update_pass<T, W>(Qb, Bp, w, n, r, max(r0, h), min(r1, e), Tm + r * W);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Small-node level kernel.  One CTA per node with sides of at most MS rows and
// rank in (RLO, R].  The node's basis rows and each chunk of ancestor columns
// are staged in shared memory, and every reduction is computed by one thread
// per output entry (a dot product over the node's rows): no cross-thread FP64
// reductions, so FP64 instructions are spent on the products alone.
// ---------------------------------------------------------------------------
template <typename T, int R, int RLO, int MS, int W>
__global__ void __launch_bounds__(128) k_level_small(const FactDesc* __restrict__ Fd, int lvl) {
  Fd += blockIdx.y;  // problem of a batched launch
  if (Fd->skip && *Fd->skip) return;
  constexpr int R2 = 2 * R;
  __shared__ double Xs[2][R][MS];   // side-major basis rows (FP64 during the QR)
  __shared__ T Bs[W][2 * MS];       // ancestor-column chunk on the node's rows
  __shared__ double Gm[R * R], Ri[R * R], R1[R * R], RU[R * R], RV[R * R];
  __shared__ double S[R2 * R2], Si[R2 * R2];
  __shared__ double Pm[R2 * W];
  __shared__ T Tm[R2 * W];
  __shared__ double red[40];
  __shared__ int iflag[4];
  __shared__ int rpre[FIFA_LEVELS_MAX + 1];  // prefix sums of the ancestor ranks
  __shared__ int ccode[W];                    // (level << 8) | column of the chunk's columns
  const int bi = blockIdx.x;
  const int nid = node_id(lvl, bi);
  const int r = Fd->rank[nid];
  if (r > R || r <= RLO) return;  // another bucket's launch takes this node
  const int cap = Fd->cap, nleaf = Fd->nleaf;
  const int64_t n = Fd->n;
  const int* bnd = Fd->bnd;
  int s, h, e;
  node_range(bnd, lvl, bi, s, h, e);
  if (r == 0) {
    if (threadIdx.x == 0) Fd->ld_parts[nleaf + nid] = 0.0;
    return;
  }
  T* Qall = (T*)Fd->Q;
  T* Qb = Qall + (size_t)lvl * cap * n;
  int* status = Fd->status;
  const int mu = h - s, mv = e - h;  // rows per side
  for (int t = threadIdx.x; t < r * MS; t += blockDim.x) {
    const int c = t / MS, p = t % MS;
    Xs[0][c][p] = p < mu ? (double)Qb[(size_t)c * n + s + p] : 0.0;
    Xs[1][c][p] = p < mv ? (double)Qb[(size_t)c * n + h + p] : 0.0;
  }
  __syncthreads();
  bool ok = true;
  const double cg = clamp_gram<T>();
  for (int side = 0; side < 2; ++side) {
    const int m = side ? mv : mu;
    double(*X)[MS] = Xs[side];
    for (int pass = 0; pass < 2; ++pass) {
      // Gram matrix, one thread per entry a <= b
      for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
        const int a = t / r, b = t % r;
        if (a <= b) {
          double acc = 0.0;
          for (int p = 0; p < m; ++p) acc += X[a][p] * X[b][p];
          Gm[a * R + b] = acc;
          Gm[b * R + a] = acc;
        }
      }
      __syncthreads();
      ok = blk_chol_upper(Gm, R, r, iflag, cg) && ok;
      if (pass == 0) {
        for (int t = threadIdx.x; t < R * R; t += blockDim.x) R1[t] = Gm[t];
      } else {
        double* Rs = side ? RV : RU;
        for (int t = threadIdx.x; t < R * R; t += blockDim.x) {
          const int i = t / R, j = t % R;
          double v = 0.0;
          if (i < r && j < r && i <= j)
            for (int k = i; k <= j; ++k) v += Gm[i * R + k] * R1[k * R + j];
          Rs[t] = v;
        }
      }
      __syncthreads();
      blk_triinv_upper(Gm, R, Ri, R, r);
      // X <- X Ri, one thread per row (the row is read before it is overwritten)
      for (int p = threadIdx.x; p < m; p += blockDim.x) {
        double xr[R];
#pragma unroll
        for (int c = 0; c < R; ++c) xr[c] = c < r ? X[c][p] : 0.0;
#pragma unroll
        for (int c = 0; c < R; ++c) {
          if (c < r) {
            double v = 0.0;
#pragma unroll
            for (int a = 0; a <= c; ++a) v += xr[a] * Ri[a * R + c];
            X[c][p] = (double)(T)v;  // the stored basis is rounded to T
          }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < r * MS; t += blockDim.x) {
    const int c = t / MS, p = t % MS;
    if (p < mu) Qb[(size_t)c * n + s + p] = (T)Xs[0][c][p];
    if (p < mv) Qb[(size_t)c * n + h + p] = (T)Xs[1][c][p];
  }
  // capacitance: S = I + R X R^T, L_S = chol(S) = R_S^T
  const int r2 = 2 * r;
  for (int t = threadIdx.x; t < r2 * r2; t += blockDim.x) {
    const int a = t / r2, b = t % r2;
    double v = (a == b) ? 1.0 : 0.0;
    if (a < r && b >= r) {
      for (int k = 0; k < r; ++k) v += RU[a * R + k] * RV[(b - r) * R + k];
    } else if (a >= r && b < r) {
      for (int k = 0; k < r; ++k) v += RV[(a - r) * R + k] * RU[b * R + k];
    }
    S[a * R2 + b] = v;
  }
  __syncthreads();
  ok = blk_chol_upper(S, R2, r2, iflag, clamp_cap<T>()) && ok;
  double ls = 0.0;
  for (int k = threadIdx.x; k < r2; k += blockDim.x) ls += log(S[k * R2 + k]);
  ls = block_sum(ls, red);
  blk_triinv_upper(S, R2, Si, R2, r2);
  const int ld2 = 2 * cap;
  double* Zf = Fd->Zf + (size_t)nid * ld2 * ld2;
  double* Zi = Fd->Zi + (size_t)nid * ld2 * ld2;
  for (int t = threadIdx.x; t < r2 * r2; t += blockDim.x) {
    const int a = t / r2, b = t % r2;
    const double d = (a == b) ? 1.0 : 0.0;
    Zf[a * ld2 + b] = (a >= b ? S[b * R2 + a] : 0.0) - d;
    Zi[a * ld2 + b] = (a >= b ? Si[b * R2 + a] : 0.0) - d;
  }
  if (threadIdx.x == 0) {
    Fd->ld_parts[nleaf + nid] = ls;
    if (!ok) atomicOr(status, FIFA_DEV_NOT_SPD);
  }
  if (lvl == 0) return;
  // ancestor bases on the node's rows: B <- B + Q (L_S^-1 - I) Q^T B
  if (threadIdx.x == 0) {
    int c = 0;
    for (int j = 0; j < lvl; ++j) {
      rpre[j] = c;
      c += Fd->rank[node_id(j, bi >> (lvl - j))];
    }
    rpre[lvl] = c;
  }
  __syncthreads();
  const int na = rpre[lvl], mn = e - s;
  for (int c0 = 0; c0 < na; c0 += W) {
    const int w = min(W, na - c0);
    if (threadIdx.x < w) {  // ancestor column c0 + t: level j with rpre[j] <= c < rpre[j + 1]
      const int c = c0 + threadIdx.x;
      int j = 0;
      while (rpre[j + 1] <= c) ++j;
      ccode[threadIdx.x] = (j << 8) | (c - rpre[j]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < w * mn; t += blockDim.x) {
      const int j = t / mn, p = t % mn;
      const int code = ccode[j];
      Bs[j][p] = Qall[((size_t)(code >> 8) * cap + (code & 255)) * n + s + p];
    }
    __syncthreads();
    // P[a][j] = Q^T B: rows a < r from the left child, r <= a < 2r from the right
    for (int t = threadIdx.x; t < r2 * w; t += blockDim.x) {
      const int a = t / w, j = t % w;
      const int side = a >= r, c = side ? a - r : a, m = side ? mv : mu, off = side ? mu : 0;
      T acc = (T)0;
      for (int p = 0; p < m; ++p) acc += (T)Xs[side][c][p] * Bs[j][off + p];
      Pm[a * W + j] = (double)acc;
    }
    __syncthreads();
    // T = (L_S^-1 - I) P
    for (int t = threadIdx.x; t < r2 * w; t += blockDim.x) {
      const int a = t / w, j = t % w;
      double v = -Pm[a * W + j];
      for (int b = 0; b <= a; ++b) v += Si[b * R2 + a] * Pm[b * W + j];
      Tm[a * W + j] = (T)v;
    }
    __syncthreads();
    // B += Q T, one thread per (row, column)
    for (int t = threadIdx.x; t < w * mn; t += blockDim.x) {
      const int j = t / mn, p = t % mn;
      const int side = p >= mu, pp = side ? p - mu : p, toff = side ? r : 0;
      T acc = Bs[j][p];
      for (int a = 0; a < r; ++a) acc += (T)Xs[side][a][pp] * Tm[(toff + a) * W + j];
      const int code = ccode[j];
      Qall[((size_t)(code >> 8) * cap + (code & 255)) * n + s + p] = acc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Multi-node small-level kernel: NPC nodes of one level per CTA (sides of at
// most MS rows, rank <= R), the same arithmetic as k_level_small.  Every step
// is spread over the nodes: the per-node dense algebra (Cholesky, triangular
// inverse, capacitance) runs one thread per node and side, and the row and
// column work runs over all the CTA's nodes at once, so few lanes idle while
// FP64 instructions issue.
// ---------------------------------------------------------------------------
#define LM_W 8  // ancestor columns per chunk

// Double-buffered ancestor chunks only for one node per CTA: with several
// nodes the second buffer costs a co-resident CTA per SM (measured slower).
template <int NPC> struct LmDB { static constexpr int nbuf = NPC == 1 ? 2 : 1; };

template <int R, int MS, int NPC>
struct LmLayout {
  static constexpr int R2 = 2 * R;
  static constexpr size_t xs = (size_t)NPC * 2 * R * MS;  // doubles
  static constexpr size_t mats = (size_t)NPC * 2 * R * R;  // Gm / Ri / R1 / rinv (doubles each)
  static constexpr size_t ruv = (size_t)NPC * R * R;       // RU / RV
  static constexpr size_t sm = (size_t)NPC * R2 * R2;      // S / Si
  static constexpr size_t pm = (size_t)NPC * R2 * LM_W;    // Pm / Tm
  static constexpr size_t doubles = xs + 3 * mats + (size_t)NPC * 2 * R + 2 * ruv + 2 * sm + pm;
  static size_t bytes(int elt) {
    return doubles * sizeof(double) + (size_t)LmDB<NPC>::nbuf * NPC * LM_W * 2 * MS * elt + pm * elt +
           (size_t)NPC * (FIFA_LEVELS_MAX + 1 + LmDB<NPC>::nbuf * LM_W + 8) * sizeof(int) + 64;
  }
};

template <typename T, int R, int MS, int NPC>
__global__ void __launch_bounds__(256) k_level_multi(const FactDesc* __restrict__ Fd, int lvl, int nodes) {
  Fd += blockIdx.y;  // problem of a batched launch
  if (Fd->skip && *Fd->skip) return;
  using LY = LmLayout<R, MS, NPC>;
  constexpr int R2 = 2 * R;
  extern __shared__ double smd[];
  double* Xs = smd;                       // [j][side][c][p]
  double* Gm = Xs + LY::xs;               // [j][side][R*R]
  double* Ri = Gm + LY::mats;
  double* R1 = Ri + LY::mats;
  double* rv = R1 + LY::mats;             // [j][side][R] reciprocal pivots
  double* RU = rv + NPC * 2 * R;          // [j][R*R]
  double* RV = RU + LY::ruv;
  double* S = RV + LY::ruv;               // [j][R2*R2]
  double* Si = S + LY::sm;
  double* Pm = Si + LY::sm;               // [j][R2][LM_W]
  constexpr int NB = LmDB<NPC>::nbuf;
  T* Bs2 = (T*)(Pm + LY::pm);             // NB buffers of [j][LM_W][2 MS]
  T* Tm = Bs2 + NB * (size_t)NPC * LM_W * 2 * MS;  // [j][R2][LM_W]
  int* ib = (int*)(Tm + LY::pm);
  int* rpre = ib;                          // [j][LEVELS_MAX + 1]
  int* ccode2 = rpre + NPC * (FIFA_LEVELS_MAX + 1);  // NB buffers of [j][LM_W]
  int* info = ccode2 + NB * NPC * LM_W;    // [j][8]: r, s, h, e, active, ok

  const int cap = Fd->cap, nleaf = Fd->nleaf;
  const int64_t n = Fd->n;
  const int* bnd = Fd->bnd;
  T* Qall = (T*)Fd->Q;
  T* Qb = Qall + (size_t)lvl * cap * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int b0 = blockIdx.x * NPC;

  if (tid < NPC) {
    const int bi = b0 + tid;
    int* in = info + tid * 8;
    in[4] = 0;
    in[5] = 1;
    if (bi < nodes) {
      const int nid = node_id(lvl, bi);
      const int r = Fd->rank[nid];
      int s, h, e;
      node_range(bnd, lvl, bi, s, h, e);
      in[0] = r;
      in[1] = s;
      in[2] = h;
      in[3] = e;
      if (r == 0) Fd->ld_parts[nleaf + nid] = 0.0;
      in[4] = (r > 0 && r <= R) ? 1 : 0;  // larger ranks: another launch takes the node
    }
  }
  __syncthreads();
  // stage the bases of every node's two sides (FP64 during the QR)
  for (int t = tid; t < NPC * 2 * R * MS; t += nt) {
    const int j = t / (2 * R * MS), rem = t % (2 * R * MS), side = rem / (R * MS), c = (rem / MS) % R, p = rem % MS;
    const int* in = info + j * 8;
    double v = 0.0;
    if (in[4] && c < in[0]) {
      const int a0 = side ? in[2] : in[1], m = side ? in[3] - in[2] : in[2] - in[1];
      if (p < m) v = (double)Qb[(size_t)c * n + a0 + p];
    }
    Xs[t] = v;
  }
  __syncthreads();
  const double cg = clamp_gram<T>();
  for (int pass = 0; pass < 2; ++pass) {
    // Gram entries (j, side, a <= b), one thread each, serial over the side's
    // rows.  Pairs in column order of the upper triangle (q < r (r + 1) / 2 are
    // exactly a rank-r node's pairs) and the nodes' sides fastest: the active
    // lanes are the first threads, not a few in every warp.
    constexpr int NPAIR = R * (R + 1) / 2;
    for (int t = tid; t < NPC * 2 * NPAIR; t += nt) {
      const int q = t / (NPC * 2), js = t % (NPC * 2), j = js / 2, side = js % 2;
      const int* in = info + j * 8;
      const int r = in[0];
      if (!in[4]) continue;
      int b = 0;
      while ((b + 1) * (b + 2) / 2 <= q) ++b;
      const int a = q - b * (b + 1) / 2;
      if (b >= r) continue;
      const int m = side ? in[3] - in[2] : in[2] - in[1];
      const double* X = Xs + (size_t)js * R * MS;
      double acc = 0.0;
      for (int p = 0; p < m; ++p) acc += X[a * MS + p] * X[b * MS + p];
      Gm[js * R * R + a * R + b] = acc;
      Gm[js * R * R + b * R + a] = acc;
    }
    __syncthreads();
    // Cholesky, R1 / R = R2 R1, inverse: one thread per (node, side)
    if (tid < NPC * 2) {
      const int js = tid, j = js / 2, side = js % 2;
      int* in = info + j * 8;
      if (in[4]) {
        const int r = in[0];
        double* G = Gm + js * R * R;
        if (!thr_chol_upper(G, R, r, rv + js * R, cg)) atomicAnd(&in[5], 0);
        if (pass == 0) {
          for (int t = 0; t < R * R; ++t) R1[js * R * R + t] = G[t];
        } else {
          double* Rs = (side ? RV : RU) + j * R * R;
          for (int i = 0; i < R; ++i)
            for (int jj = 0; jj < R; ++jj) {
              double v = 0.0;
              if (i < r && jj < r && i <= jj)
                for (int k = i; k <= jj; ++k) v += G[i * R + k] * R1[js * R * R + k * R + jj];
              Rs[i * R + jj] = v;
            }
        }
        thr_triinv_upper(G, R, rv + js * R, Ri + js * R * R, R, r);
      }
    }
    __syncthreads();
    // X <- X Ri, one thread per row (rounded to the storage precision)
    for (int t = tid; t < NPC * 2 * MS; t += nt) {
      const int js = t / MS, p = t % MS, j = js / 2, side = js % 2;
      const int* in = info + j * 8;
      if (!in[4]) continue;
      const int r = in[0], m = side ? in[3] - in[2] : in[2] - in[1];
      if (p >= m) continue;
      double* X = Xs + (size_t)js * R * MS;
      const double* Rij = Ri + js * R * R;
      double xr[R];
#pragma unroll
      for (int c = 0; c < R; ++c) xr[c] = c < r ? X[c * MS + p] : 0.0;
#pragma unroll
      for (int c = 0; c < R; ++c)
        if (c < r) {
          double v = 0.0;
#pragma unroll
          for (int a = 0; a <= c; ++a) v += xr[a] * Rij[a * R + c];
          X[c * MS + p] = (double)(T)v;
        }
    }
    __syncthreads();
  }
  // orthonormal bases back to global memory
  for (int t = tid; t < NPC * 2 * R * MS; t += nt) {
    const int j = t / (2 * R * MS), rem = t % (2 * R * MS), side = rem / (R * MS), c = (rem / MS) % R, p = rem % MS;
    const int* in = info + j * 8;
    if (!in[4] || c >= in[0]) continue;
    const int a0 = side ? in[2] : in[1], m = side ? in[3] - in[2] : in[2] - in[1];
    if (p < m) Qb[(size_t)c * n + a0 + p] = (T)Xs[t];
  }
  // capacitance S = I + R X R^T, L_S = chol(S) = R_S^T, one thread per node
  if (tid < NPC) {
    const int j = tid;
    int* in = info + j * 8;
    if (in[4]) {
      const int r = in[0], r2 = 2 * r;
      const double* ru = RU + j * R * R;
      const double* rvv = RV + j * R * R;
      double* Sj = S + j * R2 * R2;
      for (int a = 0; a < r2; ++a)
        for (int b = 0; b < r2; ++b) {
          double v = (a == b) ? 1.0 : 0.0;
          if (a < r && b >= r) {
            for (int k = 0; k < r; ++k) v += ru[a * R + k] * rvv[(b - r) * R + k];
          } else if (a >= r && b < r) {
            for (int k = 0; k < r; ++k) v += rvv[(a - r) * R + k] * ru[b * R + k];
          }
          Sj[a * R2 + b] = v;
        }
      double srv[R2];
      if (!thr_chol_upper(Sj, R2, r2, srv, clamp_cap<T>())) in[5] = 0;
      // log det L_S from one logarithm of the pivots' product (a serial chain
      // of r2 logarithms here costs more than the rest of the node's algebra);
      // a product out of range falls back to the sum of logarithms
      double prod = 1.0;
      for (int k = 0; k < r2; ++k) prod *= Sj[k * R2 + k];
      double ls = 0.0;
      if (prod > 0.0 && prod < INFINITY && prod > 1e-300) {
        ls = log(prod);
      } else {
        for (int k = 0; k < r2; ++k) ls += log(Sj[k * R2 + k]);
      }
      thr_triinv_upper(Sj, R2, srv, Si + j * R2 * R2, R2, r2);
      const int nid = node_id(lvl, b0 + j), ld2 = 2 * cap;
      double* Zf = Fd->Zf + (size_t)nid * ld2 * ld2;
      double* Zi = Fd->Zi + (size_t)nid * ld2 * ld2;
      for (int a = 0; a < r2; ++a)
        for (int b = 0; b < r2; ++b) {
          const double d = (a == b) ? 1.0 : 0.0;
          Zf[a * ld2 + b] = (a >= b ? Sj[b * R2 + a] : 0.0) - d;
          Zi[a * ld2 + b] = (a >= b ? Si[j * R2 * R2 + b * R2 + a] : 0.0) - d;
        }
      Fd->ld_parts[nleaf + nid] = ls;
      if (!in[5]) atomicOr(Fd->status, FIFA_DEV_NOT_SPD);
      // ancestor columns of this node: prefix sums of the ancestor ranks
      int* rp = rpre + j * (FIFA_LEVELS_MAX + 1);
      int c = 0;
      for (int a = 0; a < lvl; ++a) {
        rp[a] = c;
        c += Fd->rank[node_id(a, (b0 + j) >> (lvl - a))];
      }
      rp[lvl] = c;
    }
  }
  __syncthreads();
  if (lvl == 0) return;
  int nmax = 0;
  for (int j = 0; j < NPC; ++j)
    if (info[j * 8 + 4]) nmax = max(nmax, rpre[j * (FIFA_LEVELS_MAX + 1) + lvl]);
  // B <- B + Q (L_S^-1 - I) Q^T B for every ancestor column, LM_W at a time;
  // the next chunk's columns are copied in (asynchronously for FP64 storage)
  // while the current chunk is projected and updated
  auto chunk_codes = [&](int c0, int* cc) {
    if (tid < NPC * LM_W) {
      const int j = tid / LM_W, w = tid % LM_W;
      const int* rp = rpre + j * (FIFA_LEVELS_MAX + 1);
      int code = -1;
      if (info[j * 8 + 4] && c0 + w < rp[lvl]) {
        const int c = c0 + w;
        int a = 0;
        while (rp[a + 1] <= c) ++a;
        code = (a << 8) | (c - rp[a]);
      }
      cc[tid] = code;
    }
  };
  auto chunk_stage = [&](const int* cc, T* B) {
    for (int t = tid; t < NPC * LM_W * 2 * MS; t += nt) {
      const int j = t / (LM_W * 2 * MS), w = (t / (2 * MS)) % LM_W, p = t % (2 * MS);
      const int code = cc[j * LM_W + w];
      const int* in = info + j * 8;
      if (code >= 0 && p < in[3] - in[1]) {
        const T* src = Qall + ((size_t)(code >> 8) * cap + (code & 255)) * n + in[1] + p;
        if constexpr (sizeof(T) == sizeof(double)) cp_async8((double*)(B + t), src);
        else B[t] = *src;
      } else {
        B[t] = (T)0;
      }
    }
  };
  if (NB == 2) {
    chunk_codes(0, ccode2);
    __syncthreads();
    chunk_stage(ccode2, Bs2);
    cp_async_commit();
  }
  for (int c0 = 0, k = 0; c0 < nmax; c0 += LM_W, ++k) {
    const int cur = NB == 2 ? (k & 1) : 0;
    const int* ccode = ccode2 + cur * NPC * LM_W;
    const T* Bs = Bs2 + (size_t)cur * NPC * LM_W * 2 * MS;
    if (NB == 2) {
      int* cnext = ccode2 + (cur ^ 1) * NPC * LM_W;
      T* bnext = Bs2 + (size_t)(cur ^ 1) * NPC * LM_W * 2 * MS;
      const bool more = c0 + LM_W < nmax;
      if (more) chunk_codes(c0 + LM_W, cnext);
      __syncthreads();
      if (more) chunk_stage(cnext, bnext);
      cp_async_commit();
      cp_async_wait_prev();  // this chunk's copies have landed
    } else {
      chunk_codes(c0, ccode2);
      __syncthreads();
      chunk_stage(ccode2, Bs2);
      cp_async_commit();
      cp_async_wait_all();
    }
    __syncthreads();
    // P[a][w] = Q^T B (rows a < r from the left child, r <= a < 2r from the right)
    for (int t = tid; t < NPC * R2 * LM_W; t += nt) {
      const int j = t / (R2 * LM_W), a = (t / LM_W) % R2, w = t % LM_W;
      const int* in = info + j * 8;
      const int r = in[0];
      T acc = (T)0;
      if (in[4] && ccode[j * LM_W + w] >= 0 && a < 2 * r) {
        const int side = a >= r, c = side ? a - r : a;
        const int m = side ? in[3] - in[2] : in[2] - in[1], off = side ? in[2] - in[1] : 0;
        const double* X = Xs + ((size_t)(j * 2 + side) * R + c) * MS;
        const T* B = Bs + ((size_t)j * LM_W + w) * 2 * MS + off;
        for (int p = 0; p < m; ++p) acc += (T)X[p] * B[p];
      }
      Pm[t] = (double)acc;
    }
    __syncthreads();
    // T = (L_S^-1 - I) P, in the node's compact 2r layout
    for (int t = tid; t < NPC * R2 * LM_W; t += nt) {
      const int j = t / (R2 * LM_W), a = (t / LM_W) % R2, w = t % LM_W;
      const int* in = info + j * 8;
      const int r = in[0];
      double v = 0.0;
      if (in[4] && a < 2 * r) {
        // a is the compact index of the 2r x 2r factor (a < r: left child, else right)
        const double* Sij = Si + j * R2 * R2;
        const double* P = Pm + (size_t)j * R2 * LM_W;
        v = -P[a * LM_W + w];
        for (int b = 0; b <= a; ++b) v += Sij[b * R2 + a] * P[b * LM_W + w];
      }
      Tm[t] = (T)v;
    }
    __syncthreads();
    // B += Q T, one thread per (node, column, row), written back
    for (int t = tid; t < NPC * LM_W * 2 * MS; t += nt) {
      const int j = t / (LM_W * 2 * MS), w = (t / (2 * MS)) % LM_W, p = t % (2 * MS);
      const int code = ccode[j * LM_W + w];
      const int* in = info + j * 8;
      const int mu = in[2] - in[1], mn = in[3] - in[1];
      if (code < 0 || p >= mn) continue;
      const int r = in[0], side = p >= mu, pp = side ? p - mu : p, toff = side ? r : 0;
      const double* X = Xs + (size_t)(j * 2 + side) * R * MS;
      const T* Tj = Tm + (size_t)j * R2 * LM_W;
      T acc = Bs[t];
      for (int a = 0; a < r; ++a) acc += (T)X[a * MS + pp] * Tj[(toff + a) * LM_W + w];
      Qall[((size_t)(code >> 8) * cap + (code & 255)) * n + in[1] + p] = acc;
    }
    __syncthreads();
  }
}

template <typename T, int R, int MS, int NPC>
static cudaError_t launch_level_multi(const FactDesc* Fd, int lvl, int nodes, cudaStream_t st, int nprob) {
  const size_t smem = LmLayout<R, MS, NPC>::bytes(sizeof(T));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_level_multi<T, R, MS, NPC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_level_multi<T, R, MS, NPC><<<dim3((nodes + NPC - 1) / NPC, nprob), 256, smem, st>>>(Fd, lvl, nodes);
  return cudaGetLastError();
}

__global__ void k_logdet_reduce(const FactDesc* __restrict__ Fd) {
  Fd += blockIdx.y;  // problem of a batched launch
  if (Fd->skip && *Fd->skip) return;
  __shared__ double red[40];
  const int cnt = Fd->nleaf + (1 << Fd->L) - 1;
  double v = 0.0;
#pragma unroll 8
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) v += Fd->ld_parts[t];  // eight loads in flight per thread
  v = block_sum(v, red);
  if (threadIdx.x == 0) Fd->logdet[0] = 2.0 * v;
}

// ---------------------------------------------------------------------------
size_t leaf_factor_smem(int Bm, int L, int cap, int prec) {
  const size_t ld = Bm + 1;
  size_t b = (size_t)Bm * ld * sizeof(double);                   // FP64 Cholesky
  if (prec) b += ((size_t)Bm * ld + 1) / 2 * sizeof(double);      // FP32 copy of L
  b += (size_t)lf_nch(Bm) * ld * (prec ? sizeof(float) : sizeof(double));  // right-hand sides
  b += 16 + 40 * sizeof(double) + (4 + (size_t)L * cap) * sizeof(int);
  return b;
}
size_t level_smem(int ldm, int cap) {
  const size_t W = LEVEL_W(ldm);
  return ((size_t)6 * ldm * ldm + 16 + 2 * (size_t)(ldm + W) * LV_TRP + 256 + LV_RED + 4 * (size_t)ldm * W) * sizeof(double) +
         W * sizeof(void*) + (4 + (size_t)FIFA_LEVELS_MAX * cap) * sizeof(int);
}

static int smem_optin() {
  static std::atomic<int> cached{-1};  // several host threads may launch at once
  int v = cached.load(std::memory_order_relaxed);
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 48 * 1024;
    cached.store(v, std::memory_order_relaxed);
  }
  return v;
}

template <typename T>
static cudaError_t launch_leaf_factor_t(const HmatDesc* Hd, const FactDesc* Fd, int nleaf, size_t smem, cudaStream_t st,
                                        int nprob) {
  if (smem > (size_t)smem_optin()) return cudaErrorInvalidConfiguration;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_leaf_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_leaf_factor<T><<<dim3(nleaf, nprob), 256, smem, st>>>(Hd, Fd);
  return cudaGetLastError();
}

// Factorizations are computed in FP64 (prec 0); an FP32 factor is only ever a
// rounded copy of an FP64 one (k_mixed.cu), never factored directly.
cudaError_t launch_leaf_factor(const HmatDesc* Hd, const FactDesc* Fd, int prec, int nleaf, int Bm, int L, int cap,
                               cudaStream_t st, int nprob) {
  if (prec != 0) return cudaErrorInvalidValue;
  size_t smem = leaf_factor_smem(Bm, L, cap, 0);
  return launch_leaf_factor_t<double>(Hd, Fd, nleaf, smem, st, nprob);
}

template <typename T, int RB, int RLO>
static cudaError_t launch_level_bucket(const FactDesc* Fd, int lvl, int nodes, int G, int cap, double* part,
                                       unsigned int* bar, int* abort_flag, int skip, cudaStream_t st, int nprob,
                                       size_t sstride) {
  const size_t smem = level_smem(RB > 0 ? RB : cap, cap);
  if (smem > (size_t)smem_optin()) return cudaErrorInvalidConfiguration;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_level<T, RB, RLO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nodes * G, nprob);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = G > 1 ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_level<T, RB, RLO>, Fd, lvl, G, part, bar, abort_flag, skip, sstride);
}

template <typename T>
static cudaError_t launch_level_t(const FactDesc* Fd, int lvl, int nodes, const int* G, int cap, double* part,
                                  unsigned int* bar, int bar_stride, int* abort_flag, int side_max, cudaStream_t st,
                                  int nprob, size_t sstride) {
  int skip = -1;
  if (G[0] == 1 && side_max <= 128) {  // (nodes this small are never split over CTAs)
    // small nodes: rank <= 4 several nodes per CTA, rank 5..8 one node per CTA
    // (static shared memory); larger nodes take the tiled bucket kernels below,
    // whose output-major Gram and projection passes use the lanes better
    cudaError_t e0 = side_max <= 32   ? launch_level_multi<T, 4, 32, 4>(Fd, lvl, nodes, st, nprob)
                     : side_max <= 64 ? launch_level_multi<T, 4, 64, 2>(Fd, lvl, nodes, st, nprob)
                                      : launch_level_multi<T, 4, 128, 1>(Fd, lvl, nodes, st, nprob);
    if (e0 != cudaSuccess) return e0;
    k_level_small<T, 8, 4, 128, 8><<<dim3(nodes, nprob), 128, 0, st>>>(Fd, lvl);
    skip = 8;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // rank buckets: (.., 4] and (4, 16] with small-matrix storage sized by the
  // bucket, then (16, cap]; a node's CTAs skip the launches of other buckets
  // (buckets entirely below the small kernels' ranks are not launched)
  cudaError_t e = cudaSuccess;
  if ((G[0] > 1 || G[1] > 1) && nodes <= 64) {
    // a top level with CTA groups has few nodes, often of both rank buckets:
    // one launch for every rank <= 16 instead of two launches that would each
    // leave the other bucket's groups idle (measured: the split is faster only
    // at levels of >= 128 nodes, which are mostly of one bucket)
    e = launch_level_bucket<T, 16, -1>(Fd, lvl, nodes, G[1], cap, part, bar + bar_stride, abort_flag, skip, st, nprob, sstride);
    if (e == cudaSuccess && cap > 16)
      e = launch_level_bucket<T, 0, 16>(Fd, lvl, nodes, G[2], cap, part, bar + 2 * bar_stride, abort_flag, skip, st, nprob, sstride);
    return e;
  }
  if (skip < 4) e = launch_level_bucket<T, 4, -1>(Fd, lvl, nodes, G[0], cap, part, bar, abort_flag, skip, st, nprob, sstride);
  if (e == cudaSuccess && cap > 4 && skip < 16)
    e = launch_level_bucket<T, 16, 4>(Fd, lvl, nodes, G[1], cap, part, bar + bar_stride, abort_flag, skip, st, nprob, sstride);
  if (e == cudaSuccess && cap > 16)
    e = launch_level_bucket<T, 0, 16>(Fd, lvl, nodes, G[2], cap, part, bar + 2 * bar_stride, abort_flag, skip, st, nprob, sstride);
  return e;
}

cudaError_t launch_level(const FactDesc* Fd, int prec, int lvl, int nodes, const int* G, int cap, double* part,
                         unsigned int* bar, int bar_stride, int* abort_flag, int side_max, cudaStream_t st, int nprob,
                         size_t sstride) {
  if (prec != 0) return cudaErrorInvalidValue;
  return launch_level_t<double>(Fd, lvl, nodes, G, cap, part, bar, bar_stride, abort_flag, side_max, st, nprob,
                                sstride);
}

template <typename T, int RB, int RLO>
static int level_bucket_per_sm(int cap) {
  const size_t smem = level_smem(RB > 0 ? RB : cap, cap);
  if (smem > (size_t)smem_optin()) return 0;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_level<T, RB, RLO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level<T, RB, RLO>, 256, smem) != cudaSuccess) per_sm = 0;
  cudaGetLastError();
  return per_sm;
}

int level_bucket_coresident(int prec, int b, int cap) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  (void)prec;  // factorizations run in FP64 only
  int per_sm = 0;
  if (b == 0) per_sm = level_bucket_per_sm<double, 4, -1>(cap);
  else if (b == 1)  // also launched as <16, -1> at levels with CTA groups
    per_sm = std::min(level_bucket_per_sm<double, 16, 4>(cap), level_bucket_per_sm<double, 16, -1>(cap));
  else per_sm = level_bucket_per_sm<double, 0, 16>(cap);
  return sms * per_sm;
}

cudaError_t launch_logdet_reduce(const FactDesc* Fd, cudaStream_t st, int nprob) {
  k_logdet_reduce<<<dim3(1, nprob), 1024, 0, st>>>(Fd);
  return cudaGetLastError();
}
