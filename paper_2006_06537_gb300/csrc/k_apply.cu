// Application kernels: W, W^T, W^-1, W^-T sweeps (SI: W = A_L ... A_0 with
// node factors I + Q Z Q^T) and the H-matrix product (leaf products plus the
// low-rank off-diagonal blocks), for nrhs column-major vectors.
#include <algorithm>

#include "fifa_common.cuh"
#include "fifa_launch.h"

#define SW_RHS_MAX 2

// ---------------------------------------------------------------------------
// Level sweep, pass 1: partial projections p = Q_side^T v over this CTA's rows
// of one node.  part[cta][(a) * nrhs + j], a < 2cap (a < r: left child rows).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_proj(const FactDesc* __restrict__ Fd, int lvl, int G,
                                                    const double* __restrict__ v, int nrhs, double* __restrict__ part,
                                                    const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int bi = blockIdx.x / G, g = blockIdx.x % G;
  const int nid = node_id(lvl, bi);
  const int r = Fd->rank[nid];
  if (r == 0) return;
  const int cap = Fd->cap;
  const int64_t n = Fd->n;
  int s, h, e;
  node_range(Fd->bnd, lvl, bi, s, h, e);
  const int len = e - s, rc = (len + G - 1) / G;
  const int r0 = s + min(len, g * rc), r1 = s + min(len, g * rc + rc);
  const T* Qb = (const T*)Fd->Q + (size_t)lvl * cap * n;
  __shared__ double red[40];
  double* out = part + (size_t)blockIdx.x * 2 * cap * SW_RHS_MAX;
  for (int side = 0; side < 2; ++side) {
    const int a0 = side == 0 ? max(r0, s) : max(r0, h);
    const int a1 = side == 0 ? min(r1, h) : min(r1, e);
    for (int a = 0; a < r; ++a) {
      const T* Qc = Qb + (size_t)a * n;
      for (int j = 0; j < nrhs; ++j) {
        const double* vj = v + (size_t)j * n;
        double acc = 0.0;
        for (int p = a0 + threadIdx.x; p < a1; p += blockDim.x) acc += to_d(Qc[p]) * vj[p];
        acc = block_sum(acc, red);
        if (threadIdx.x == 0) out[(side * r + a) * SW_RHS_MAX + j] = acc;
      }
    }
  }
}

// Pass 2: reduce the node's partials (fixed order), t = op(Z) p, v += Q t.
// zsel: 0 -> Zf, 1 -> Zi; ztrans: use the transpose.
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_upd(const FactDesc* __restrict__ Fd, int lvl, int G, double* __restrict__ v,
                                                   int nrhs, const double* __restrict__ part, int zsel, int ztrans,
                                                   const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int bi = blockIdx.x / G, g = blockIdx.x % G, base = blockIdx.x - g;
  const int nid = node_id(lvl, bi);
  const int r = Fd->rank[nid];
  if (r == 0) return;
  const int cap = Fd->cap;
  const int64_t n = Fd->n;
  int s, h, e;
  node_range(Fd->bnd, lvl, bi, s, h, e);
  const int len = e - s, rc = (len + G - 1) / G;
  const int r0 = s + min(len, g * rc), r1 = s + min(len, g * rc + rc);
  const T* Qb = (const T*)Fd->Q + (size_t)lvl * cap * n;
  const int r2 = 2 * r, ld2 = 2 * cap;
  const double* Z = (zsel ? Fd->Zi : Fd->Zf) + (size_t)nid * ld2 * ld2;
  __shared__ double pv[2 * FIFA_CAP_MAX * SW_RHS_MAX];
  __shared__ double tv[2 * FIFA_CAP_MAX * SW_RHS_MAX];
  for (int t = threadIdx.x; t < r2 * nrhs; t += blockDim.x) {
    int a = t / nrhs, j = t % nrhs;
    double acc = 0.0;
    for (int q = 0; q < G; ++q) acc += part[(size_t)(base + q) * 2 * cap * SW_RHS_MAX + a * SW_RHS_MAX + j];
    pv[a * SW_RHS_MAX + j] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < r2 * nrhs; t += blockDim.x) {
    int a = t / nrhs, j = t % nrhs;
    double acc = 0.0;
    for (int b = 0; b < r2; ++b) acc += (ztrans ? Z[b * ld2 + a] : Z[a * ld2 + b]) * pv[b * SW_RHS_MAX + j];
    tv[a * SW_RHS_MAX + j] = acc;
  }
  __syncthreads();
  for (int p = r0 + threadIdx.x; p < r1; p += blockDim.x) {
    const int off = p < h ? 0 : r;
    double acc[SW_RHS_MAX] = {0.0, 0.0};
    for (int a = 0; a < r; ++a) {
      double q = to_d(Qb[(size_t)a * n + p]);
      for (int j = 0; j < nrhs; ++j) acc[j] += q * tv[(off + a) * SW_RHS_MAX + j];
    }
    for (int j = 0; j < nrhs; ++j) v[(size_t)j * n + p] += acc[j];
  }
}

template <typename T, int N>
__device__ __forceinline__ T reg_sel(const T (&a)[N], int q) {
  T r = a[0];
#pragma unroll
  for (int t = 1; t < N; ++t)
    if (q == t) r = a[t];
  return r;
}

// ---------------------------------------------------------------------------
// Leaf step of one leaf by one warp, on m entries at vj (global or shared
// memory, element type V), in the factor's precision T (FP64, or FP32 for an
// FP32 copy of a factor: every product and sum in T).  mode 0: v <- L v, 1: v <- L^-1 v, 2: v <- L^T v, 3: v <- L^-T v.
// L column-major (L[i][k] at k*Bm + i, i >= k) with L^T mirrored into the
// upper triangle (L[k][j] at k*Bm + j, j < k): every step reads one contiguous
// column, L's for modes 0 / 1 and L^T's for modes 2 / 3.
// ---------------------------------------------------------------------------
template <typename T, typename V, int RPL>  // RPL: rows per lane, 32 RPL >= m; dinv: reciprocal pivots
__device__ __forceinline__ void leaf_warp_apply_r(const T* __restrict__ Lm, const T* __restrict__ dinv, int Bm,
                                                  int m, V* vj, int mode, int lane) {
  T x[RPL], o[RPL];
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    int i = lane + 32 * q;
    x[q] = i < m ? (T)vj[i] : (T)0;
    o[q] = (T)0;
  }
  if (mode == 0) {  // o_i = sum_{k<=i} L[i][k] x_k
    for (int k = 0; k < m; ++k) {
      T xk = __shfl_sync(0xffffffffu, reg_sel<T, RPL>(x, k >> 5), k & 31);
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        int i = lane + 32 * q;
        if (i >= k && i < m) o[q] += Lm[(size_t)k * Bm + i] * xk;
      }
    }
  } else if (mode == 1) {  // forward substitution
#pragma unroll
    for (int q = 0; q < RPL; ++q) o[q] = x[q];
    for (int k = 0; k < m; ++k) {
      const int qk = k >> 5;
      T ok = (T)0;
#pragma unroll
      for (int q = 0; q < RPL; ++q)
        if (q == qk) ok = o[q];
      T xk = __shfl_sync(0xffffffffu, ok, k & 31) * dinv[k];
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        int i = lane + 32 * q;
        if (i == k) o[q] = xk;
        else if (i > k && i < m) o[q] -= Lm[(size_t)k * Bm + i] * xk;
      }
    }
  } else if (mode == 2) {  // o_j = sum_{k>=j} L[k][j] x_k, right-looking over k
    // row k of L is column k of the stored upper triangle (L^T mirrored there):
    // coalesced, and no cross-lane sums
    for (int k = 0; k < m; ++k) {
      const T xk = __shfl_sync(0xffffffffu, reg_sel<T, RPL>(x, k >> 5), k & 31);
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int j = lane + 32 * q;
        if (j <= k) o[q] += Lm[(size_t)k * Bm + j] * xk;
      }
    }
  } else {  // backward substitution L^T x = v, column-oriented (x_k, then o_j -= L[k][j] x_k for j < k)
#pragma unroll
    for (int q = 0; q < RPL; ++q) o[q] = x[q];
    for (int k = m - 1; k >= 0; --k) {
      const int qk = k >> 5;
      T ok = (T)0;
#pragma unroll
      for (int q = 0; q < RPL; ++q)
        if (q == qk) ok = o[q];
      const T xk = __shfl_sync(0xffffffffu, ok, k & 31) * dinv[k];
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int j = lane + 32 * q;
        if (j == k) o[q] = xk;
        else if (j < k) o[q] -= Lm[(size_t)k * Bm + j] * xk;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    int i = lane + 32 * q;
    if (i < m) vj[i] = (V)o[q];
  }
}

// Leaves of at most 32 rows, both right-hand sides at once (v1 nullable).  Lane
// i holds the entries Lm[k Bm + i] of every column k it needs (L[i][k] below
// the diagonal, L[k][i] = L^T mirrored above it), loaded in chunks of CH
// columns before any of them is used, so a chunk's loads are in flight
// together instead of one dependent load per substitution step.  MODE as
// leaf_warp_apply_r.
template <typename T, typename V, int CH, int MODE>
__device__ __forceinline__ void leaf_warp_apply32_m(const T* __restrict__ Lm, const T* __restrict__ dinv, int Bm, int m,
                                                    V* v0, V* v1, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr bool subst = MODE == 1 || MODE == 3;
  const bool in = lane < Bm;
  const bool two = v1 != nullptr;
  const T x0 = lane < m ? (T)v0[lane] : (T)0;
  const T x1 = (two && lane < m) ? (T)v1[lane] : (T)0;
  const T dl = (subst && in) ? dinv[lane] : (T)1;
  T o0 = subst ? x0 : (T)0, o1 = subst ? x1 : (T)0;
  for (int t0 = 0; t0 < m; t0 += CH) {
    T Lc[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int k = MODE == 3 ? m - 1 - (t0 + u) : t0 + u;
      Lc[u] = (in && t0 + u < m) ? Lm[(size_t)k * Bm + lane] : (T)0;
    }
    const int cnt = min(CH, m - t0);
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (u < cnt) {
        const int k = MODE == 3 ? m - 1 - (t0 + u) : t0 + u;
        const T a = Lc[u];
        if (!subst) {  // mode 0: o_i += L[i][k] x_k (i >= k);  mode 2: o_j += L[k][j] x_k (j <= k)
          const T xk0 = __shfl_sync(FULL, x0, k), xk1 = __shfl_sync(FULL, x1, k);
          if (MODE == 0 ? (lane >= k && lane < m) : (lane <= k)) {
            o0 += a * xk0;
            o1 += a * xk1;
          }
        } else {  // mode 1: forward, mode 3: backward substitution with the reciprocal pivots
          const T dk = __shfl_sync(FULL, dl, k);
          const T xk0 = __shfl_sync(FULL, o0, k) * dk, xk1 = __shfl_sync(FULL, o1, k) * dk;
          if (lane == k) {
            o0 = xk0;
            o1 = xk1;
          } else if (MODE == 1 ? (lane > k && lane < m) : (lane < k)) {
            o0 -= a * xk0;
            o1 -= a * xk1;
          }
        }
      }
    }
  }
  if (lane < m) {
    v0[lane] = (V)o0;
    if (two) v1[lane] = (V)o1;
  }
}

template <typename T, typename V>
__device__ __forceinline__ void leaf_warp_apply32(const T* __restrict__ Lm, const T* __restrict__ dinv, int Bm, int m,
                                                  V* v0, V* v1, int mode, int lane) {
  constexpr int CH = sizeof(T) == 4 ? 16 : 8;  // register budget of the fused sweep (64 per thread)
  switch (mode) {
    case 0: leaf_warp_apply32_m<T, V, CH, 0>(Lm, dinv, Bm, m, v0, v1, lane); break;
    case 1: leaf_warp_apply32_m<T, V, CH, 1>(Lm, dinv, Bm, m, v0, v1, lane); break;
    case 2: leaf_warp_apply32_m<T, V, CH, 2>(Lm, dinv, Bm, m, v0, v1, lane); break;
    default: leaf_warp_apply32_m<T, V, CH, 3>(Lm, dinv, Bm, m, v0, v1, lane); break;
  }
}

template <typename T, typename V>
__device__ __forceinline__ void leaf_warp_apply(const T* __restrict__ Lm, const T* __restrict__ dinv, int Bm, int m,
                                                V* vj, int mode, int lane) {
  if (Bm <= 32) leaf_warp_apply_r<T, V, 1>(Lm, dinv, Bm, m, vj, mode, lane);
  else if (Bm <= 64) leaf_warp_apply_r<T, V, 2>(Lm, dinv, Bm, m, vj, mode, lane);
  else leaf_warp_apply_r<T, V, FIFA_LEAF_MAX / 32>(Lm, dinv, Bm, m, vj, mode, lane);
}

// Leaf step over all leaves: one warp per leaf.
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_leaf(const FactDesc* __restrict__ Fd, double* __restrict__ v, int nrhs,
                                                    int mode, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int L = Fd->L, Bm = Fd->Bm, nleaf = Fd->nleaf;
  if (warp >= nleaf) return;
  const int64_t n = Fd->n;
  const int s = Fd->bnd[bnd_off(L) + warp], e = Fd->bnd[bnd_off(L) + warp + 1];
  const T* Lm = (const T*)Fd->Lleaf + (size_t)warp * Bm * Bm;
  const T* dinv = (const T*)Fd->Ldinv + (size_t)warp * Bm;
  if (Bm <= 32) {
    leaf_warp_apply32<T, double>(Lm, dinv, Bm, e - s, v + s, nrhs > 1 ? v + n + s : nullptr,
                                                           mode, lane);
    return;
  }
  for (int j = 0; j < nrhs; ++j) leaf_warp_apply<T, double>(Lm, dinv, Bm, e - s, v + (size_t)j * n + s, mode, lane);
}

// ---------------------------------------------------------------------------
// Fused sweep: a whole W / W^-1 / W^T / W^-T application in one cooperative
// launch of 2^ls CTAs.  CTA c owns the rows [S, E) of the level-ls node c and
// keeps v on them in shared memory for the whole sweep, so v crosses HBM once
// each way.  The leaves and every level >= ls act inside one CTA (a node there
// lies in one CTA's rows); each level < ls exchanges one partial projection
// per CTA through `part` (two buffers alternating by level) around one grid
// barrier.  Same arithmetic as the per-level kernels above:
//   p = [Q_left^T v_left ; Q_right^T v_right],  t = op(Z) p,  v += Q t.
// ---------------------------------------------------------------------------
#define FS_WARPS 8
#define FS_K (2 * FIFA_CAP_MAX * SW_RHS_MAX)  // stride of one CTA's partial in `part`

// Ask L2 to fetch the 128-byte line holding p (no data is returned; p must
// point into an allocation).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Prefetch the basis columns a < r of level l on rows [a0, a1) into L2, the
// CTA's threads sharing the lines.
template <typename T>
__device__ __forceinline__ void prefetch_cols_l2(const T* __restrict__ Qb, int64_t n, int r, int a0, int a1) {
  constexpr int PER = 128 / (int)sizeof(T);
  const int first = a0 / PER, last = (a1 - 1) / PER;
  if (a1 <= a0) return;
  const int nl = last - first + 1;
  for (int t = threadIdx.x; t < r * nl; t += blockDim.x) {
    const int a = t / nl, li = first + t % nl;
    prefetch_l2(Qb + (size_t)a * n + (size_t)li * PER);
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over rows [a0, a1) of Bl[col][p] * xs[j][p - S] for K outputs
// o = (unit, c, j) described by fn(o, &a0, &a1, &col, &j) (col < 0: skip);
// results to out[o], accumulated in TX.  Threads take (output, row chunk)
// pairs; chunk partials are combined in a fixed order.
template <typename TB, typename TX, typename F>
__device__ void tile_dots(int K, const TB* __restrict__ Bl, int64_t n, const TX* xs, int rows, int S, F fn,
                          TX* red, TX* out) {
  const int nt = blockDim.x;
  const int nch = K >= nt ? 1 : nt / K;
  for (int o0 = 0; o0 < K; o0 += nt) {
    const int kk = min(nt, K - o0);
    const int ch = nch == 1 ? 0 : threadIdx.x / kk;
    const int o = o0 + (nch == 1 ? threadIdx.x : threadIdx.x % kk);
    TX acc = (TX)0;
    if ((nch == 1 && threadIdx.x < kk) || (nch > 1 && ch < nch)) {
      int a0, a1, col, j;
      fn(o, a0, a1, col, j);
      if (col >= 0) {
        const TB* b = Bl + (size_t)col * n;
        const TX* xj = xs + (size_t)j * rows - S;
#pragma unroll 8
        for (int p = a0 + ch; p < a1; p += nch) acc += (TX)b[p] * xj[p];
      }
    }
    __syncthreads();
    if (nch > 1) {
      if (ch < nch) red[ch * kk + (threadIdx.x % kk)] = acc;
      __syncthreads();
      if ((int)threadIdx.x < kk) {
        TX v = (TX)0;
        for (int q = 0; q < nch; ++q) v += red[q * kk + threadIdx.x];
        out[o0 + threadIdx.x] = v;
      }
    } else if ((int)threadIdx.x < kk) {
      out[o] = acc;
    }
    __syncthreads();
  }
}

#define FS_BUF 512  // entries of node projections (and of op(Z) p) per batch

// Shared scratch carved after v; T is the arithmetic type of the sweep.
template <typename T>
struct FsShared {
  T* pj;                  // FS_BUF: projections p of a batch of nodes
  T* tv;                  // FS_BUF: t = op(Z) p of the batch
  T* red;                 // 256 reduction partials
  unsigned short* lmap;   // rows: local leaf of each row
};

// basis columns whose loads a thread issues together (fewer FP64 ones: the
// register budget of the fused sweep is 64 per thread)
#define FS_RG_OF(T) (sizeof(T) == 4 ? 4 : 2)

// v_p += sum_{a < r} Q[a][p] t[a] for one row p (two right-hand sides in acc0,
// acc1; t interleaved by right-hand side), FS_RG_OF(T) loads in flight at a time.
template <typename T, int NR>
__device__ __forceinline__ void fs_row_update(const T* __restrict__ Qb, int64_t n, int p, int r, const T* tn, T& acc0,
                                              T& acc1) {
  constexpr int nrhs = NR;
  constexpr int RG = FS_RG_OF(T);
  for (int a0 = 0; a0 < r; a0 += RG) {
    T q[RG];
#pragma unroll
    for (int u = 0; u < RG; ++u) q[u] = a0 + u < r ? Qb[(size_t)(a0 + u) * n + p] : (T)0;
#pragma unroll
    for (int u = 0; u < RG; ++u) {
      if (a0 + u < r) {
        acc0 += q[u] * tn[(a0 + u) * nrhs];
        if (nrhs > 1) acc1 += q[u] * tn[(a0 + u) * nrhs + 1];
      }
    }
  }
}

// One level >= ls inside CTA c (rows [S, S + R)): the level's nodes in c's
// subtree in batches whose projections fit FS_BUF; each batch takes one pass of
// dot products (output-major, no cross-lane reductions), t = op(Z) p per
// node, and the row update v += Q t.  All arithmetic in T.
template <typename T, int NR>
__device__ void fs_local_level(const FactDesc* __restrict__ Fd, int l, int ls, int c, T* vs, int rows, int S,
                               int R, int zsel, int zt, FsShared<T>& sh) {
  constexpr int nrhs = NR;
  const int L = Fd->L, cap = Fd->cap, ld2 = 2 * cap;
  const int64_t n = Fd->n;
  const int* bnd = Fd->bnd;
  const int nsub = 1 << (l - ls), i0 = c << (l - ls);
  const T* Qb = (const T*)Fd->Q + (size_t)l * cap * n;
  int rmax = 0;
  for (int q = 0; q < nsub; ++q) rmax = max(rmax, Fd->rank[node_id(l, i0 + q)]);
  if (rmax == 0) return;
  const int per = 2 * rmax * nrhs;  // entries per node: (side, a, j)
  const int nb = max(1, FS_BUF / per);
  for (int b0 = 0; b0 < nsub; b0 += nb) {
    const int bn = min(nb, nsub - b0);
    tile_dots<T, T>(bn * per, Qb, n, vs, rows, S,
                    [&](int o, int& a0, int& a1, int& col, int& j) {
                      const int node = o / per, rem = o % per, side = rem / (rmax * nrhs), aj = rem % (rmax * nrhs);
                      const int a = aj / nrhs;
                      j = aj % nrhs;
                      int s0, h0, e0;
                      node_range(bnd, l, i0 + b0 + node, s0, h0, e0);
                      a0 = side ? h0 : s0;
                      a1 = side ? e0 : h0;
                      col = a < Fd->rank[node_id(l, i0 + b0 + node)] ? a : -1;
                    },
                    sh.red, sh.pj);
    for (int k = threadIdx.x; k < bn * per; k += blockDim.x) {
      const int node = k / per, rem = k % per, sa = rem / nrhs, j = rem % nrhs;
      const int side = sa / rmax, a = sa % rmax;
      const int nid = node_id(l, i0 + b0 + node);
      const int r = Fd->rank[nid];
      T acc = (T)0;
      if (a < r) {
        const double* Z = (zsel ? Fd->Zi : Fd->Zf) + (size_t)nid * ld2 * ld2;
        const int row = side * r + a;
        const T* pn = sh.pj + node * per;
        for (int bb = 0; bb < 2 * r; ++bb) {
          const int bs = bb >= r ? 1 : 0, ba = bb - bs * r;
          acc += (T)(zt ? Z[bb * ld2 + row] : Z[row * ld2 + bb]) * pn[(bs * rmax + ba) * nrhs + j];
        }
      }
      sh.tv[k] = acc;
    }
    __syncthreads();
    for (int p = S + (int)threadIdx.x; p < S + R; p += blockDim.x) {
      const int node = ((int)sh.lmap[p - S] >> (L - l)) - b0;
      if (node < 0 || node >= bn) continue;
      const int gi = i0 + b0 + node;
      const int r = Fd->rank[node_id(l, gi)];
      int s0, h0, e0;
      node_range(bnd, l, gi, s0, h0, e0);
      const T* tn = sh.tv + node * per + (p < h0 ? 0 : rmax) * nrhs;
      // the products accumulate onto v itself (no separate add per row)
      T acc0 = vs[p - S], acc1 = nrhs > 1 ? vs[rows + p - S] : (T)0;
      fs_row_update<T, NR>(Qb, n, p, r, tn, acc0, acc1);
      vs[p - S] = acc0;
      if (nrhs > 1) vs[rows + p - S] = acc1;
    }
    __syncthreads();
  }
}

// One level < ls: node i = c >> (ls - l) spans 2^(ls - l) CTAs; c's rows lie in
// one child (side).  The CTAs exchange their partial projections in FP64
// (`part`).  Returns false if the grid barrier gave up.
template <typename T, int NR>
__device__ bool fs_global_level(const FactDesc* __restrict__ Fd, int l, int ls, int c, T* vs, int rows, int S,
                                int E, int zsel, int zt, double* __restrict__ part, int buf,
                                unsigned int* bar, unsigned int& phase, int* abort_flag, FsShared<T>& sh,
                                int lnext) {
  constexpr int nrhs = NR;
  constexpr int RG = FS_RG_OF(T);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = gridDim.x;
  const int cap = Fd->cap, ld2 = 2 * cap;
  const int64_t n = Fd->n;
  const int span = ls - l, i = c >> span, side = (c >> (span - 1)) & 1;
  const int nid = node_id(l, i);
  const int r = Fd->rank[nid];
  const T* Qb = (const T*)Fd->Q + (size_t)l * cap * n;
  double* mine = part + ((size_t)buf * C + c) * FS_K;
  // partial projection of this CTA's rows onto its side's r columns: every
  // thread takes rows p = S + tid + 256 i and RG columns at a time (their
  // loads issued together), then a fixed-order block reduction
  for (int a0 = 0; a0 < r; a0 += RG) {
    T acc0[RG], acc1[RG];
#pragma unroll
    for (int u = 0; u < RG; ++u) acc0[u] = acc1[u] = (T)0;
#pragma unroll 2
    for (int p = S + (int)threadIdx.x; p < E; p += blockDim.x) {
      const T v0 = vs[p - S], v1 = nrhs > 1 ? vs[rows + p - S] : (T)0;
      T q[RG];
#pragma unroll
      for (int u = 0; u < RG; ++u) q[u] = a0 + u < r ? Qb[(size_t)(a0 + u) * n + p] : (T)0;
#pragma unroll
      for (int u = 0; u < RG; ++u) {
        if (a0 + u < r) {  // uniform over the CTA: no arithmetic on the columns past the rank
          acc0[u] += q[u] * v0;
          if (nrhs > 1) acc1[u] += q[u] * v1;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < RG; ++u) {
      if (a0 + u < r) {  // uniform: no reduction for the columns past the rank
        acc0[u] = warp_sum_t(acc0[u]);
        if (nrhs > 1) acc1[u] = warp_sum_t(acc1[u]);
      }
    }
    if (lane == 0)
#pragma unroll
      for (int u = 0; u < RG; ++u) {
        sh.red[(warp * RG + u) * 2] = acc0[u];
        sh.red[(warp * RG + u) * 2 + 1] = acc1[u];
      }
    __syncthreads();
    if ((int)threadIdx.x < RG * nrhs) {
      const int u = threadIdx.x / nrhs, j = threadIdx.x % nrhs;
      if (a0 + u < r) {
        T t = (T)0;
        for (int w = 0; w < FS_WARPS; ++w) t += sh.red[(w * RG + u) * 2 + j];
        __stcg(mine + (a0 + u) * nrhs + j, (double)t);
      }
    }
    __syncthreads();
  }
  (void)lane;
  if (sizeof(T) == 4 && lnext >= 0)  // FP32: the next level's basis rows, fetched into L2 while the grid waits
    prefetch_cols_l2<T>((const T*)Fd->Q + (size_t)lnext * cap * n, n, Fd->rank[node_id(lnext, c >> (ls - lnext))], S,
                        E);
  ++phase;
  if (!group_barrier(bar, (unsigned)C * phase, Fd->status, abort_flag, Fd->spin)) return false;
  if (r == 0) return true;
  // p over the node: the left half of its CTAs for rows of the left child, the
  // right half for the right child, summed in a fixed order
  const int K = 2 * r * nrhs, half = 1 << (span - 1), c0 = i << span;
  const int nch = blockDim.x / K;
  T* red = sh.red;
  if ((int)threadIdx.x < nch * K) {
    const int k = threadIdx.x % K, ch = threadIdx.x / K;
    const int sd = (k / nrhs) >= r ? 1 : 0, kk = k - sd * r * nrhs;
    const double* src = part + ((size_t)buf * C + c0 + sd * half) * FS_K + kk;
    double acc = 0.0;
    for (int q = ch; q < half; q += nch) acc += __ldcg(src + (size_t)q * FS_K);
    red[ch * K + k] = (T)acc;
  }
  __syncthreads();
  if ((int)threadIdx.x < K) {
    T acc = (T)0;
    for (int ch = 0; ch < nch; ++ch) acc += red[ch * K + threadIdx.x];
    sh.pj[threadIdx.x] = acc;
  }
  __syncthreads();
  if ((int)threadIdx.x < K) {
    const int a = threadIdx.x / nrhs, j = threadIdx.x % nrhs;
    const double* Z = (zsel ? Fd->Zi : Fd->Zf) + (size_t)nid * ld2 * ld2;
    T acc = (T)0;
    for (int b = 0; b < 2 * r; ++b) acc += (T)(zt ? Z[b * ld2 + a] : Z[a * ld2 + b]) * sh.pj[b * nrhs + j];
    sh.tv[threadIdx.x] = acc;
  }
  __syncthreads();
  const int off = side * r;
#pragma unroll 2
  for (int p = S + (int)threadIdx.x; p < E; p += blockDim.x) {
    T acc0 = vs[p - S], acc1 = nrhs > 1 ? vs[rows + p - S] : (T)0;
    fs_row_update<T, NR>(Qb, n, p, r, sh.tv + off * nrhs, acc0, acc1);
    vs[p - S] = acc0;
    if (nrhs > 1) vs[rows + p - S] = acc1;
  }
  __syncthreads();
  return true;
}

template <typename T, int NR>
__device__ void fs_leaves(const FactDesc* __restrict__ Fd, int ls, int c, T* vs, int rows, int S, int mode) {
  constexpr int nrhs = NR;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = Fd->L, Bm = Fd->Bm;
  const int nl = 1 << (L - ls), first = c << (L - ls);
  for (int q = warp; q < nl; q += FS_WARPS) {
    const int leaf = first + q;
    const int s = Fd->bnd[bnd_off(L) + leaf], e = Fd->bnd[bnd_off(L) + leaf + 1];
    const T* Lm = (const T*)Fd->Lleaf + (size_t)leaf * Bm * Bm;
    const T* dinv = (const T*)Fd->Ldinv + (size_t)leaf * Bm;
    if (Bm <= 32) {
      leaf_warp_apply32<T, T>(Lm, dinv, Bm, e - s, vs + (s - S),
                                                        nrhs > 1 ? vs + rows + (s - S) : nullptr, mode, lane);
      continue;
    }
    for (int j = 0; j < nrhs; ++j)
      leaf_warp_apply<T, T>(Lm, dinv, Bm, e - s, vs + (size_t)j * rows + (s - S), mode, lane);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Warp-owned subtrees.  Below the fused level ls every warp of the CTA owns
// the subtree of one level-lw node, lw = min(L, ls + FS_WL) (eight warps: three
// levels), and applies the leaves and the levels >= lw of that subtree alone:
// lanes stride over the node's rows, projections are reduced with warp
// shuffles, and no block barrier is passed.  Levels ls <= l < lw combine one
// partial projection per warp through shared memory with one block barrier
// per level.  The per-warp arrays: p and t of the current node (pj, 2 FS_WSL
// entries per warp) and the warp partials of the block levels (tv, two
// buffers alternating by level).  Ranks above FS_RFAST(T, NR) take the
// block-wide path instead.  FP32 only: in FP64 the shuffle reductions (two
// 32-bit shuffles and a DADD per step) cost more FP64 issue than the block
// barriers they replace (the FP64 W^-1 sweep at n = 2^20: 1.06 ms block-wide,
// 1.21 ms warp-owned).
// ---------------------------------------------------------------------------
#define FS_WARP_OWNED(T, NR) (sizeof(T) == 4)
#define FS_WL 3
#define FS_WSL 32                                           // p or t entries per warp: 2 r nrhs <= 32
#define FS_RFAST(T, NR) ((sizeof(T) == 4 ? 16 : 8) / (NR))  // ranks the warp path takes

template <typename T>
__device__ __forceinline__ T warp_allsum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// t = op(Z) p for a node of rank r: lane k < 2 r nrhs computes t[k]
// (k = (row, j)); p and t interleaved by right-hand side.
template <typename T, int NR>
__device__ __forceinline__ void fw_apply_z(const double* __restrict__ Z, int ld2, int r, int zt, const T* pw, T* tw,
                                           int lane) {
  constexpr int nrhs = NR;
  if (lane < 2 * r * nrhs) {
    const int row = lane / nrhs, j = lane % nrhs;
    T acc = (T)0;
    for (int b = 0; b < 2 * r; ++b) acc += (T)(zt ? Z[b * ld2 + row] : Z[row * ld2 + b]) * pw[b * nrhs + j];
    tw[lane] = acc;
  }
  __syncwarp();
}

// Projection of rows [a0, a1) onto the r columns of Qb, accumulated per lane
// (rows lane, lane + 32, ...) and reduced over the warp; every lane ends with
// the sums, lane 0 stores them at out[a nrhs + j].
template <typename T, int NR>
__device__ __forceinline__ void fw_project(const T* __restrict__ Qb, int64_t n, int r, const T* vs, int rows, int S,
                                           int a0, int a1, T* out, int lane) {
  constexpr int nrhs = NR;
  constexpr int CG = 8 / NR;  // columns per pass over the rows (registers: CG NR accumulators)
  for (int c0 = 0; c0 < r; c0 += CG) {
    T acc[CG][NR];
#pragma unroll
    for (int a = 0; a < CG; ++a)
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[a][j] = (T)0;
    for (int p = a0 + lane; p < a1; p += 32) {
      T v[NR];
#pragma unroll
      for (int j = 0; j < NR; ++j) v[j] = vs[(size_t)j * rows + p - S];
      T q[CG];
#pragma unroll
      for (int a = 0; a < CG; ++a) q[a] = c0 + a < r ? Qb[(size_t)(c0 + a) * n + p] : (T)0;
#pragma unroll
      for (int a = 0; a < CG; ++a)
        if (c0 + a < r)
#pragma unroll
          for (int j = 0; j < NR; ++j) acc[a][j] += q[a] * v[j];
    }
#pragma unroll
    for (int a = 0; a < CG; ++a)
      if (c0 + a < r)
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          const T t = warp_allsum(acc[a][j]);
          if (lane == 0) out[(c0 + a) * nrhs + j] = t;
        }
  }
}

// v_p += sum_a Q[a][p] t[(off + a) nrhs + j] for rows [a0, a1), lanes striding.
template <typename T, int NR>
__device__ __forceinline__ void fw_update(const T* __restrict__ Qb, int64_t n, int r, T* vs, int rows, int S, int a0,
                                          int a1, const T* tw, int off) {
  const int lane = threadIdx.x & 31;
#pragma unroll 2
  for (int p = a0 + lane; p < a1; p += 32) {
    T acc0 = vs[p - S], acc1 = NR > 1 ? vs[rows + p - S] : (T)0;
    fs_row_update<T, NR>(Qb, n, p, r, tw + off * NR, acc0, acc1);
    vs[p - S] = acc0;
    if (NR > 1) vs[rows + p - S] = acc1;
  }
}

// One node of a warp-owned level: projection of both sides, t = op(Z) p, update.
template <typename T, int NR>
__device__ void fw_node(const FactDesc* __restrict__ Fd, int l, int i, T* vs, int rows, int S, int zsel, int zt,
                        T* pw, T* tw, int lane) {
  const int cap = Fd->cap, ld2 = 2 * cap;
  const int64_t n = Fd->n;
  const int nid = node_id(l, i);
  const int r = Fd->rank[nid];
  if (r == 0) return;
  int s0, h0, e0;
  node_range(Fd->bnd, l, i, s0, h0, e0);
  const T* Qb = (const T*)Fd->Q + (size_t)l * cap * n;
  fw_project<T, NR>(Qb, n, r, vs, rows, S, s0, h0, pw, lane);
  fw_project<T, NR>(Qb, n, r, vs, rows, S, h0, e0, pw + r * NR, lane);
  __syncwarp();
  fw_apply_z<T, NR>((zsel ? Fd->Zi : Fd->Zf) + (size_t)nid * ld2 * ld2, ld2, r, zt, pw, tw, lane);
  fw_update<T, NR>(Qb, n, r, vs, rows, S, s0, h0, tw, 0);
  fw_update<T, NR>(Qb, n, r, vs, rows, S, h0, e0, tw, r);
  __syncwarp();
}

// The leaves and levels >= lw of warp w's subtree (root node wi at level lw),
// in the sweep's order: up = leaves first, then levels L-1 .. lw; else the
// levels lw .. L-1, then the leaves.
template <typename T, int NR>
__device__ void fw_subtree(const FactDesc* __restrict__ Fd, int lw, int wi, T* vs, int rows, int S, int mode, bool up,
                           int zsel, int zt, T* pw, T* tw, int lane) {
  const int L = Fd->L, Bm = Fd->Bm;
  auto leaves = [&]() {
    const int nl = 1 << (L - lw), first = wi << (L - lw);
    for (int q = 0; q < nl; ++q) {
      const int leaf = first + q;
      const int s = Fd->bnd[bnd_off(L) + leaf], e = Fd->bnd[bnd_off(L) + leaf + 1];
      const T* Lm = (const T*)Fd->Lleaf + (size_t)leaf * Bm * Bm;
      const T* dinv = (const T*)Fd->Ldinv + (size_t)leaf * Bm;
      if (Bm <= 32)
        leaf_warp_apply32<T, T>(Lm, dinv, Bm, e - s, vs + (s - S), NR > 1 ? vs + rows + (s - S) : nullptr, mode,
                                lane);
      else
        for (int j = 0; j < NR; ++j) leaf_warp_apply<T, T>(Lm, dinv, Bm, e - s, vs + (size_t)j * rows + (s - S), mode, lane);
      __syncwarp();
    }
  };
  if (up) {
    leaves();
    for (int l = L - 1; l >= lw; --l)
      for (int q = 0; q < (1 << (l - lw)); ++q) fw_node<T, NR>(Fd, l, (wi << (l - lw)) + q, vs, rows, S, zsel, zt, pw, tw, lane);
  } else {
    for (int l = lw; l < L; ++l)
      for (int q = 0; q < (1 << (l - lw)); ++q) fw_node<T, NR>(Fd, l, (wi << (l - lw)) + q, vs, rows, S, zsel, zt, pw, tw, lane);
    leaves();
  }
}

// One level ls <= l < lw: warp w's rows (those of its level-lw node) lie in
// one side of a level-l node; one partial per warp in shared memory, one block
// barrier, then every warp forms p from its node's warps (fixed order),
// t = op(Z) p and updates its own rows.  nsub: warps that own a subtree.
template <typename T, int NR>
__device__ void fw_block_level(const FactDesc* __restrict__ Fd, int l, int lw, int c, int nsub, T* vs, int rows,
                               int S, int zsel, int zt, T* part, T* pw, T* tw, int warp, int lane) {
  constexpr int nrhs = NR;
  const int cap = Fd->cap, ld2 = 2 * cap;
  const int64_t n = Fd->n;
  const bool own = warp < nsub;
  const int wi = (c * nsub) + warp;           // the warp's level-lw node
  const int span = lw - l, i = wi >> span;    // its level-l node
  const int nid = node_id(l, i);
  const int r = Fd->rank[nid];
  const T* Qb = (const T*)Fd->Q + (size_t)l * cap * n;
  if (own && r > 0) {
    const int a0 = Fd->bnd[bnd_off(lw) + wi], a1 = Fd->bnd[bnd_off(lw) + wi + 1];
    fw_project<T, NR>(Qb, n, r, vs, rows, S, a0, a1, part + warp * FS_WSL, lane);
  }
  __syncthreads();
  if (!own || r == 0) return;
  // warps of node i: [i << span, (i + 1) << span) - c nsub, left half first
  const int w0 = (i << span) - c * nsub, half = 1 << (span - 1);
  const int side = (wi >> (span - 1)) & 1;
  if (lane < 2 * r * nrhs) {
    const int sd = lane / (r * nrhs), k = lane % (r * nrhs);
    T acc = (T)0;
    for (int q = 0; q < half; ++q) acc += part[(w0 + sd * half + q) * FS_WSL + k];
    pw[lane] = acc;
  }
  __syncwarp();
  fw_apply_z<T, NR>((zsel ? Fd->Zi : Fd->Zf) + (size_t)nid * ld2 * ld2, ld2, r, zt, pw, tw, lane);
  const int a0 = Fd->bnd[bnd_off(lw) + wi], a1 = Fd->bnd[bnd_off(lw) + wi + 1];
  fw_update<T, NR>(Qb, n, r, vs, rows, S, a0, a1, tw, side * r);
  __syncwarp();
}

// mode 0: v <- W v, 1: W^-1 v, 2: W^T v, 3: W^-T v; mode 4: v <- W^-T W^-1 v
// (both inverse sweeps, v kept in shared memory in between: a full solve with
// the factor).  Arithmetic in T: FP64 for an FP64 factor, FP32 for an FP32
// copy (the global v stays FP64, converted on load and store).  active
// (nullable): when *active == 0 the launch does nothing (a converged
// iteration).  Dynamic shared memory: nrhs * rows entries of T (rows >= the
// longest level-ls node), then the FsShared arrays.  vlist (nullable): several
// factors of one plan in one launch, problem blockIdx.y: its descriptor
// Fd[blockIdx.y], its vector vlist[blockIdx.y], its partials, barrier and
// abort flag pstride bytes after the previous problem's.
template <typename T, int NR, bool BATCH = false>
__global__ void __launch_bounds__(256, 4) k_sweep_fused(const FactDesc* __restrict__ Fd, double* __restrict__ v,
                                                        int mode, int ls, int rows, double* __restrict__ part,
                                                        unsigned int* __restrict__ bar, int* __restrict__ abort_flag,
                                                        const int* __restrict__ active, double* const* vlist,
                                                        size_t pstride) {
  constexpr int nrhs = NR;
  if (active && *active == 0) return;
  // (a separate instantiation: re-pointed arguments live in registers for the
  // whole kernel, which the single-problem kernels cannot afford)
  if constexpr (BATCH) {
    Fd += blockIdx.y;
    v = vlist[blockIdx.y];
    part = (double*)((char*)part + blockIdx.y * pstride);
    bar = (unsigned int*)((char*)bar + blockIdx.y * pstride);
    abort_flag = (int*)((char*)abort_flag + blockIdx.y * pstride);
  }
  extern __shared__ __align__(16) unsigned char fs_smem[];
  T* vs = (T*)fs_smem;
  FsShared<T> sh;
  sh.pj = vs + (size_t)rows * nrhs;
  sh.tv = sh.pj + FS_BUF;
  sh.red = sh.tv + FS_BUF;
  sh.lmap = (unsigned short*)(sh.red + 256);
  const int c = blockIdx.x;
  const int L = Fd->L;
  const int64_t n = Fd->n;
  const int S = Fd->bnd[bnd_off(ls) + c], E = Fd->bnd[bnd_off(ls) + c + 1];
  // warp-owned subtrees when every rank of the CTA's levels >= ls is small
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lw = min(L, ls + FS_WL), nsub = 1 << (lw - ls);
  __shared__ int rk_big;
  if (threadIdx.x == 0) rk_big = 0;
  for (int j = 0; j < nrhs; ++j)
    for (int p = threadIdx.x; p < E - S; p += blockDim.x) vs[(size_t)j * rows + p] = (T)v[(size_t)j * n + S + p];
  __syncthreads();
  __shared__ int rml[FIFA_LEVELS_MAX];  // the largest rank of each local level in this CTA
  if constexpr (FS_WARP_OWNED(T, NR)) {
    for (int l = threadIdx.x; l < FIFA_LEVELS_MAX; l += blockDim.x) rml[l] = 0;
    __syncthreads();
    for (int l = ls; l < L; ++l)
      for (int q = threadIdx.x; q < (1 << (l - ls)); q += blockDim.x) {
        const int rq = Fd->rank[node_id(l, (c << (l - ls)) + q)];
        if (rq > FS_RFAST(T, NR)) rk_big = 1;
        atomicMax(&rml[l], rq);
      }
  }
  __syncthreads();
  // FP32: the CTA's basis rows of every local level, fetched into L2 ahead of
  // use (measured: 4% off the preconditioner solve; in FP64 the prefetches
  // cost more than they save)
  if constexpr (FS_WARP_OWNED(T, NR))
    for (int l = ls; l < L; ++l) prefetch_cols_l2<T>((const T*)Fd->Q + (size_t)l * Fd->cap * n, n, rml[l], S, E);
  const bool fast = FS_WARP_OWNED(T, NR) && !rk_big && nsub <= FS_WARPS;
  if (!fast) {  // the block-wide path: the local leaf of every row
    const int nl = 1 << (L - ls), first = c << (L - ls);
    for (int q = threadIdx.x; q < nl; q += blockDim.x) {
      const int s0 = Fd->bnd[bnd_off(L) + first + q], e0 = Fd->bnd[bnd_off(L) + first + q + 1];
      for (int p = s0; p < e0; ++p) sh.lmap[p - S] = (unsigned short)q;
    }
    __syncthreads();
  }
  unsigned int phase = 0;
  bool ok = true;
  T* pw = sh.pj + warp * 2 * FS_WSL;  // p of the warp's node
  T* tw = pw + FS_WSL;                // t of the warp's node
  auto local_up = [&](int md, int zsel, int zt) {
    if (!fast) {
      fs_leaves<T, NR>(Fd, ls, c, vs, rows, S, md);
      for (int l = L - 1; l >= ls; --l) fs_local_level<T, NR>(Fd, l, ls, c, vs, rows, S, E - S, zsel, zt, sh);
      return;
    }
    if constexpr (FS_WARP_OWNED(T, NR)) {
      if (warp < nsub)
        fw_subtree<T, NR>(Fd, lw, (c << (lw - ls)) + warp, vs, rows, S, md, true, zsel, zt, pw, tw, lane);
      for (int l = lw - 1; l >= ls; --l)
        fw_block_level<T, NR>(Fd, l, lw, c, nsub, vs, rows, S, zsel, zt, sh.tv + (l & 1) * FS_WARPS * FS_WSL, pw, tw,
                              warp, lane);
      __syncthreads();
    }
  };
  auto local_down = [&](int md, int zsel, int zt) {
    if (!fast) {
      for (int l = ls; l < L; ++l) fs_local_level<T, NR>(Fd, l, ls, c, vs, rows, S, E - S, zsel, zt, sh);
      fs_leaves<T, NR>(Fd, ls, c, vs, rows, S, md);
      return;
    }
    if constexpr (FS_WARP_OWNED(T, NR)) {
      for (int l = ls; l < lw; ++l)
        fw_block_level<T, NR>(Fd, l, lw, c, nsub, vs, rows, S, zsel, zt, sh.tv + (l & 1) * FS_WARPS * FS_WSL, pw, tw,
                              warp, lane);
      if (warp < nsub)
        fw_subtree<T, NR>(Fd, lw, (c << (lw - ls)) + warp, vs, rows, S, md, false, zsel, zt, pw, tw, lane);
      __syncthreads();
    }
  };
  auto up = [&](int md) {  // leaves first, then the levels upward (W^-1, W^T)
    const int zsel = md == 1 ? 1 : 0, zt = md == 2 ? 1 : 0;
    local_up(md, zsel, zt);
    for (int l = ls - 1; l >= 0 && ok; --l)
      ok = fs_global_level<T, NR>(Fd, l, ls, c, vs, rows, S, E, zsel, zt, part, phase & 1, bar, phase, abort_flag,
                              sh, l - 1);
  };
  auto down = [&](int md) {  // the levels downward, then the leaves (W, W^-T)
    const int zsel = md == 3 ? 1 : 0, zt = md == 3 ? 1 : 0;
    for (int l = 0; l < ls && ok; ++l)
      ok = fs_global_level<T, NR>(Fd, l, ls, c, vs, rows, S, E, zsel, zt, part, phase & 1, bar, phase, abort_flag,
                              sh, l + 1 < ls ? l + 1 : -1);
    if (ok) local_down(md, zsel, zt);
  };
  if (mode == 1 || mode == 2) {
    up(mode);
  } else if (mode == 5) {  // W^-1's leaves and levels >= ls only (no grid barrier)
    local_up(1, 1, 0);
  } else if (mode == 6) {  // W^-1's levels < ls only, on v that mode 5 left
    for (int l = ls - 1; l >= 0 && ok; --l)
      ok = fs_global_level<T, NR>(Fd, l, ls, c, vs, rows, S, E, 1, 0, part, phase & 1, bar, phase, abort_flag, sh,
                                  l - 1);
  } else if (mode == 4) {
    up(1);
    if (ok) down(3);
  } else {
    down(mode);
  }
  if (!ok) return;  // the status word carries TIMEOUT; v is left as it was
  for (int j = 0; j < nrhs; ++j)
    for (int p = threadIdx.x; p < E - S; p += blockDim.x) v[(size_t)j * n + S + p] = (double)vs[(size_t)j * rows + p];
}

size_t sweep_fused_smem(int rows, int nrhs, int prec) {
  const size_t esz = prec ? sizeof(float) : sizeof(double);
  return esz * ((size_t)rows * nrhs + 2 * FS_BUF + 256) + sizeof(unsigned short) * (size_t)rows;
}

template <typename T, int NR, bool BATCH = false>
static int sweep_fused_per_sm(size_t smem) {
  int per_sm = 0;
  cudaFuncSetAttribute(k_sweep_fused<T, NR, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_fused<T, NR, BATCH>, 256, smem) != cudaSuccess)
    per_sm = 0;
  cudaGetLastError();
  return per_sm;
}

int sweep_fused_coresident(int prec, int rows, int cap) {
  (void)cap;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = sweep_fused_smem(rows, SW_RHS_MAX, prec);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)optin) return 0;
  const int per_sm =
      prec ? std::min(sweep_fused_per_sm<float, 1>(smem), sweep_fused_per_sm<float, 2>(smem))
           : std::min(std::min(sweep_fused_per_sm<double, 1>(smem), sweep_fused_per_sm<double, 2>(smem)),
                      sweep_fused_per_sm<double, 1, true>(smem));
  return sms * per_sm;
}

template <typename T, int NR, bool BATCH = false>
static cudaError_t launch_sweep_fused_t(cudaLaunchConfig_t& cfg, const FactDesc* Fd, double* v, int mode, int ls,
                                        int rows, double* part, unsigned int* bar, int* abort_flag,
                                        const int* active, int prec, double* const* vlist = nullptr,
                                        size_t pstride = 0) {
  cudaFuncSetAttribute(k_sweep_fused<T, NR, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sweep_fused_smem(rows, SW_RHS_MAX, prec));
  return cudaLaunchKernelEx(&cfg, k_sweep_fused<T, NR, BATCH>, Fd, v, mode, ls, rows, part, bar, abort_flag, active,
                            vlist, pstride);
}

// nprob FP64 factors of one plan (descriptor array Fd), one right-hand side
// each at vlist[q], in one cooperative launch of 2^ls x nprob CTAs.
cudaError_t launch_sweep_fused_batched(const FactDesc* Fd, int ls, int rows, double* const* vlist, int nprob,
                                       int mode, double* part, unsigned int* bar, int* abort_flag, size_t pstride,
                                       cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1u << ls, nprob);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = sweep_fused_smem(rows, 1, 0);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return launch_sweep_fused_t<double, 1, true>(cfg, Fd, nullptr, mode, ls, rows, part, bar, abort_flag, nullptr, 0,
                                               vlist, pstride);
}

cudaError_t launch_sweep_fused(const FactDesc* Fd, int prec, int ls, int rows, int cap, double* v, int nrhs,
                               int mode, double* part, unsigned int* bar, int* abort_flag, cudaStream_t st,
                               const int* active) {
  (void)cap;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1u << ls);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = sweep_fused_smem(rows, nrhs, prec);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = mode == 5 ? 0 : 1;  // mode 5's CTAs never wait on each other
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (prec)
    return nrhs > 1 ? launch_sweep_fused_t<float, 2>(cfg, Fd, v, mode, ls, rows, part, bar, abort_flag, active, prec)
                    : launch_sweep_fused_t<float, 1>(cfg, Fd, v, mode, ls, rows, part, bar, abort_flag, active, prec);
  return nrhs > 1 ? launch_sweep_fused_t<double, 2>(cfg, Fd, v, mode, ls, rows, part, bar, abort_flag, active, prec)
                  : launch_sweep_fused_t<double, 1>(cfg, Fd, v, mode, ls, rows, part, bar, abort_flag, active, prec);
}

// ---------------------------------------------------------------------------
// Fused H-matrix product y = scale (C~ x) + shift x in one cooperative launch
// of 2^ls CTAs (the fused sweep's decomposition).  CTA c owns the rows [S, E)
// of level-ls node c: x on them sits in shared memory and each thread keeps
// the sums for its rows (S + tid + 256 i) in registers.  The leaf blocks and
// the levels >= ls (whose nodes lie in the CTA) need nothing from other CTAs;
// each level < ls needs the projection of the partner child, which spans
// other CTAs: every CTA writes its partial projections for all those levels,
// passes ONE grid barrier, and sums the partner half's partials.
//   row p in the left child of a level-l node:  y_p += U_p (V^T x_right)
//   row p in the right child:                   y_p += V_p (U^T x_left)
// (U, V share one basis array: row p holds U if p is in the left child.)
// ---------------------------------------------------------------------------
#define MV_PROJ_BUF 1024                       // doubles of node projections per batch
#define MV_PART_STRIDE (FIFA_CAP_MAX * SW_RHS_MAX)  // one CTA's partial of one level

// BATCH: several H-matrices of one plan in one launch, problem blockIdx.y: its
// descriptor Hd[blockIdx.y], input xlist[blockIdx.y] and output ylist[...],
// its partials, barrier and abort flag pstride bytes after the previous
// problem's (a separate instantiation: re-pointed arguments stay in registers).
template <int RPT, bool BATCH = false>
__global__ void __launch_bounds__(256, RPT <= 8 ? 4 : 2) k_mv_fused(const HmatDesc* __restrict__ Hd, const double* __restrict__ x, int nrhs,
                                                  double* __restrict__ y, int ls, int rows, double* __restrict__ part,
                                                  unsigned int* __restrict__ bar, int* __restrict__ abort_flag,
                                                  const int* __restrict__ active, const double* const* xlist,
                                                  double* const* ylist, size_t pstride) {
  if (active && *active == 0) return;  // a converged iteration: nothing to compute
  if constexpr (BATCH) {
    Hd += blockIdx.y;
    x = xlist[blockIdx.y];
    y = ylist[blockIdx.y];
    part = (double*)((char*)part + blockIdx.y * pstride);
    bar = (unsigned int*)((char*)bar + blockIdx.y * pstride);
    abort_flag = (int*)((char*)abort_flag + blockIdx.y * pstride);
  }
  extern __shared__ double sm[];
  double* xs = sm;                                   // nrhs x rows
  double* pj = xs + (size_t)rows * nrhs;             // MV_PROJ_BUF node projections
  double* red = pj + MV_PROJ_BUF;                    // 256 reduction partials
  int* lmap = (int*)(red + 256);                     // rows: local leaf of each row
  const int c = blockIdx.x, C = gridDim.x, tid = threadIdx.x;
  const int L = Hd->L, cap = Hd->cap, Bm = Hd->Bm;
  const int64_t n = Hd->n;
  const int* bnd = Hd->bnd;
  const int S = bnd[bnd_off(ls) + c], E = bnd[bnd_off(ls) + c + 1], R = E - S;
  for (int j = 0; j < nrhs; ++j)
    for (int p = tid; p < R; p += blockDim.x) xs[(size_t)j * rows + p] = x[(size_t)j * n + S + p];
  const int nl = 1 << (L - ls), first = c << (L - ls);
  for (int q = tid; q < nl; q += blockDim.x) {
    const int s0 = bnd[bnd_off(L) + first + q], e0 = bnd[bnd_off(L) + first + q + 1];
    for (int p = s0; p < e0; ++p) lmap[p - S] = q;
  }
  __syncthreads();
  double acc[RPT][SW_RHS_MAX];
#pragma unroll
  for (int i = 0; i < RPT; ++i) acc[i][0] = acc[i][1] = 0.0;
  // leaf blocks: y_p = sum_k D[p][k] x_k over the leaf of p
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int p = S + tid + i * (int)blockDim.x;
    if (p < E) {
      const int q = lmap[p - S], leaf = first + q;
      const int s0 = bnd[bnd_off(L) + leaf], e0 = bnd[bnd_off(L) + leaf + 1];
      const double* D = Hd->leaves + (size_t)leaf * Bm * Bm + (p - s0);
      double a0 = 0.0, a1 = 0.0;
      for (int k = s0; k < e0; ++k) {
        const double dv = D[(size_t)(k - s0) * Bm];
        a0 += dv * xs[k - S];
        if (nrhs > 1) a1 += dv * xs[rows + k - S];
      }
      acc[i][0] = a0;
      acc[i][1] = a1;
    }
  }
  // levels >= ls: nodes inside this CTA, in batches whose projections fit pj
  for (int l = ls; l < L; ++l) {
    const double* Bl = Hd->bases + (size_t)l * cap * n;
    const int nsub = 1 << (l - ls), i0 = c << (l - ls);
    int rmax = 0;
    for (int q = 0; q < nsub; ++q) rmax = max(rmax, Hd->rank[node_id(l, i0 + q)]);
    if (rmax == 0) continue;
    const int per = 2 * rmax * nrhs;  // projection entries per node: (side, c, j)
    const int nb = max(1, MV_PROJ_BUF / per);
    for (int b0 = 0; b0 < nsub; b0 += nb) {
      const int bn = min(nb, nsub - b0);
      tile_dots(bn * per, Bl, n, xs, rows, S,
              [&](int o, int& a0, int& a1, int& col, int& j) {
                const int node = o / per, rem = o % per, side = rem / (rmax * nrhs), cj = rem % (rmax * nrhs);
                const int cc = cj / nrhs;
                j = cj % nrhs;
                const int nid = node_id(l, i0 + b0 + node);
                int s0, h0, e0;
                node_range(bnd, l, i0 + b0 + node, s0, h0, e0);
                a0 = side ? h0 : s0;
                a1 = side ? e0 : h0;
                col = cc < Hd->rank[nid] ? cc : -1;
              },
              red, pj);
      // rows of the batch's nodes: y_p += basis_l[p] . proj(partner side)
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int p = S + tid + i * (int)blockDim.x;
        if (p < E) {
          const int node = (lmap[p - S] >> (L - l)) - b0;
          if (node >= 0 && node < bn) {
            const int gi = i0 + b0 + node;
            const int r = Hd->rank[node_id(l, gi)];
            int s0, h0, e0;
            node_range(bnd, l, gi, s0, h0, e0);
            const int other = p < h0 ? 1 : 0;
            const double* pr = pj + node * per + other * rmax * nrhs;
            double a0 = acc[i][0], a1 = acc[i][1];  // products accumulate onto the row sums
            for (int cc = 0; cc < r; ++cc) {
              const double bv = Bl[(size_t)cc * n + p];
              a0 += bv * pr[cc * nrhs];
              if (nrhs > 1) a1 += bv * pr[cc * nrhs + 1];
            }
            acc[i][0] = a0;
            acc[i][1] = a1;
          }
        }
      }
      __syncthreads();
    }
  }
  // levels < ls: partial projections of this CTA's rows for every such level
  for (int l = 0; l < ls; ++l) {
    const double* Bl = Hd->bases + (size_t)l * cap * n;
    const int r = Hd->rank[node_id(l, c >> (ls - l))];
    tile_dots(r * nrhs, Bl, n, xs, rows, S,
            [&](int o, int& a0, int& a1, int& col, int& j) {
              a0 = S;
              a1 = E;
              col = o / nrhs;
              j = o % nrhs;
            },
            red, pj);
    for (int k = tid; k < r * nrhs; k += blockDim.x) __stcg(part + ((size_t)c * ls + l) * MV_PART_STRIDE + k, pj[k]);
    __syncthreads();
  }
  if (ls > 0) {
    unsigned int phase = 1;
    if (!group_barrier(bar, (unsigned)C * phase, Hd->status, abort_flag, Hd->spin)) return;
  }
  // levels < ls: the partner half's projection, then the rows' sums
  for (int l = 0; l < ls; ++l) {
    const double* Bl = Hd->bases + (size_t)l * cap * n;
    const int span = ls - l, i = c >> span, side = (c >> (span - 1)) & 1;
    const int r = Hd->rank[node_id(l, i)];
    if (r == 0) continue;
    const int K = r * nrhs, half = 1 << (span - 1);
    const int c0 = (i << span) + (1 - side) * half;  // first CTA of the partner child
    const int nch = max(1, (int)blockDim.x / K);
    if (tid < nch * K) {
      const int k = tid % K, ch = tid / K;
      double v = 0.0;
      for (int q = ch; q < half; q += nch) v += __ldcg(part + ((size_t)(c0 + q) * ls + l) * MV_PART_STRIDE + k);
      red[ch * K + k] = v;
    }
    __syncthreads();
    if (tid < K) {
      double v = 0.0;
      for (int ch = 0; ch < nch; ++ch) v += red[ch * K + tid];
      pj[tid] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < RPT; ++ii) {
      const int p = S + tid + ii * (int)blockDim.x;
      if (p < E) {
        double a0 = acc[ii][0], a1 = acc[ii][1];
        for (int cc = 0; cc < r; ++cc) {
          const double bv = Bl[(size_t)cc * n + p];
          a0 += bv * pj[cc * nrhs];
          if (nrhs > 1) a1 += bv * pj[cc * nrhs + 1];
        }
        acc[ii][0] = a0;
        acc[ii][1] = a1;
      }
    }
    __syncthreads();
  }
  const double sc = Hd->scale, shf = Hd->shift;
  const double* dg = Hd->diag;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int p = S + tid + i * (int)blockDim.x;
    if (p < E) {
      const bool plain = !dg && shf == 0.0 && sc == 1.0;
      const double sh = dg ? dg[p] : shf;
      y[p] = plain ? acc[i][0] : sc * acc[i][0] + sh * xs[p - S];
      if (nrhs > 1) y[n + p] = plain ? acc[i][1] : sc * acc[i][1] + sh * xs[rows + p - S];
    }
  }
}

size_t mv_fused_smem(int rows) {
  return sizeof(double) * ((size_t)rows * SW_RHS_MAX + MV_PROJ_BUF + 256) + sizeof(int) * (size_t)rows;
}

template <int RPT, bool BATCH>
static int mv_fused_per_sm_v(int rows) {
  const size_t smem = mv_fused_smem(rows);
  int dev = 0, optin = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)optin) return 0;
  cudaFuncSetAttribute(k_mv_fused<RPT, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mv_fused<RPT, BATCH>, 256, smem) != cudaSuccess)
    per_sm = 0;
  cudaGetLastError();
  return per_sm;
}

// the smaller of the single-problem and the multi-problem instantiations
template <int RPT>
static int mv_fused_per_sm(int rows) {
  return std::min(mv_fused_per_sm_v<RPT, false>(rows), mv_fused_per_sm_v<RPT, true>(rows));
}

static int mv_rpt(int rows) {
  int rpt = 1;
  while (rpt * 256 < rows) rpt *= 2;
  return rpt;
}

int mv_fused_coresident(int rows) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  switch (mv_rpt(rows)) {
    case 1: return sms * mv_fused_per_sm<1>(rows);
    case 2: return sms * mv_fused_per_sm<2>(rows);
    case 4: return sms * mv_fused_per_sm<4>(rows);
    case 8: return sms * mv_fused_per_sm<8>(rows);
    case 16: return sms * mv_fused_per_sm<16>(rows);
    default: return 0;
  }
}

template <int RPT, bool BATCH = false>
static cudaError_t launch_mv_fused_t(const HmatDesc* Hd, int ls, int rows, const double* x, int nrhs, double* y,
                                     double* part, unsigned int* bar, int* abort_flag, cudaStream_t st,
                                     const int* active, const double* const* xlist = nullptr,
                                     double* const* ylist = nullptr, int nprob = 1, size_t pstride = 0) {
  const size_t smem = mv_fused_smem(rows);
  cudaFuncSetAttribute(k_mv_fused<RPT, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1u << ls, nprob);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_mv_fused<RPT, BATCH>, Hd, x, nrhs, y, ls, rows, part, bar, abort_flag, active,
                            xlist, ylist, pstride);
}

// nprob H-matrices of one plan (descriptor array Hd), one right-hand side each
// (xlist[q] -> ylist[q]), in one cooperative launch of 2^ls x nprob CTAs.
cudaError_t launch_mv_fused_batched(const HmatDesc* Hd, int ls, int rows, const double* const* xlist,
                                    double* const* ylist, int nprob, double* part, unsigned int* bar, int* abort_flag,
                                    size_t pstride, cudaStream_t st) {
#define MVB(R)                                                                                                    \
  launch_mv_fused_t<R, true>(Hd, ls, rows, nullptr, 1, nullptr, part, bar, abort_flag, st, nullptr, xlist, ylist, \
                             nprob, pstride)
  switch (mv_rpt(rows)) {
    case 1: return MVB(1);
    case 2: return MVB(2);
    case 4: return MVB(4);
    case 8: return MVB(8);
    case 16: return MVB(16);
    default: return cudaErrorInvalidValue;
  }
#undef MVB
}

cudaError_t launch_mv_fused(const HmatDesc* Hd, int ls, int rows, const double* x, int nrhs, double* y, double* part,
                            unsigned int* bar, int* abort_flag, cudaStream_t st, const int* active) {
  switch (mv_rpt(rows)) {
    case 1: return launch_mv_fused_t<1>(Hd, ls, rows, x, nrhs, y, part, bar, abort_flag, st, active);
    case 2: return launch_mv_fused_t<2>(Hd, ls, rows, x, nrhs, y, part, bar, abort_flag, st, active);
    case 4: return launch_mv_fused_t<4>(Hd, ls, rows, x, nrhs, y, part, bar, abort_flag, st, active);
    case 8: return launch_mv_fused_t<8>(Hd, ls, rows, x, nrhs, y, part, bar, abort_flag, st, active);
    case 16: return launch_mv_fused_t<16>(Hd, ls, rows, x, nrhs, y, part, bar, abort_flag, st, active);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// H-matrix product y = scale * C~ x + shift * x.
// Pass 1 (one CTA per leaf): per level, the projection of the leaf's rows onto
//   the level's basis: part[(leaf * L + l) * cap + c][j].
// Pass 2 (one CTA per level node side): sum of the partials of its leaves.
//   proj[((l-node) * 2 + side) * cap + c][j].
// Pass 3 (one CTA per leaf): y = scale (D x + sum_l basis_l proj_other) + shift x.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mv_proj(const HmatDesc* __restrict__ Hd, const double* __restrict__ x, int nrhs,
                                                 double* __restrict__ part, const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int leaf = blockIdx.x;
  const int L = Hd->L, cap = Hd->cap;
  const int64_t n = Hd->n;
  const int* bnd = Hd->bnd;
  const int s = bnd[bnd_off(L) + leaf], e = bnd[bnd_off(L) + leaf + 1], m = e - s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int l = 0; l < L; ++l) {
    const int r = Hd->rank[node_id(l, leaf >> (L - l))];  // level-l ancestor of the leaf
    for (int t = warp; t < r * nrhs; t += nw) {
      const int c = t / nrhs, j = t % nrhs;
      const double* bc = Hd->bases + ((size_t)l * cap + c) * n + s;
      const double* xj = x + (size_t)j * n + s;
      double acc = 0.0;
      for (int i = lane; i < m; i += 32) acc += bc[i] * xj[i];
      acc = warp_sum(acc);
      if (lane == 0) part[(((size_t)leaf * L + l) * cap + c) * SW_RHS_MAX + j] = acc;
    }
  }
}

__global__ void __launch_bounds__(256) k_mv_sum(const HmatDesc* __restrict__ Hd, int nrhs, const double* __restrict__ part,
                                                double* __restrict__ proj, const int* __restrict__ active) {
  if (active && *active == 0) return;
  // blockIdx.x enumerates (level node, side) pairs in heap order: 2 * node + side
  const int L = Hd->L, cap = Hd->cap;
  const int nid = blockIdx.x >> 1, side = blockIdx.x & 1;
  int l = 31 - __clz(nid + 1);
  const int i = nid + 1 - (1 << l);
  const int r = Hd->rank[nid];
  // leaves of this side: child node (l+1, 2i+side) spans 2^(L-l-1) leaves
  const int nl = 1 << (L - l - 1);
  const int first = (2 * i + side) * nl;
  __shared__ double red[40];
  for (int t = 0; t < r * nrhs; ++t) {
    const int c = t / nrhs, j = t % nrhs;
    double acc = 0.0;
    for (int q = threadIdx.x; q < nl; q += blockDim.x)
      acc += part[(((size_t)(first + q) * L + l) * cap + c) * SW_RHS_MAX + j];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) proj[(((size_t)nid * 2 + side) * cap + c) * SW_RHS_MAX + j] = acc;
  }
}

__global__ void __launch_bounds__(128) k_mv_expand(const HmatDesc* __restrict__ Hd, const double* __restrict__ x, int nrhs,
                                                   const double* __restrict__ proj, double* __restrict__ y,
                                                   const int* __restrict__ active) {
  if (active && *active == 0) return;
  const int leaf = blockIdx.x;
  const int L = Hd->L, cap = Hd->cap, Bm = Hd->Bm;
  const int64_t n = Hd->n;
  const int* bnd = Hd->bnd;
  const double sc = Hd->scale, shf = Hd->shift;
  const int s = bnd[bnd_off(L) + leaf], e = bnd[bnd_off(L) + leaf + 1], m = e - s;
  const double* D = Hd->leaves + (size_t)leaf * Bm * Bm;
  __shared__ double xs[FIFA_LEAF_MAX * SW_RHS_MAX];
  __shared__ double pr[FIFA_LEVELS_MAX * FIFA_CAP_MAX * SW_RHS_MAX];
  __shared__ int rk[FIFA_LEVELS_MAX];
  for (int t = threadIdx.x; t < m * nrhs; t += blockDim.x) {
    int i = t % m, j = t / m;
    xs[j * FIFA_LEAF_MAX + i] = x[(size_t)j * n + s + i];
  }
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    const int nid = node_id(l, leaf >> (L - l));           // level-l ancestor of the leaf
    rk[l] = Hd->rank[nid];
    const int other = ((leaf >> (L - l - 1)) & 1) ? 0 : 1;  // rows in the left child use V^T x_right
    for (int c = 0; c < rk[l]; ++c)
      for (int j = 0; j < nrhs; ++j)
        pr[(l * FIFA_CAP_MAX + c) * SW_RHS_MAX + j] = proj[(((size_t)nid * 2 + other) * cap + c) * SW_RHS_MAX + j];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double acc[SW_RHS_MAX] = {0.0, 0.0};
    for (int k = 0; k < m; ++k) {
      double d = D[(size_t)k * Bm + i];
      for (int j = 0; j < nrhs; ++j) acc[j] += d * xs[j * FIFA_LEAF_MAX + k];
    }
    for (int l = 0; l < L; ++l) {
      const double* bl = Hd->bases + (size_t)l * cap * n + s + i;
      for (int c = 0; c < rk[l]; ++c) {
        double b = bl[(size_t)c * n];
        for (int j = 0; j < nrhs; ++j) acc[j] += b * pr[(l * FIFA_CAP_MAX + c) * SW_RHS_MAX + j];
      }
    }
    for (int j = 0; j < nrhs; ++j) {
      double xv = xs[j * FIFA_LEAF_MAX + i];
      const double sh = Hd->diag ? Hd->diag[s + i] : shf;
      y[(size_t)j * n + s + i] = (!Hd->diag && shf == 0.0 && sc == 1.0) ? acc[j] : sc * acc[j] + sh * xv;
    }
  }
}

// ---------------------------------------------------------------------------
cudaError_t launch_sweep_level(const FactDesc* Fd, int prec, int lvl, int nodes, int G, double* v, int nrhs, double* part,
                               int zsel, int ztrans, cudaStream_t st, const int* active) {
  const int grid = nodes * G;
  if (prec) {
    k_sweep_proj<float><<<grid, 256, 0, st>>>(Fd, lvl, G, v, nrhs, part, active);
    k_sweep_upd<float><<<grid, 256, 0, st>>>(Fd, lvl, G, v, nrhs, part, zsel, ztrans, active);
  } else {
    k_sweep_proj<double><<<grid, 256, 0, st>>>(Fd, lvl, G, v, nrhs, part, active);
    k_sweep_upd<double><<<grid, 256, 0, st>>>(Fd, lvl, G, v, nrhs, part, zsel, ztrans, active);
  }
  return cudaGetLastError();
}

cudaError_t launch_sweep_leaf(const FactDesc* Fd, int prec, int nleaf, double* v, int nrhs, int mode, cudaStream_t st,
                              const int* active) {
  const int grid = (nleaf * 32 + 255) / 256;
  if (prec) k_sweep_leaf<float><<<grid, 256, 0, st>>>(Fd, v, nrhs, mode, active);
  else k_sweep_leaf<double><<<grid, 256, 0, st>>>(Fd, v, nrhs, mode, active);
  return cudaGetLastError();
}

cudaError_t launch_matvec(const HmatDesc* Hd, int nleaf, int L, const double* x, int nrhs, double* part, double* proj,
                          double* y, cudaStream_t st, const int* active) {
  if (L > 0) {
    k_mv_proj<<<nleaf, 256, 0, st>>>(Hd, x, nrhs, part, active);
    k_mv_sum<<<2 * ((1 << L) - 1), 256, 0, st>>>(Hd, nrhs, part, proj, active);
  }
  k_mv_expand<<<nleaf, 128, 0, st>>>(Hd, x, nrhs, proj, y, active);
  return cudaGetLastError();
}
