// Application kernels: W, W^T, W^-1, W^-T sweeps (SI: W = A_L ... A_0 with
// node factors I + Q Z Q^T) and the H-matrix product (leaf products plus the
// low-rank off-diagonal blocks), for nrhs column-major vectors.
#include "fifa_common.cuh"
#include "fifa_launch.h"

#define SW_RHS_MAX 2

// ---------------------------------------------------------------------------
// Level sweep, pass 1: partial projections p = Q_side^T v over this CTA's rows
// of one node.  part[cta][(a) * nrhs + j], a < 2cap (a < r: left child rows).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_proj(const FactDesc* __restrict__ Fd, int lvl, int G,
                                                    const double* __restrict__ v, int nrhs, double* __restrict__ part) {
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
                                                   int nrhs, const double* __restrict__ part, int zsel, int ztrans) {
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

template <int N>
__device__ __forceinline__ double reg_sel(const double (&a)[N], int q) {
  double r = a[0];
#pragma unroll
  for (int t = 1; t < N; ++t)
    if (q == t) r = a[t];
  return r;
}

// ---------------------------------------------------------------------------
// Leaf step: one warp per leaf.  mode 0: v <- L v, 1: v <- L^-1 v,
// 2: v <- L^T v, 3: v <- L^-T v.  L column-major (L[i][k] at k*Bm + i).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_leaf(const FactDesc* __restrict__ Fd, double* __restrict__ v, int nrhs, int mode) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int L = Fd->L, Bm = Fd->Bm, nleaf = Fd->nleaf;
  if (warp >= nleaf) return;
  const int64_t n = Fd->n;
  const int s = Fd->bnd[bnd_off(L) + warp], e = Fd->bnd[bnd_off(L) + warp + 1], m = e - s;
  const T* Lm = (const T*)Fd->Lleaf + (size_t)warp * Bm * Bm;
  constexpr int RPL = FIFA_LEAF_MAX / 32;  // rows per lane
  for (int j = 0; j < nrhs; ++j) {
    double* vj = v + (size_t)j * n + s;
    double x[RPL], o[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      int i = lane + 32 * q;
      x[q] = i < m ? vj[i] : 0.0;
      o[q] = 0.0;
    }
    if (mode == 0) {  // o_i = sum_{k<=i} L[i][k] x_k
      for (int k = 0; k < m; ++k) {
        double xk = __shfl_sync(0xffffffffu, reg_sel<RPL>(x, k >> 5), k & 31);
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          int i = lane + 32 * q;
          if (i >= k && i < m) o[q] += to_d(Lm[(size_t)k * Bm + i]) * xk;
        }
      }
    } else if (mode == 1) {  // forward substitution
#pragma unroll
      for (int q = 0; q < RPL; ++q) o[q] = x[q];
      for (int k = 0; k < m; ++k) {
        const int qk = k >> 5;
        double ok = 0.0;
#pragma unroll
        for (int q = 0; q < RPL; ++q)
          if (q == qk) ok = o[q];
        double xk = __shfl_sync(0xffffffffu, ok, k & 31) / to_d(Lm[(size_t)k * Bm + k]);
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          int i = lane + 32 * q;
          if (i == k) o[q] = xk;
          else if (i > k && i < m) o[q] -= to_d(Lm[(size_t)k * Bm + i]) * xk;
        }
      }
    } else if (mode == 2) {  // o_j = sum_{k>=j} L[k][j] x_k (column j contiguous)
      for (int jj = 0; jj < m; ++jj) {
        double part = 0.0;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          int k = lane + 32 * q;
          if (k >= jj && k < m) part += to_d(Lm[(size_t)jj * Bm + k]) * x[q];
        }
        part = warp_sum(part);
        part = __shfl_sync(0xffffffffu, part, 0);
#pragma unroll
        for (int q = 0; q < RPL; ++q)
          if (lane + 32 * q == jj) o[q] = part;
      }
    } else {  // backward substitution L^T x = v
      for (int jj = m - 1; jj >= 0; --jj) {
        double part = 0.0;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          int k = lane + 32 * q;
          if (k > jj && k < m) part += to_d(Lm[(size_t)jj * Bm + k]) * o[q];
        }
        part = warp_sum(part);
        part = __shfl_sync(0xffffffffu, part, 0);
        const double xj = (__shfl_sync(0xffffffffu, reg_sel<RPL>(x, jj >> 5), jj & 31) - part) /
                          to_d(Lm[(size_t)jj * Bm + jj]);
#pragma unroll
        for (int q = 0; q < RPL; ++q)
          if (lane + 32 * q == jj) o[q] = xj;
      }
    }
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      int i = lane + 32 * q;
      if (i < m) vj[i] = o[q];
    }
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
                                                 double* __restrict__ part) {
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
                                                double* __restrict__ proj) {
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
                                                   const double* __restrict__ proj, double* __restrict__ y) {
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
      y[(size_t)j * n + s + i] = (shf == 0.0 && sc == 1.0) ? acc[j] : sc * acc[j] + shf * xv;
    }
  }
}

// ---------------------------------------------------------------------------
cudaError_t launch_sweep_level(const FactDesc* Fd, int prec, int lvl, int nodes, int G, double* v, int nrhs, double* part,
                               int zsel, int ztrans, cudaStream_t st) {
  const int grid = nodes * G;
  if (prec) {
    k_sweep_proj<float><<<grid, 256, 0, st>>>(Fd, lvl, G, v, nrhs, part);
    k_sweep_upd<float><<<grid, 256, 0, st>>>(Fd, lvl, G, v, nrhs, part, zsel, ztrans);
  } else {
    k_sweep_proj<double><<<grid, 256, 0, st>>>(Fd, lvl, G, v, nrhs, part);
    k_sweep_upd<double><<<grid, 256, 0, st>>>(Fd, lvl, G, v, nrhs, part, zsel, ztrans);
  }
  return cudaGetLastError();
}

cudaError_t launch_sweep_leaf(const FactDesc* Fd, int prec, int nleaf, double* v, int nrhs, int mode, cudaStream_t st) {
  const int grid = (nleaf * 32 + 255) / 256;
  if (prec) k_sweep_leaf<float><<<grid, 256, 0, st>>>(Fd, v, nrhs, mode);
  else k_sweep_leaf<double><<<grid, 256, 0, st>>>(Fd, v, nrhs, mode);
  return cudaGetLastError();
}

cudaError_t launch_matvec(const HmatDesc* Hd, int nleaf, int L, const double* x, int nrhs, double* part, double* proj,
                          double* y, cudaStream_t st) {
  if (L > 0) {
    k_mv_proj<<<nleaf, 256, 0, st>>>(Hd, x, nrhs, part);
    k_mv_sum<<<2 * ((1 << L) - 1), 256, 0, st>>>(Hd, nrhs, part, proj);
  }
  k_mv_expand<<<nleaf, 128, 0, st>>>(Hd, x, nrhs, proj, y);
  return cudaGetLastError();
}
