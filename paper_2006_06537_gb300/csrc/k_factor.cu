// Symmetric factorization A = W W^T, W = A_L A_{L-1} ... A_0, of a HODLR matrix
// (SI "HODLR decomposition and factorization", after Ambikasaran et al. 2014,
// Theorem 3.1) and its log-determinant (SI "Determinant computation speedup").
//
//  k_leaf_factor : per leaf, L_i = chol(scale * D_i + shift * I) in FP64 shared
//                  memory, log-det partial, and L_i^-1 applied to the rows of
//                  every ancestor basis lying in the leaf (the first transform).
//  k_level       : per node of one level (bottom-up), the orthonormal bases
//                  Q_U, Q_V of the transformed U~, V~ by CholeskyQR2 (two Gram
//                  passes; stable here because the column-scaled bases are
//                  well conditioned), R = R2 R1, L_S = chol(I + R X R^T),
//                  Zf = L_S - I, Zi = L_S^-1 - I, and the inverse node factor
//                  I + Q Zi Q^T applied to every ancestor basis on the node's rows.
//                  Small nodes: one CTA each.  Large nodes: G CTAs split the rows
//                  and exchange partial sums through bounded-spin group barriers.
#include "fifa_common.cuh"
#include "fifa_launch.h"

#define LF_NCH 32
#define LV_TR 32
#define LV_NC 16

template <typename T>
__global__ void __launch_bounds__(256) k_leaf_factor(const HmatDesc* __restrict__ Hd, const FactDesc* __restrict__ Fd) {
  extern __shared__ double sm[];
  const int leaf = blockIdx.x;
  const int L = Fd->L, Bm = Fd->Bm, cap = Fd->cap;
  const int64_t n = Fd->n;
  const double sc = Hd->scale, shf = Hd->shift;
  const int* bnd = Fd->bnd;
  const int s = bnd[bnd_off(L) + leaf], e = bnd[bnd_off(L) + leaf + 1], m = e - s;
  const int ld = Bm + 1;
  double* A = sm;                          // FP64 Cholesky, column-major A[j*ld + i]
  T* La = sizeof(T) == sizeof(double) ? (T*)A : (T*)(A + (size_t)Bm * ld);  // L in the TRSM precision
  T* X = (T*)(A + (size_t)Bm * ld + (sizeof(T) == sizeof(double) ? 0 : ((size_t)Bm * ld + 1) / 2));
  double* red = (double*)(X + (size_t)LF_NCH * ld) + 1;  // 40 doubles (8-byte aligned past X)
  red = (double*)(((uintptr_t)red) & ~(uintptr_t)7);
  int* flag = (int*)(red + 40);
  int* clist = flag + 4;                   // L * cap entries: (level << 8) | col
  const double* D = Hd->leaves + (size_t)leaf * Bm * Bm;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t % m, j = t / m;
    double v = __dmul_rn(sc, D[(size_t)j * Bm + i]);
    if (i == j) v = __dadd_rn(v, shf);
    A[j * ld + i] = v;
  }
  if (threadIdx.x == 0) flag[0] = 0;
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      double d = A[k * ld + k];
      if (!(d > 0.0)) { flag[0] = 1; d = 1.0; }
      A[k * ld + k] = sqrt(d);
    }
    __syncthreads();
    const double dk = A[k * ld + k];
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) A[k * ld + i] /= dk;
    __syncthreads();
    const int w = m - k - 1;
    for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
      int i = k + 1 + t % w, j = k + 1 + t / w;
      if (i >= j) A[j * ld + i] -= A[k * ld + i] * A[k * ld + j];
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
  T* Lout = (T*)Fd->Lleaf + (size_t)leaf * Bm * Bm;
  for (int t = threadIdx.x; t < Bm * Bm; t += blockDim.x) {
    int i = t % Bm, j = t / Bm;
    double v = (i < m && j < m && i >= j) ? A[j * ld + i] : 0.0;
    Lout[t] = (T)v;
  }
  if (sizeof(T) != sizeof(double)) {
    for (int t = threadIdx.x; t < m * ld; t += blockDim.x) La[t] = (T)A[t];
  }
  // column list of all ancestor bases restricted to this leaf
  __shared__ int ncols;
  if (threadIdx.x == 0) {
    int c = 0;
    for (int l = 0; l < L; ++l) {
      int a = node_of_row(bnd, l, s);
      int r = Hd->rank[node_id(l, a)];
      for (int q = 0; q < r; ++q) clist[c++] = (l << 8) | q;
    }
    ncols = c;
  }
  __syncthreads();
  const int nc = ncols;
  for (int c0 = 0; c0 < nc; c0 += LF_NCH) {
    const int w = min(LF_NCH, nc - c0);
    for (int t = threadIdx.x; t < w * m; t += blockDim.x) {
      int cc = t / m, i = t % m;
      int code = clist[c0 + cc], l = code >> 8, q = code & 255;
      int a = node_of_row(bnd, l, s);
      int as, ah, ae;
      node_range(bnd, l, a, as, ah, ae);
      double scl = (s < ah) ? sc : 1.0;  // U rows of the view are scaled
      double v = Hd->bases[((size_t)l * cap + q) * n + s + i];
      X[cc * ld + i] = (T)((scl == 1.0) ? v : __dmul_rn(scl, v));
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
      if (threadIdx.x < w) X[threadIdx.x * ld + k] /= La[k * ld + k];
      __syncthreads();
      const int rem = m - k - 1;
      for (int t = threadIdx.x; t < rem * w; t += blockDim.x) {
        int cc = t / rem, i = k + 1 + t % rem;
        X[cc * ld + i] -= La[k * ld + i] * X[cc * ld + k];
      }
      __syncthreads();
    }
    T* Q = (T*)Fd->Q;
    for (int t = threadIdx.x; t < w * m; t += blockDim.x) {
      int cc = t / m, i = t % m;
      int code = clist[c0 + cc], l = code >> 8, q = code & 255;
      Q[((size_t)l * cap + q) * n + s + i] = X[cc * ld + i];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Level kernel helpers.
// ---------------------------------------------------------------------------
// Partial Gram (upper triangle + mirror) of columns 0..r-1 of Xb over rows [a0, a1).
template <typename T>
__device__ void gram_rows(const T* Xb, int64_t n, int r, int a0, int a1, double* tile, double* out, int ld) {
  const int npair = r * (r + 1) / 2;
  double acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = 0.0;
  for (int p0 = a0; p0 < a1; p0 += LV_TR) {
    const int tr = min(LV_TR, a1 - p0);
    __syncthreads();
    for (int t = threadIdx.x; t < tr * r; t += blockDim.x) {
      int c = t / tr, p = t % tr;
      tile[p * FIFA_CAP_MAX + c] = to_d(Xb[(size_t)c * n + p0 + p]);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      int pr = threadIdx.x + q * blockDim.x;
      if (pr < npair) {
        int a = 0, rem = pr;
        while (rem >= r - a) { rem -= r - a; ++a; }
        int b = a + rem;
        double sacc = 0.0;
        for (int p = 0; p < tr; ++p) sacc += tile[p * FIFA_CAP_MAX + a] * tile[p * FIFA_CAP_MAX + b];
        acc[q] += sacc;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    int pr = threadIdx.x + q * blockDim.x;
    if (pr < npair) {
      int a = 0, rem = pr;
      while (rem >= r - a) { rem -= r - a; ++a; }
      int b = a + rem;
      out[a * ld + b] = acc[q];
      out[b * ld + a] = acc[q];
    }
  }
  __syncthreads();
}

// Xb rows [a0, a1) <- Xb rows * Ri (r x r upper), optionally accumulating the
// Gram matrix of the result into out (r x r, ld).
template <typename T>
__device__ void rowmul_rows(T* Xb, int64_t n, int r, int a0, int a1, const double* Ri, int ldr, double* tile,
                            double* tile2, double* out, int ld, bool gram) {
  const int npair = r * (r + 1) / 2;
  double acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = 0.0;
  for (int p0 = a0; p0 < a1; p0 += LV_TR) {
    const int tr = min(LV_TR, a1 - p0);
    __syncthreads();
    for (int t = threadIdx.x; t < tr * r; t += blockDim.x) {
      int c = t / tr, p = t % tr;
      tile[p * FIFA_CAP_MAX + c] = to_d(Xb[(size_t)c * n + p0 + p]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tr * r; t += blockDim.x) {
      int c = t / tr, p = t % tr;
      double v = 0.0;
      for (int a = 0; a <= c; ++a) v += tile[p * FIFA_CAP_MAX + a] * Ri[a * ldr + c];
      tile2[p * FIFA_CAP_MAX + c] = v;
      Xb[(size_t)c * n + p0 + p] = (T)v;
    }
    __syncthreads();
    if (gram) {
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        int pr = threadIdx.x + q * blockDim.x;
        if (pr < npair) {
          int a = 0, rem = pr;
          while (rem >= r - a) { rem -= r - a; ++a; }
          int b = a + rem;
          double sacc = 0.0;
          for (int p = 0; p < tr; ++p) {
            // use the stored (possibly rounded) values so Gram2 sees what Q holds
            double va = to_d((T)tile2[p * FIFA_CAP_MAX + a]), vb = to_d((T)tile2[p * FIFA_CAP_MAX + b]);
            sacc += va * vb;
          }
          acc[q] += sacc;
        }
      }
    }
  }
  if (gram) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      int pr = threadIdx.x + q * blockDim.x;
      if (pr < npair) {
        int a = 0, rem = pr;
        while (rem >= r - a) { rem -= r - a; ++a; }
        int b = a + rem;
        out[a * ld + b] = acc[q];
        out[b * ld + a] = acc[q];
      }
    }
  }
  __syncthreads();
}

// Reduce `count` doubles of the G partials of this group (slot order fixed)
// into dst; if G == 1 the partial already sits in dst.
__device__ inline bool group_reduce(double* dst, const double* src_local, int count, int G, int g, int base,
                                    double* part, size_t pstride, unsigned int* bar, unsigned int& phase,
                                    int* status, int* abort_flag) {
  if (G == 1) return true;
  // two slot sets alternate with the barrier count: a slot is rewritten only
  // after a later barrier that every reader of its previous contents has passed
  const size_t set = (size_t)(phase & 1u) * gridDim.x;
  double* mine = part + (set + base + g) * pstride;
  for (int t = threadIdx.x; t < count; t += blockDim.x) mine[t] = src_local[t];
  ++phase;
  if (!group_barrier(bar + base, (unsigned)G * phase, status, abort_flag)) return false;
  for (int t = threadIdx.x; t < count; t += blockDim.x) {
    double v = 0.0;
    for (int q = 0; q < G; ++q) v += __ldcg(part + (set + base + q) * pstride + t);
    dst[t] = v;
  }
  __syncthreads();
  return true;
}

template <typename T>
__global__ void __launch_bounds__(256) k_level(const FactDesc* __restrict__ Fd, int lvl, int G, double* __restrict__ part,
                                               unsigned int* __restrict__ bar, int* __restrict__ abort_flag) {
  extern __shared__ double sm[];
  const int bi = blockIdx.x / G, g = blockIdx.x % G, base = blockIdx.x - g;
  const int nid = node_id(lvl, bi);
  const int cap = Fd->cap, nleaf = Fd->nleaf;
  const int64_t n = Fd->n;
  const int* bnd = Fd->bnd;
  int s, h, e;
  node_range(bnd, lvl, bi, s, h, e);
  const int r = Fd->rank[nid];
  if (r == 0) {
    if (g == 0 && threadIdx.x == 0) Fd->ld_parts[nleaf + nid] = 0.0;
    return;
  }
  int* status = Fd->status;
  T* Qall = (T*)Fd->Q;
  T* Qb = Qall + (size_t)lvl * cap * n;
  const int len = e - s, rc = (len + G - 1) / G;
  const int r0 = s + min(len, g * rc), r1 = s + min(len, g * rc + rc);
  const int cc2 = cap * cap;
  double* Gm = sm;
  double* Ri = Gm + cc2;
  double* R1 = Ri + cc2;
  double* RU = R1 + cc2;
  double* RV = RU + cc2;
  double* tile = RV + cc2;                 // LV_TR x FIFA_CAP_MAX
  double* tile2 = tile + LV_TR * FIFA_CAP_MAX;
  double* Pm = tile2 + LV_TR * FIFA_CAP_MAX;  // 2cap x LV_NC
  double* red = Pm + 2 * cap * LV_NC;       // 40
  int* iflag = (int*)(red + 40);
  int* alist = iflag + 4;                  // ancestor columns (level << 8 | col)
  const size_t pstride = (size_t)max(cc2, 2 * cap * LV_NC);
  unsigned int phase = 0;
  bool ok = true;

  for (int side = 0; side < 2; ++side) {
    const int a0 = side == 0 ? max(r0, s) : max(r0, h);
    const int a1 = side == 0 ? min(r1, h) : min(r1, e);
    T* Xb = Qb;  // columns at Qb + c*n, rows a0..a1
    // Gram 1
    for (int t = threadIdx.x; t < cc2; t += blockDim.x) Gm[t] = 0.0;
    __syncthreads();
    if (a1 > a0) gram_rows<T>(Xb, n, r, a0, a1, tile, Gm, cap);
    if (!group_reduce(Gm, Gm, cc2, G, g, base, part, pstride, bar, phase, status, abort_flag)) return;
    ok = blk_chol_upper(Gm, cap, r, iflag) && ok;
    for (int t = threadIdx.x; t < cc2; t += blockDim.x) R1[t] = Gm[t];
    __syncthreads();
    blk_triinv_upper(Gm, cap, Ri, cap, r);
    // Q1 = X R1^-1 in place, and its Gram
    for (int t = threadIdx.x; t < cc2; t += blockDim.x) Gm[t] = 0.0;
    __syncthreads();
    if (a1 > a0) rowmul_rows<T>(Xb, n, r, a0, a1, Ri, cap, tile, tile2, Gm, cap, true);
    if (!group_reduce(Gm, Gm, cc2, G, g, base, part, pstride, bar, phase, status, abort_flag)) return;
    ok = blk_chol_upper(Gm, cap, r, iflag) && ok;
    blk_triinv_upper(Gm, cap, Ri, cap, r);
    double* Rs = side == 0 ? RU : RV;
    for (int t = threadIdx.x; t < cc2; t += blockDim.x) {
      int i = t / cap, j = t % cap;
      double v = 0.0;
      if (i < r && j < r && i <= j)
        for (int k = i; k <= j; ++k) v += Gm[i * cap + k] * R1[k * cap + j];
      Rs[t] = v;
    }
    __syncthreads();
    // Q = Q1 R2^-1 in place
    if (a1 > a0) rowmul_rows<T>(Xb, n, r, a0, a1, Ri, cap, tile, tile2, nullptr, cap, false);
  }
  if (!ok && g == 0 && threadIdx.x == 0) atomicOr(status, FIFA_DEV_NOT_SPD);

  // capacitance: S = I + R X R^T, L_S = chol(S) (computed by the group's first CTA)
  const int r2 = 2 * r, ld2 = 2 * cap;
  double* Zf = Fd->Zf + (size_t)nid * ld2 * ld2;
  double* Zi = Fd->Zi + (size_t)nid * ld2 * ld2;
  if (g == 0) {
    for (int t = threadIdx.x; t < r2 * r2; t += blockDim.x) {
      int a = t / r2, b = t % r2;
      double v = (a == b) ? 1.0 : 0.0;
      if (a < r && b >= r) {
        int bb = b - r;
        for (int k = 0; k < r; ++k) v += RU[a * cap + k] * RV[bb * cap + k];
      } else if (a >= r && b < r) {
        int aa = a - r;
        for (int k = 0; k < r; ++k) v += RV[aa * cap + k] * RU[b * cap + k];
      }
      Zf[a * ld2 + b] = v;
    }
    __syncthreads();
    bool ok2 = blk_chol_upper(Zf, ld2, r2, iflag);  // Zf <- R_S (upper), S = R_S^T R_S, L_S = R_S^T
    double ls = 0.0;
    for (int k = threadIdx.x; k < r2; k += blockDim.x) ls += log(Zf[k * ld2 + k]);
    ls = block_sum(ls, red);
    blk_triinv_upper(Zf, ld2, Zi, ld2, r2);         // Zi <- R_S^-1 (upper) = (L_S^-1)^T
    // transpose both in place and subtract I
    for (int t = threadIdx.x; t < r2 * r2; t += blockDim.x) {
      int a = t / r2, b = t % r2;
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
    if (!group_barrier(bar + base, (unsigned)G * phase, status, abort_flag)) return;
  }
  if (lvl == 0) return;

  // ancestor columns on this node's rows
  __shared__ int nanc;
  if (threadIdx.x == 0) {
    int c = 0;
    for (int j = 0; j < lvl; ++j) {
      int a = node_of_row(bnd, j, s);
      int rj = Fd->rank[node_id(j, a)];
      for (int q = 0; q < rj; ++q) alist[c++] = (j << 8) | q;
    }
    nanc = c;
  }
  __syncthreads();
  const int na = nanc;
  for (int c0 = 0; c0 < na; c0 += LV_NC) {
    const int w = min(LV_NC, na - c0);
    // P = Q^T B over own rows: rows < h -> P[0:r), rows >= h -> P[r:2r)
    for (int t = threadIdx.x; t < 2 * cap * LV_NC; t += blockDim.x) Pm[t] = 0.0;
    __syncthreads();
    for (int t = threadIdx.x; t < r2 * w; t += blockDim.x) {
      int a = t / w, cc = t % w;
      int code = alist[c0 + cc], jl = code >> 8, q = code & 255;
      const T* Bc = Qall + ((size_t)jl * cap + q) * n;
      int p0 = a < r ? max(r0, s) : max(r0, h);
      int p1 = a < r ? min(r1, h) : min(r1, e);
      const T* Qc = Qb + (size_t)(a < r ? a : a - r) * n;
      T acc = 0;
      for (int p = p0; p < p1; ++p) acc += Qc[p] * Bc[p];
      Pm[a * LV_NC + cc] = (double)acc;
    }
    __syncthreads();
    if (!group_reduce(Pm, Pm, 2 * cap * LV_NC, G, g, base, part, pstride, bar, phase, status, abort_flag)) return;
    // T = Zi P
    double tv[8];
    int cnt = 0;
    for (int t = threadIdx.x; t < r2 * w; t += blockDim.x) {
      int a = t / w, cc = t % w;
      double acc = 0.0;
      for (int b = 0; b < r2; ++b) acc += Zi[a * ld2 + b] * Pm[b * LV_NC + cc];
      tv[cnt++] = acc;
    }
    __syncthreads();
    cnt = 0;
    for (int t = threadIdx.x; t < r2 * w; t += blockDim.x) {
      int a = t / w, cc = t % w;
      Pm[a * LV_NC + cc] = tv[cnt++];
    }
    __syncthreads();
    // B += Q T over own rows (storage precision)
    T* Tt = (T*)tile2;  // 2cap x LV_NC copy of T in the storage precision
    for (int t = threadIdx.x; t < r2 * w; t += blockDim.x) {
      int a = t / w, cc = t % w;
      Tt[a * LV_NC + cc] = (T)Pm[a * LV_NC + cc];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < (r1 - r0) * w; t += blockDim.x) {
      int cc = t / (r1 - r0), p = r0 + t % (r1 - r0);
      int code = alist[c0 + cc], jl = code >> 8, q = code & 255;
      T* Bc = Qall + ((size_t)jl * cap + q) * n;
      const int off = p < h ? 0 : r;
      T acc = Bc[p];
      for (int a = 0; a < r; ++a) acc += Qb[(size_t)a * n + p] * Tt[(off + a) * LV_NC + cc];
      Bc[p] = acc;
    }
    __syncthreads();
  }
}

__global__ void k_logdet_reduce(const FactDesc* __restrict__ Fd) {
  __shared__ double red[40];
  const int cnt = Fd->nleaf + (1 << Fd->L) - 1;
  double v = 0.0;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) v += Fd->ld_parts[t];
  v = block_sum(v, red);
  if (threadIdx.x == 0) Fd->logdet[0] = 2.0 * v;
}

// ---------------------------------------------------------------------------
size_t leaf_factor_smem(int Bm, int L, int cap, int prec) {
  const size_t ld = Bm + 1;
  size_t b = (size_t)Bm * ld * sizeof(double);                   // FP64 Cholesky
  if (prec) b += ((size_t)Bm * ld + 1) / 2 * sizeof(double);      // FP32 copy of L
  b += (size_t)LF_NCH * ld * (prec ? sizeof(float) : sizeof(double));  // right-hand sides
  b += 16 + 40 * sizeof(double) + (4 + (size_t)L * cap) * sizeof(int);
  return b;
}
size_t level_smem(int cap) {
  return ((size_t)5 * cap * cap + 2 * LV_TR * FIFA_CAP_MAX + 2 * (size_t)cap * LV_NC + 40) * sizeof(double) +
         (4 + (size_t)FIFA_LEVELS_MAX * cap) * sizeof(int);
}
size_t level_part_stride(int cap) { return (size_t)(cap * cap > 2 * cap * LV_NC ? cap * cap : 2 * cap * LV_NC); }

static int smem_optin() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 48 * 1024;
  }
  return v;
}

template <typename T>
static cudaError_t launch_leaf_factor_t(const HmatDesc* Hd, const FactDesc* Fd, int nleaf, size_t smem, cudaStream_t st) {
  if (smem > (size_t)smem_optin()) return cudaErrorInvalidConfiguration;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_leaf_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_leaf_factor<T><<<nleaf, 256, smem, st>>>(Hd, Fd);
  return cudaGetLastError();
}

cudaError_t launch_leaf_factor(const HmatDesc* Hd, const FactDesc* Fd, int prec, int nleaf, int Bm, int L, int cap,
                               cudaStream_t st) {
  size_t smem = leaf_factor_smem(Bm, L, cap, prec);
  return prec ? launch_leaf_factor_t<float>(Hd, Fd, nleaf, smem, st) : launch_leaf_factor_t<double>(Hd, Fd, nleaf, smem, st);
}

template <typename T>
static cudaError_t launch_level_t(const FactDesc* Fd, int lvl, int nodes, int G, int cap, double* part, unsigned int* bar,
                                  int* abort_flag, cudaStream_t st) {
  const size_t smem = level_smem(cap);
  if (smem > (size_t)smem_optin()) return cudaErrorInvalidConfiguration;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_level<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nodes * G);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = G > 1 ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_level<T>, Fd, lvl, G, part, bar, abort_flag);
}

cudaError_t launch_level(const FactDesc* Fd, int prec, int lvl, int nodes, int G, int cap, double* part,
                         unsigned int* bar, int* abort_flag, cudaStream_t st) {
  return prec ? launch_level_t<float>(Fd, lvl, nodes, G, cap, part, bar, abort_flag, st)
              : launch_level_t<double>(Fd, lvl, nodes, G, cap, part, bar, abort_flag, st);
}

int level_max_coresident(int prec, int cap) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = level_smem(cap);
  if (smem > (size_t)smem_optin()) return 0;
  cudaError_t e;
  if (prec) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_level<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level<float>, 256, smem);
  } else {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_level<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level<double>, 256, smem);
  }
  if (e != cudaSuccess) per_sm = 1;
  return sms * per_sm;
}

cudaError_t launch_logdet_reduce(const FactDesc* Fd, cudaStream_t st) {
  k_logdet_reduce<<<1, 256, 0, st>>>(Fd);
  return cudaGetLastError();
}
