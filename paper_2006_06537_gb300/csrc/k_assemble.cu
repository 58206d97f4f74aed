// HODLR assembly kernels: dense leaves and partial-pivoted ACA of every
// off-diagonal block (Sec. 3.2; "partial-pivoted LU" in the proof of Lemma 1).
#include "fifa_common.cuh"
#include "fifa_launch.h"

// ---------------------------------------------------------------------------
// Leaf assembly: leaves[leaf](a, b) = k(x_a, x_b) + nugget [a == b], padding 0.
// One CTA per leaf.  Kernel entries are evaluated once per unordered pair:
// diagonal tiles over their lower triangle, off-diagonal tiles mirrored through
// a shared-memory tile so both stores stay coalesced.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_leaf_assemble(const HmatDesc* __restrict__ Hd) {
  Hd += blockIdx.y;  // problem of a batched launch (descriptor arrays)
  const int leaf = blockIdx.x;
  const int L = Hd->L, Bm = Hd->Bm, kind = Hd->kind;
  const double kc = Hd->kc, nug = Hd->nugget;
  const int* bnd = Hd->bnd;
  const double* x = Hd->x;
  double* D = Hd->leaves + (size_t)leaf * Bm * Bm;
  const int s = bnd[bnd_off(L) + leaf], e = bnd[bnd_off(L) + leaf + 1], m = e - s;
  __shared__ double xs[FIFA_LEAF_MAX];
  __shared__ double tile[32][33];
  for (int a = threadIdx.x; a < m; a += blockDim.x) xs[a] = x[s + a];
  __syncthreads();
  const int nt = (Bm + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  // diagonal 32 x 32 tiles: entries (a, b) with a >= b only, mirrored (the
  // kernel is symmetric bit for bit: fl(xa - xb) = -fl(xb - xa))
  for (int bd = 0; bd < nt; ++bd) {
    for (int t = threadIdx.x; t < 32 * 33 / 2; t += blockDim.x) {
      int ia = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      if ((ia + 1) * (ia + 2) / 2 <= t) ++ia;
      if (ia * (ia + 1) / 2 > t) --ia;
      const int ib = t - ia * (ia + 1) / 2;
      const int a = 32 * bd + ia, b = 32 * bd + ib;
      double v = 0.0;
      if (a < m && b < m) {
        v = kern_entry(kind, kc, xs[a], xs[b]);
        if (a == b) v = __dadd_rn(v, nug);
      }
      if (a < Bm && b < Bm) {
        D[(size_t)b * Bm + a] = v;
        D[(size_t)a * Bm + b] = v;
      }
    }
  }
  for (int bj = 0; bj < nt; ++bj) {
    for (int bi = bj + 1; bi < nt; ++bi) {
      // tile rows a in [32 bi, +32), cols b in [32 bj, +32): entry (a, b)
      for (int yy = ty; yy < 32; yy += 8) {
        int a = 32 * bi + tx, b = 32 * bj + yy;
        double v = 0.0;
        if (a < m && b < m) {
          v = kern_entry(kind, kc, xs[a], xs[b]);
          if (a == b) v = __dadd_rn(v, nug);
        }
        if (a < Bm && b < Bm) D[(size_t)b * Bm + a] = v;
        tile[yy][tx] = v;
      }
      __syncthreads();
      // mirror: entry (b, a) for b in tile cols, a in tile rows -> column a, row b
      for (int yy = ty; yy < 32; yy += 8) {
        int b = 32 * bj + tx, a = 32 * bi + yy;
        if (a < Bm && b < Bm) D[(size_t)a * Bm + b] = tile[tx][yy];
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// ACA.  work[cta] = {level, node, g, G}: the G CTAs of one group split the
// block's rows and columns; every CTA of the group takes identical pivot
// decisions from the same reduced data, so only partial maxima are exchanged.
// The arithmetic (fused multiply-adds acc - U V with l ascending, the row
// scaled by one IEEE reciprocal of the pivot) matches the CPU reference
// operation for operation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 4) k_aca(const HmatDesc* __restrict__ Hd, const int4* __restrict__ work,
                                              ArgMax* __restrict__ part, unsigned int* __restrict__ bar,
                                              int* __restrict__ abort_flag, size_t pstride) {
  // problem of a batched launch: its descriptor, its partials, barriers and
  // abort flag pstride bytes after the previous problem's
  Hd += blockIdx.y;
  part = (ArgMax*)((char*)part + blockIdx.y * pstride);
  bar = (unsigned int*)((char*)bar + blockIdx.y * pstride);
  abort_flag = (int*)((char*)abort_flag + blockIdx.y * pstride);
  const int4 w = work[blockIdx.x];
  const int lvl = w.x, bi = w.y, g = w.z, G = w.w;
  const int base = blockIdx.x - g;
  const int64_t n = Hd->n;
  const int cap = Hd->cap, kind = Hd->kind;
  const double kc = Hd->kc, eps = Hd->eps;
  const double* __restrict__ x = Hd->x;
  double* Bs = Hd->bases + (size_t)lvl * cap * n;
  int s, h, e;
  node_range(Hd->bnd, lvl, bi, s, h, e);
  const int m = h - s, p = e - h;
  const int nid = node_id(lvl, bi);
  const int rc = (m + G - 1) / G, cc = (p + G - 1) / G;
  const int r0 = min(m, g * rc), r1 = min(m, g * rc + rc);
  const int c0 = min(p, g * cc), c1 = min(p, g * cc + cc);

  __shared__ int rowp[FIFA_CAP_MAX], colp[FIFA_CAP_MAX];
  __shared__ ArgMax shA[33];
  __shared__ double shD[33];

  int i = m - 1, k = 0;
  bool hit = false;
  unsigned int phase = 0;
  if (m <= 0 || p <= 0) k = 0;
  else
    while (true) {
      if (k == cap) { hit = true; break; }
      // residual of row i over this CTA's columns, stored unnormalised in V[:, k]
      const double xi = x[s + i];
      ArgMax best{-1.0, 0x7fffffff, 0.0};
      for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
        double acc = kern_entry(kind, kc, xi, x[h + j]);
        for (int l = 0; l < k; ++l)
          acc = __fma_rn(-__ldcg(Bs + (size_t)l * n + s + i), Bs[(size_t)l * n + h + j], acc);
        Bs[(size_t)k * n + h + j] = acc;
        // an entry that would win is checked against the used columns (the
        // check runs only then: same result as checking every entry)
        const ArgMax cand{fabs(acc), j, acc};
        if (am_wins(best, cand)) {
          bool used = false;
          for (int l = 0; l < k; ++l) used |= (colp[l] == j);
          if (!used) best = cand;
        }
      }
      best = block_argmax(best, shA);
      if (G > 1) {
        if (threadIdx.x == 0) part[3 * (base + g)] = best;
        ++phase;
        if (!group_barrier(bar + base, G * phase, Hd->status, abort_flag, Hd->spin)) return;
        ArgMax t{-1.0, 0x7fffffff, 0.0};
        for (int q = threadIdx.x; q < G; q += blockDim.x) {
          const ArgMax* pq = part + 3 * (base + q);
          t = am_better(t, ArgMax{__ldcg(&pq->v), __ldcg(&pq->i), __ldcg(&pq->sv)});
        }
        best = block_argmax(t, shA);
      }
      if (!(best.v > 0.0)) break;
      const int js = best.i;
      const double piv = best.sv;
      const double rpiv = __ddiv_rn(1.0, piv);
      for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
        double* vp = Bs + (size_t)k * n + h + j;
        *vp = __dmul_rn(*vp, rpiv);
      }
      // residual of column js over this CTA's rows, stored in U[:, k]
      const double xj = x[h + js];
      double umax = 0.0;
      ArgMax nb{-1.0, 0x7fffffff, 0.0};
      for (int ii = r0 + threadIdx.x; ii < r1; ii += blockDim.x) {
        double acc = kern_entry(kind, kc, x[s + ii], xj);
        for (int l = 0; l < k; ++l)
          acc = __fma_rn(-Bs[(size_t)l * n + s + ii], __ldcg(Bs + (size_t)l * n + h + js), acc);
        Bs[(size_t)k * n + s + ii] = acc;
        umax = nn_max(umax, fabs(acc));
        const ArgMax cand{fabs(acc), ii, acc};
        if (am_wins(nb, cand)) {
          bool used = (ii == i);
          for (int l = 0; l < k; ++l) used |= (rowp[l] == ii);
          if (!used) nb = cand;
        }
      }
      umax = block_max(umax, shD);
      nb = block_argmax(nb, shA);
      if (G > 1) {
        if (threadIdx.x == 0) {
          part[3 * (base + g) + 1] = ArgMax{umax, 0, 0.0};
          part[3 * (base + g) + 2] = nb;
        }
        ++phase;
        if (!group_barrier(bar + base, G * phase, Hd->status, abort_flag, Hd->spin)) return;
        double tm = 0.0;
        ArgMax t{-1.0, 0x7fffffff, 0.0};
        for (int q = threadIdx.x; q < G; q += blockDim.x) {
          const ArgMax* pq = part + 3 * (base + q);
          tm = nn_max(tm, __ldcg(&pq[1].v));
          t = am_better(t, ArgMax{__ldcg(&pq[2].v), __ldcg(&pq[2].i), __ldcg(&pq[2].sv)});
        }
        umax = block_max(tm, shD);
        nb = block_argmax(t, shA);
        // Slots: 3*cta + {0: row phase, 1-2: column phase}.  A slot is rewritten
        // one phase later, after a barrier every reader has already passed.
      }
      if (umax <= eps) break;
      if (threadIdx.x == 0) {
        rowp[k] = i;
        colp[k] = js;
      }
      __syncthreads();
      ++k;
      if (nb.v < 0.0) break;
      i = nb.i;
    }
  if (g == 0 && threadIdx.x == 0) {
    Hd->rank[nid] = k;
    for (int l = 0; l < cap; ++l) {
      Hd->row_piv[nid * cap + l] = l < k ? rowp[l] : -1;
      Hd->col_piv[nid * cap + l] = l < k ? colp[l] : -1;
    }
    if (hit) atomicOr(Hd->status, FIFA_DEV_RANK_CAP);
  }
}

// ---------------------------------------------------------------------------
// ACA of small blocks (both sides <= ACA_WARP_MAX rows): one warp per block,
// eight independent blocks per CTA.  Same arithmetic and pivot rules as k_aca
// with G = 1 (so the same bases, bit for bit); the reductions are warp
// shuffles, with no CTA barrier and no idle warps in them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ ArgMax warp_argmax_all(ArgMax a) {
  for (int o = 16; o > 0; o >>= 1) {
    ArgMax b;
    b.v = __shfl_xor_sync(0xffffffffu, a.v, o);
    b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
    b.sv = __shfl_xor_sync(0xffffffffu, a.sv, o);
    a = am_better(a, b);
  }
  return a;
}

__global__ void __launch_bounds__(256, 3) k_aca_warp(const HmatDesc* __restrict__ Hd, const int4* __restrict__ work,
                                                  int nwork) {
  Hd += blockIdx.y;  // problem of a batched launch (descriptor arrays)
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * 8 + wl;
  if (item >= nwork) return;  // whole warp
  const int4 w = work[item];
  const int lvl = w.x, bi = w.y;
  const int64_t n = Hd->n;
  const int cap = Hd->cap, kind = Hd->kind;
  const double kc = Hd->kc, eps = Hd->eps;
  const double* __restrict__ x = Hd->x;
  double* Bs = Hd->bases + (size_t)lvl * cap * n;
  int s, h, e;
  node_range(Hd->bnd, lvl, bi, s, h, e);
  const int m = h - s, p = e - h;
  const int nid = node_id(lvl, bi);
  __shared__ int rowp_all[8][FIFA_CAP_MAX], colp_all[8][FIFA_CAP_MAX];
  int* rowp = rowp_all[wl];
  int* colp = colp_all[wl];

  int i = m - 1, k = 0;
  bool hit = false;
  if (m > 0 && p > 0)
    while (true) {
      if (k == cap) { hit = true; break; }
      // residual of row i, stored unnormalised in V[:, k]
      const double xi = x[s + i];
      ArgMax best{-1.0, 0x7fffffff, 0.0};
      for (int j = lane; j < p; j += 32) {
        double acc = kern_entry(kind, kc, xi, x[h + j]);
        for (int l = 0; l < k; ++l)
          acc = __fma_rn(-__ldcg(Bs + (size_t)l * n + s + i), __ldcg(Bs + (size_t)l * n + h + j), acc);
        Bs[(size_t)k * n + h + j] = acc;
        // an entry that would win is checked against the used columns (the
        // check runs only then: same result as checking every entry)
        const ArgMax cand{fabs(acc), j, acc};
        if (am_wins(best, cand)) {
          bool used = false;
          for (int l = 0; l < k; ++l) used |= (colp[l] == j);
          if (!used) best = cand;
        }
      }
      best = warp_argmax_all(best);
      if (!(best.v > 0.0)) break;
      const int js = best.i;
      const double piv = best.sv;
      const double rpiv = __ddiv_rn(1.0, piv);
      for (int j = lane; j < p; j += 32) {
        double* vp = Bs + (size_t)k * n + h + j;
        *vp = __dmul_rn(*vp, rpiv);
      }
      __syncwarp();
      // residual of column js, stored in U[:, k]
      const double xj = x[h + js];
      double umax = 0.0;
      ArgMax nb{-1.0, 0x7fffffff, 0.0};
      for (int ii = lane; ii < m; ii += 32) {
        double acc = kern_entry(kind, kc, x[s + ii], xj);
        for (int l = 0; l < k; ++l)
          acc = __fma_rn(-__ldcg(Bs + (size_t)l * n + s + ii), __ldcg(Bs + (size_t)l * n + h + js), acc);
        Bs[(size_t)k * n + s + ii] = acc;
        umax = nn_max(umax, fabs(acc));
        const ArgMax cand{fabs(acc), ii, acc};
        if (am_wins(nb, cand)) {
          bool used = (ii == i);
          for (int l = 0; l < k; ++l) used |= (rowp[l] == ii);
          if (!used) nb = cand;
        }
      }
      for (int o = 16; o > 0; o >>= 1) umax = nn_max(umax, __shfl_xor_sync(0xffffffffu, umax, o));
      nb = warp_argmax_all(nb);
      if (umax <= eps) break;
      if (lane == 0) {
        rowp[k] = i;
        colp[k] = js;
      }
      __syncwarp();
      ++k;
      if (nb.v < 0.0) break;
      i = nb.i;
    }
  if (lane == 0) {
    Hd->rank[nid] = k;
    for (int l = 0; l < cap; ++l) {
      Hd->row_piv[nid * cap + l] = l < k ? rowp[l] : -1;
      Hd->col_piv[nid * cap + l] = l < k ? colp[l] : -1;
    }
    if (hit) atomicOr(Hd->status, FIFA_DEV_RANK_CAP);
  }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
cudaError_t launch_aca_warp(const HmatDesc* Hd, const int4* work, int nwork, cudaStream_t st, int nprob) {
  if (nwork <= 0) return cudaSuccess;
  k_aca_warp<<<dim3((nwork + 7) / 8, nprob), 256, 0, st>>>(Hd, work, nwork);
  return cudaGetLastError();
}

cudaError_t launch_leaf_assemble(const HmatDesc* Hd, int nleaf, cudaStream_t st, int nprob) {
  k_leaf_assemble<<<dim3(nleaf, nprob), 256, 0, st>>>(Hd);
  return cudaGetLastError();
}

cudaError_t launch_aca(const HmatDesc* Hd, const int4* work, int ncta, bool cooperative, ArgMax* part,
                       unsigned int* bar, int* abort_flag, cudaStream_t st, int nprob, size_t pstride) {
  if (ncta <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ncta, nprob);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = cooperative ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_aca, Hd, work, part, bar, abort_flag, pstride);
}

int aca_max_coresident_ctas() {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_aca, 256, 0) != cudaSuccess) per_sm = 1;
  return sms * per_sm;
}
