// C ABI of the FIFA-GP GB300 library (declared in include/fifa.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "../../include/fifa.h"
#include "fifa_api_internal.h"
#include "fifa_chain.h"
#include "fifa_common.cuh"
#include "fifa_launch.h"
#include "fifa_mixed.h"

// ---------------------------------------------------------------------------
// Arena: first-fit sub-allocator over one device buffer (256-byte granules).
// ---------------------------------------------------------------------------
void* Arena::alloc(size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  for (auto it = free_.begin(); it != free_.end(); ++it) {
    if (it->second >= bytes) {
      size_t off = it->first, sz = it->second;
      free_.erase(it);
      if (sz > bytes) free_[off + bytes] = sz - bytes;
      used_[off] = bytes;
      in_use += bytes;
      peak = std::max(peak, in_use);
      return base + off;
    }
  }
  return nullptr;
}

void Arena::release(void* p) {
  if (!p) return;
  size_t off = (char*)p - base;
  auto it = used_.find(off);
  if (it == used_.end()) return;
  size_t sz = it->second;
  used_.erase(it);
  in_use -= sz;
  auto nx = free_.lower_bound(off);
  if (nx != free_.end() && nx->first == off + sz) {
    sz += nx->second;
    nx = free_.erase(nx);
  }
  if (nx != free_.begin()) {
    auto pv = std::prev(nx);
    if (pv->first + pv->second == off) {
      pv->second += sz;
      return;
    }
  }
  free_[off] = sz;
}

#define CK(call)                          \
  do {                                    \
    cudaError_t e_ = (call);              \
    if (e_ != cudaSuccess) {              \
      ctx->last_cuda = e_;                \
      return FIFA_ERR_CUDA;               \
    }                                     \
  } while (0)

static inline int64_t n_of(const Plan* P) { return P->n; }

static fifa_status dev_status_to_api(int s) {
  if (s & FIFA_DEV_TIMEOUT) return FIFA_ERR_TIMEOUT;
  if (s & FIFA_DEV_NOT_SPD) return FIFA_ERR_NOT_SPD;
  if (s & FIFA_DEV_RANK_CAP) return FIFA_ERR_RANK_CAP;
  return FIFA_OK;
}

// ---------------------------------------------------------------------------
// Plans: tree bounds and launch shapes for one (n, B).
// ---------------------------------------------------------------------------
static int levels_for(int64_t n, int B) {
  int L = 0;
  while ((n + ((int64_t)1 << L) - 1) / ((int64_t)1 << L) > B) ++L;
  return L;
}

// Partials of the fused sweep: two buffers of one projection per CTA, for up to
// min(nleaf, FS_CTAS_MAX) CTAs (none with independent CTAs: no grid barriers).
static size_t fused_sweep_part_doubles(const Plan* P, const fifa_opts& o) {
  if (o.independent_ctas) return 1;
  return (size_t)2 * std::min(P->nleaf, FS_CTAS_MAX) * FS_PART_STRIDE;
}

// Partials of the fused H-matvec: one projection per CTA and level below the
// CTA level, for up to min(nleaf, FS_CTAS_MAX) CTAs and 10 such levels.
static size_t fused_mv_part_doubles(const Plan* P, const fifa_opts& o) {
  if (o.independent_ctas) return 1;
  return (size_t)std::min(P->nleaf, FS_CTAS_MAX) * std::max(1, std::min(P->L, 10)) * FIFA_CAP_MAX * SWEEP_RHS_MAX;
}

// Host part of a plan: bounds, ACA / level / sweep groups, scratch size.
// aca_cores / lvl_cores[b]: co-resident CTA budgets of the ACA kernel and of
// the level kernel of rank bucket b.
static Plan* plan_build(int64_t n, const fifa_opts& o, int aca_cores, const int* lvl_cores, fifa_status* st) {
  Plan* P = new (std::nothrow) Plan();
  if (!P) {
    *st = FIFA_ERR_OOM;
    return nullptr;
  }
  P->n = n;
  P->B = o.leaf_size;
  P->L = levels_for(n, P->B);
  if (P->L >= FIFA_LEVELS_MAX) {
    delete P;
    *st = FIFA_ERR_UNSUPPORTED;
    return nullptr;
  }
  P->nleaf = 1 << P->L;
  P->nnodes = P->nleaf - 1;
  // bounds: level l at offset 2^l - 1 + l
  std::vector<int> b;
  b.push_back(0);
  b.push_back((int)n);
  P->bnd_host = b;
  std::vector<int> prev = b;
  for (int l = 0; l < P->L; ++l) {
    std::vector<int> nxt;
    nxt.push_back(0);
    for (size_t i = 0; i + 1 < prev.size(); ++i) {
      int s = prev[i], e = prev[i + 1];
      nxt.push_back(s + (e - s) / 2);
      nxt.push_back(e);
    }
    P->bnd_host.insert(P->bnd_host.end(), nxt.begin(), nxt.end());
    prev = nxt;
  }
  P->Bm = 0;
  for (size_t i = 0; i + 1 < prev.size(); ++i) P->Bm = std::max(P->Bm, prev[i + 1] - prev[i]);
  const int cap = o.rank_cap;
  const bool groups = !o.independent_ctas;
  // ACA groups.  A level-l block has ~n/2^l rows + columns and every level has
  // about the same total work, so the co-resident CTA budget is split evenly
  // over the top levels: level l gets G_l = budget / (levels * 2^l) CTAs per
  // block, at most one per 1024 block rows (>= 2 to be worth a group; blocks
  // from 4096 rows).  Levels below run one CTA per block in a second launch.
  // (Mid-size problems are latency-bound at their top levels: groups of one
  // CTA per 4096 rows left the level-0 block of n = 2^14 on four SMs.)
  std::vector<int> Gl(P->L, 1);
  int ncoop_levels = 0;
  for (int l = 0; groups && l < P->L; ++l) {
    const int64_t entries = n >> l;
    if (entries < 4096) break;
    ncoop_levels = l + 1;
  }
  while (ncoop_levels > 0) {
    const int per_level = aca_cores / ncoop_levels;
    if ((per_level >> (ncoop_levels - 1)) >= 2) break;
    --ncoop_levels;  // the deepest candidate level cannot get two CTAs per block
  }
  if (ncoop_levels > 0) {
    const int per_level = aca_cores / ncoop_levels;
    for (int l = 0; l < ncoop_levels; ++l) {
      const int64_t want = std::max<int64_t>(2, (n >> l) / 1024);
      Gl[l] = (int)std::min<int64_t>(want, per_level >> l);
      if (Gl[l] < 2) Gl[l] = 1;
    }
  }
  // blocks whose node spans <= 2 ACA_WARP_MAX rows take one warp each
  std::vector<int4> coop, solo, warp;
  for (int l = 0; l < P->L; ++l) {
    const int off = (1 << l) - 1 + l;
    for (int i = 0; i < (1 << l); ++i) {
      const int len = P->bnd_host[off + i + 1] - P->bnd_host[off + i];
      if (Gl[l] > 1)
        for (int g = 0; g < Gl[l]; ++g) coop.push_back(make_int4(l, i, g, Gl[l]));
      else if (len <= 2 * ACA_WARP_MAX)
        warp.push_back(make_int4(l, i, 0, 1));
      else
        solo.push_back(make_int4(l, i, 0, 1));
    }
  }
  P->aca_ncoop = (int)coop.size();
  P->aca_nsolo = (int)solo.size();
  P->aca_nwarp = (int)warp.size();
  P->work_host = coop;
  P->work_host.insert(P->work_host.end(), solo.begin(), solo.end());
  P->work_host.insert(P->work_host.end(), warp.begin(), warp.end());
  // factor / sweep groups per level: levels with fewer nodes than the
  // co-resident CTAs split each node's rows over a group of CTAs that fills
  // the GPU, each CTA with >= 512 rows (>= 256 up to n = 2^15, where the top
  // levels' latency, not their work, sets the time); each rank bucket's kernel
  // has its own CTAs per SM and so its own group size
  for (int b = 0; b < LEVEL_BUCKETS; ++b) P->lvl_G[b].assign(P->L, 1);
  P->sweep_G.assign(P->L, 1);
  const int64_t per = n <= 32768 ? 256 : 512;
  for (int l = 0; l < P->L; ++l) {
    const int64_t len = (n + ((int64_t)1 << l) - 1) >> l;
    const int64_t nodes = (int64_t)1 << l;
    for (int b = 0; b < LEVEL_BUCKETS; ++b)
      if (groups && 2 * nodes <= lvl_cores[b] && len >= 2 * per) {
        const int64_t G = std::min<int64_t>(len / per, lvl_cores[b] / nodes);
        P->lvl_G[b][l] = (int)std::max<int64_t>(1, G);
      }
    P->sweep_G[l] = (int)std::max<int64_t>(1, (len + 2047) / 2048);
  }
  // device arrays: bounds, then the ACA work list at a 16-byte offset
  P->work_off = (P->bnd_host.size() * sizeof(int) + 15) & ~(size_t)15;
  P->dev_bytes = P->work_off + P->work_host.size() * sizeof(int4);
  // scratch requirement (bytes)
  size_t need = 0;
  auto add = [&](size_t b) { need += (b + 255) & ~(size_t)255; };
  add((size_t)3 * sizeof(ArgMax) * std::max(1, P->aca_ncoop));  // ACA partials
  add(sizeof(unsigned int) * std::max(1, P->aca_ncoop));         // ACA barriers
  int64_t lvl_ctas = 1, sweep_ctas = 1;
  for (int l = 0; l < P->L; ++l) {
    for (int b = 0; b < LEVEL_BUCKETS; ++b) lvl_ctas = std::max<int64_t>(lvl_ctas, ((int64_t)1 << l) * P->lvl_G[b][l]);
    sweep_ctas = std::max<int64_t>(sweep_ctas, ((int64_t)1 << l) * P->sweep_G[l]);
  }
  P->lvl_ctas_max = (int)lvl_ctas;
  add(sizeof(double) * 2 * lvl_ctas * level_part_stride(cap));           // level partials (2 slots)
  add(sizeof(unsigned int) * LEVEL_BUCKETS * lvl_ctas);                  // level barriers, one set per rank bucket
  add(sizeof(double) * sweep_ctas * 2 * cap * SWEEP_RHS_MAX);            // sweep partials
  add(sizeof(double) * (size_t)P->nleaf * std::max(1, P->L) * cap * SWEEP_RHS_MAX);  // matvec partials
  add(sizeof(double) * (size_t)std::max(1, P->nnodes) * 2 * cap * SWEEP_RHS_MAX);     // matvec projections
  add(sizeof(double) * (size_t)n * 16);                                   // work vectors
  add(sizeof(double) * 512);                                              // reduction partials
  add(256);                                                               // flags
  add(sizeof(double) * fused_sweep_part_doubles(P, o));                   // fused sweep partials
  add(256);                                                               // fused sweep barrier
  add(sizeof(double) * fused_mv_part_doubles(P, o));                      // fused matvec partials
  add(256);                                                               // fused matvec barrier
  add(sizeof(double) * PCG_SCRATCH_DOUBLES);                              // mixed-precision solve state
  P->scratch_bytes = need;
  return P;
}

extern "C" fifa_status fifa_plan_describe(const fifa_opts* opts, int64_t n, int aca_cores, const int* lvl_cores,
                                          fifa_plan_info* info, int* bounds_out, int* aca_work_out,
                                          int* lvl_groups_out) {
  if (!opts || !lvl_cores || !info || n < 1 || opts->leaf_size < 1 || opts->rank_cap < 1 ||
      opts->rank_cap > FIFA_CAP_MAX || aca_cores < 1)
    return FIFA_ERR_INVALID_ARG;
  for (int b = 0; b < LEVEL_BUCKETS; ++b)
    if (lvl_cores[b] < 1) return FIFA_ERR_INVALID_ARG;
  fifa_status st = FIFA_OK;
  Plan* P = plan_build(n, *opts, aca_cores, lvl_cores, &st);
  if (!P) return st;
  info->levels = P->L;
  info->nleaf = P->nleaf;
  info->leaf_max = P->Bm;
  info->aca_grouped_ctas = P->aca_ncoop;
  info->aca_solo_blocks = P->aca_nsolo;
  info->aca_warp_blocks = P->aca_nwarp;
  info->scratch_bytes = (int64_t)P->scratch_bytes;
  if (bounds_out) std::copy(P->bnd_host.begin(), P->bnd_host.end(), bounds_out);
  if (aca_work_out)
    for (size_t k = 0; k < P->work_host.size(); ++k) {
      const int4 w = P->work_host[k];
      aca_work_out[4 * k] = w.x;
      aca_work_out[4 * k + 1] = w.y;
      aca_work_out[4 * k + 2] = w.z;
      aca_work_out[4 * k + 3] = w.w;
    }
  if (lvl_groups_out)
    for (int b = 0; b < LEVEL_BUCKETS; ++b)
      for (int l = 0; l < P->L; ++l) lvl_groups_out[b * P->L + l] = P->lvl_G[b][l];
  delete P;
  return FIFA_OK;
}

Plan* get_plan(fifa_ctx* ctx, int64_t n, fifa_status* st) {
  auto key = std::make_pair(n, ctx->opts.leaf_size);
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) return it->second;
  Plan* P = plan_build(n, ctx->opts, ctx->aca_coresident, ctx->level_coresident, st);
  if (!P) return nullptr;
  // fused sweep: the largest power-of-two grid (<= nleaf, FS_CTAS_MAX) whose
  // CTAs, each holding the longest level-k node in shared memory, are all
  // co-resident (for both factor precisions)
  if (!ctx->opts.independent_ctas) {
    for (int k = std::min(P->L, 10); k >= 0; --k) {
      if ((1 << k) > FS_CTAS_MAX) continue;
      int rows = 0;
      for (int i = 0; i < (1 << k); ++i)
        rows = std::max(rows, P->bnd_host[bnd_off(k) + i + 1] - P->bnd_host[bnd_off(k) + i]);
      const int cap = ctx->opts.rank_cap;
      const int co = std::min(sweep_fused_coresident(0, rows, cap), sweep_fused_coresident(1, rows, cap)) /
                     coresident_share(ctx->opts);
      if (co >= (1 << k)) {
        P->fs_ls = k;
        P->fs_rows = rows;
        break;
      }
    }
    // fused H-matvec: the same kind of grid, rows per CTA <= MV_FUSED_ROWS_MAX
    for (int k = std::min(P->L, 10); k >= 0; --k) {
      int rows = 0;
      for (int i = 0; i < (1 << k); ++i)
        rows = std::max(rows, P->bnd_host[bnd_off(k) + i + 1] - P->bnd_host[bnd_off(k) + i]);
      if (rows > MV_FUSED_ROWS_MAX) break;
      if (mv_fused_coresident(rows) / coresident_share(ctx->opts) >= (1 << k)) {
        P->mv_ls = k;
        P->mv_rows = rows;
        break;
      }
    }
  }
  char* mem = (char*)ctx->arena.alloc(P->dev_bytes);
  if (!mem) {
    delete P;
    *st = FIFA_ERR_OOM;
    return nullptr;
  }
  P->bnd_dev = (int*)mem;
  P->aca_work = (int4*)(mem + P->work_off);
  cudaError_t e = cudaMemcpyAsync(P->bnd_dev, P->bnd_host.data(), P->bnd_host.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess && !P->work_host.empty())
    e = cudaMemcpyAsync(P->aca_work, P->work_host.data(), P->work_host.size() * sizeof(int4), cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // the host vectors stay, but keep the copy simple
  if (e != cudaSuccess) {
    ctx->last_cuda = e;
    ctx->arena.release(mem);
    delete P;
    *st = FIFA_ERR_CUDA;
    return nullptr;
  }
  ctx->plans[key] = P;
  return P;
}

// Device bytes of one arena allocation of b bytes.
static inline size_t arena_round(size_t b) { return b == 0 ? 256 : (b + 255) & ~(size_t)255; }

size_t hmat_bytes(const Plan* P, int cap) {
  const size_t nn = std::max(1, P->nnodes);
  return arena_round(sizeof(double) * (size_t)P->nleaf * P->Bm * P->Bm) +
         arena_round(sizeof(double) * (size_t)std::max(1, P->L) * cap * P->n) + arena_round(sizeof(int) * nn) +
         2 * arena_round(sizeof(int) * nn * cap) + arena_round(sizeof(int)) + arena_round(sizeof(HmatDesc));
}

size_t fact_bytes(const Plan* P, int cap, int with32) {
  const size_t nn = std::max(1, P->nnodes);
  size_t b = arena_round(sizeof(double) * (size_t)P->nleaf * P->Bm * P->Bm) +
             arena_round(sizeof(double) * (size_t)P->nleaf * P->Bm) +
             arena_round(sizeof(double) * (size_t)std::max(1, P->L) * cap * P->n) +
             2 * arena_round(sizeof(double) * nn * 4 * cap * cap) + arena_round(sizeof(int) * nn) +
             arena_round(sizeof(double) * (P->nleaf + nn)) + arena_round(sizeof(double)) + arena_round(sizeof(int)) +
             arena_round(sizeof(FactDesc));
  if (with32)  // the FP32 copy: leaf factors, reciprocal pivots, bases, descriptor
    b += arena_round(sizeof(float) * (size_t)P->nleaf * P->Bm * P->Bm) +
         arena_round(sizeof(float) * (size_t)P->nleaf * P->Bm) +
         arena_round(sizeof(float) * (size_t)std::max(1, P->L) * cap * P->n) + arena_round(sizeof(FactDesc));
  return b;
}

extern "C" fifa_status fifa_chain_bytes(const fifa_opts* opts, int64_t n, size_t* bytes_out) {
  if (!opts || !bytes_out || n < 2) return FIFA_ERR_INVALID_ARG;
  if (opts->leaf_size < 1 || opts->rank_cap < 1) return FIFA_ERR_INVALID_ARG;
  if (opts->leaf_size > FIFA_LEAF_MAX || opts->rank_cap > FIFA_CAP_MAX) return FIFA_ERR_UNSUPPORTED;
  fifa_status st = FIFA_OK;
  int lvl_cores[LEVEL_BUCKETS];
  for (int b = 0; b < LEVEL_BUCKETS; ++b)
    lvl_cores[b] = std::min(level_bucket_coresident(0, b, opts->rank_cap), level_bucket_coresident(1, b, opts->rank_cap)) /
                   coresident_share(*opts);
  Plan* P = plan_build(n, *opts, aca_max_coresident_ctas() / coresident_share(*opts), lvl_cores, &st);
  if (!P) return st;
  *bytes_out = arena_round(256) /* context flags */ + arena_round(P->dev_bytes) + chain_bytes(P, *opts);
  delete P;
  return FIFA_OK;
}

// Carve the context scratch for a plan (after ensure_scratch).
Scratch carve(fifa_ctx* ctx, Plan* P) {
  Scratch S;
  char* p = (char*)(ctx->active_scratch ? ctx->active_scratch : ctx->scratch);
  auto take = [&](size_t b) {
    char* r = p;
    p += (b + 255) & ~(size_t)255;
    return (void*)r;
  };
  const int cap = ctx->opts.rank_cap;
  S.aca_part = (ArgMax*)take((size_t)3 * sizeof(ArgMax) * std::max(1, P->aca_ncoop));
  S.aca_bar = (unsigned int*)take(sizeof(unsigned int) * std::max(1, P->aca_ncoop));
  S.lvl_part = (double*)take(sizeof(double) * 2 * (size_t)P->lvl_ctas_max * level_part_stride(cap));
  S.lvl_bar = (unsigned int*)take(sizeof(unsigned int) * LEVEL_BUCKETS * P->lvl_ctas_max);
  int64_t sweep_ctas = 1;
  for (int l = 0; l < P->L; ++l) sweep_ctas = std::max<int64_t>(sweep_ctas, ((int64_t)1 << l) * P->sweep_G[l]);
  S.sweep_part = (double*)take(sizeof(double) * sweep_ctas * 2 * cap * SWEEP_RHS_MAX);
  S.mv_part = (double*)take(sizeof(double) * (size_t)P->nleaf * std::max(1, P->L) * cap * SWEEP_RHS_MAX);
  S.mv_proj = (double*)take(sizeof(double) * (size_t)std::max(1, P->nnodes) * 2 * cap * SWEEP_RHS_MAX);
  S.vec = (double*)take(sizeof(double) * (size_t)P->n * 16);
  S.red = (double*)take(sizeof(double) * 512);
  S.flags = (int*)take(256);
  S.fs_part = (double*)take(sizeof(double) * fused_sweep_part_doubles(P, ctx->opts));
  S.fs_bar = (unsigned int*)take(256);
  S.mv_fpart = (double*)take(sizeof(double) * fused_mv_part_doubles(P, ctx->opts));
  S.mv_bar = (unsigned int*)take(256);
  S.pcg = (double*)take(sizeof(double) * PCG_SCRATCH_DOUBLES);
  return S;
}

fifa_status ensure_scratch(fifa_ctx* ctx, Plan* P) {
  if (ctx->active_scratch) return FIFA_OK;  // a chain enqueues into its own scratch
  if (ctx->scratch_bytes >= P->scratch_bytes) return FIFA_OK;
  if (ctx->capturing) return FIFA_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->arena.release(ctx->scratch);
  ctx->scratch = ctx->arena.alloc(P->scratch_bytes);
  if (!ctx->scratch) {
    ctx->scratch_bytes = 0;
    return FIFA_ERR_OOM;
  }
  ctx->scratch_bytes = P->scratch_bytes;
  return FIFA_OK;
}

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
extern "C" fifa_status fifa_create(fifa_ctx** out, const fifa_opts* opts, void* cuda_stream, void* arena_dev,
                                   size_t arena_bytes) {
  if (!out || !opts) return FIFA_ERR_INVALID_ARG;
  *out = nullptr;
  if (opts->leaf_size < 1 || opts->rank_cap < 1 || !(opts->aca_tol >= 0.0)) return FIFA_ERR_INVALID_ARG;
  if (opts->leaf_size > FIFA_LEAF_MAX || opts->rank_cap > FIFA_CAP_MAX) return FIFA_ERR_UNSUPPORTED;
  if (opts->prec != FIFA_FP64 && opts->prec != FIFA_MIXED) return FIFA_ERR_INVALID_ARG;
  if (opts->independent_ctas != 0 && opts->independent_ctas != 1) return FIFA_ERR_INVALID_ARG;
  if (opts->wait_polls < 0) return FIFA_ERR_INVALID_ARG;
  if (opts->coresident_share < 0 || opts->coresident_share > 64) return FIFA_ERR_INVALID_ARG;
  if (opts->overlap_proposal != 0 && opts->overlap_proposal != 1) return FIFA_ERR_INVALID_ARG;
  if (arena_bytes < (1u << 20)) return FIFA_ERR_INVALID_ARG;
  fifa_ctx* ctx = new (std::nothrow) fifa_ctx();
  if (!ctx) return FIFA_ERR_OOM;
  ctx->opts = *opts;
  if (ctx->opts.refine_max < 0) ctx->opts.refine_max = 0;
  ctx->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&ctx->device);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (arena_dev) {
    ctx->arena.base = (char*)arena_dev;
    ctx->own_arena = false;
  } else {
    void* p = nullptr;
    if (cudaMalloc(&p, arena_bytes) != cudaSuccess) {
      delete ctx;
      return FIFA_ERR_OOM;
    }
    ctx->arena.base = (char*)p;
    ctx->own_arena = true;
  }
  ctx->arena.size = arena_bytes & ~(size_t)255;
  ctx->arena.free_[0] = ctx->arena.size;
  // the context's share of the CTAs the GPU holds at once (coresident_share)
  ctx->aca_coresident = aca_max_coresident_ctas() / coresident_share(ctx->opts);
  for (int b = 0; b < LEVEL_BUCKETS; ++b)
    ctx->level_coresident[b] = std::min(level_bucket_coresident(0, b, ctx->opts.rank_cap),
                                        level_bucket_coresident(1, b, ctx->opts.rank_cap)) /
                               coresident_share(ctx->opts);
  ctx->flags = (int*)ctx->arena.alloc(256);
  ctx->host_flags = nullptr;
  cudaMallocHost((void**)&ctx->host_flags, 256);
  if (!ctx->flags || !ctx->host_flags) {
    fifa_destroy_ctx(ctx);
    return FIFA_ERR_OOM;
  }
  if (ctx->aca_coresident <= 0 || *std::min_element(ctx->level_coresident, ctx->level_coresident + LEVEL_BUCKETS) <= 0) {
    fifa_destroy_ctx(ctx);
    return FIFA_ERR_UNSUPPORTED;
  }
  // leave no error behind for the caller's next runtime call to pick up
  cudaError_t pending = cudaGetLastError();
  if (pending != cudaSuccess) {
    ctx->last_cuda = pending;
    fifa_destroy_ctx(ctx);
    return FIFA_ERR_CUDA;
  }
  *out = ctx;
  return FIFA_OK;
}

fifa_status ctx_rebind_arena(fifa_ctx* ctx, void* base, size_t bytes) {
  if (!ctx || !base || bytes < 1024) return FIFA_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->own_arena) return FIFA_ERR_INVALID_ARG;
  for (auto& kv : ctx->plans) delete kv.second;
  ctx->plans.clear();
  ctx->arena.base = (char*)base;
  ctx->arena.size = bytes & ~(size_t)255;
  ctx->arena.in_use = ctx->arena.peak = 0;
  ctx->arena.free_.clear();
  ctx->arena.used_.clear();
  ctx->arena.free_[0] = ctx->arena.size;
  ctx->scratch = nullptr;
  ctx->scratch_bytes = 0;
  ctx->active_scratch = nullptr;
  ctx->flags = (int*)ctx->arena.alloc(256);
  return ctx->flags ? FIFA_OK : FIFA_ERR_OOM;
}

extern "C" void fifa_destroy_ctx(fifa_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->plans) delete kv.second;
  if (ctx->own_arena && ctx->arena.base) cudaFree(ctx->arena.base);
  if (ctx->host_flags) cudaFreeHost(ctx->host_flags);
  delete ctx;
}

// ---------------------------------------------------------------------------
// H-matrix objects
// ---------------------------------------------------------------------------
static fifa_status upload_desc(fifa_ctx* ctx, fifa_hmat* H) {
  CK(cudaMemcpyAsync(H->dev, &H->host, sizeof(HmatDesc), cudaMemcpyHostToDevice, ctx->stream));
  return FIFA_OK;
}

fifa_status hmat_alloc(fifa_ctx* ctx, Plan* P, int kind, fifa_hmat** out) {
  fifa_hmat* H = new (std::nothrow) fifa_hmat();
  if (!H) return FIFA_ERR_OOM;
  H->plan = P;
  const int cap = ctx->opts.rank_cap;
  const size_t nn = std::max(1, P->nnodes);
  HmatDesc& d = H->host;
  memset(&d, 0, sizeof(d));
  d.n = P->n;
  d.L = P->L;
  d.nleaf = P->nleaf;
  d.Bm = P->Bm;
  d.cap = cap;
  d.kind = kind;
  d.bnd = P->bnd_dev;
  d.scale = 1.0;
  d.shift = 0.0;
  d.eps = ctx->opts.aca_tol;
  d.spin = ctx->opts.wait_polls > 0 ? (unsigned int)ctx->opts.wait_polls : 0u;
  d.leaves = (double*)ctx->arena.alloc(sizeof(double) * (size_t)P->nleaf * P->Bm * P->Bm);
  d.bases = (double*)ctx->arena.alloc(sizeof(double) * (size_t)std::max(1, P->L) * cap * P->n);
  d.rank = (int*)ctx->arena.alloc(sizeof(int) * nn);
  d.row_piv = (int*)ctx->arena.alloc(sizeof(int) * nn * cap);
  d.col_piv = (int*)ctx->arena.alloc(sizeof(int) * nn * cap);
  d.status = (int*)ctx->arena.alloc(sizeof(int));
  H->dev = (HmatDesc*)ctx->arena.alloc(sizeof(HmatDesc));
  if (!d.leaves || !d.bases || !d.rank || !d.row_piv || !d.col_piv || !d.status || !H->dev) {
    fifa_destroy_hmat(ctx, H);
    return FIFA_ERR_OOM;
  }
  H->owns = true;
  *out = H;
  return FIFA_OK;
}

// Enqueue assembly of H for inputs x (device) with kernel constant kc (host value).
fifa_status hmat_assemble_enqueue(fifa_ctx* ctx, fifa_hmat* H) {
  fifa_status st = hmat_assemble_grouped_enqueue(ctx, H);
  return st == FIFA_OK ? hmat_assemble_rest_enqueue(ctx, H) : st;
}

// First part of the assembly: descriptor reset and the grouped ACA launch (the
// only assembly kernel whose CTAs wait on each other).
fifa_status hmat_assemble_grouped_enqueue(fifa_ctx* ctx, fifa_hmat* H) {
  Plan* P = H->plan;
  fifa_status st = ensure_scratch(ctx, P);
  if (st != FIFA_OK) return st;
  Scratch S = carve(ctx, P);
  cudaStream_t s = ctx->stream;
  CK(launch_prep_hmat(H->dev, P->nnodes, s));
  if (P->aca_ncoop > 0) {
    CK(cudaMemsetAsync(S.aca_bar, 0, sizeof(unsigned int) * P->aca_ncoop, s));
    CK(cudaMemsetAsync(S.flags, 0, sizeof(int), s));
    CK(launch_aca(H->dev, P->aca_work, P->aca_ncoop, true, S.aca_part, S.aca_bar, S.flags, s));
  }
  return FIFA_OK;
}

// Second part (after the first in stream order): dense leaves, one-CTA and
// one-warp ACA blocks; independent CTAs only.
fifa_status hmat_assemble_rest_enqueue(fifa_ctx* ctx, fifa_hmat* H) {
  Plan* P = H->plan;
  fifa_status st = ensure_scratch(ctx, P);
  if (st != FIFA_OK) return st;
  Scratch S = carve(ctx, P);
  cudaStream_t s = ctx->stream;
  CK(launch_leaf_assemble(H->dev, P->nleaf, s));
  if (P->aca_nsolo > 0) CK(launch_aca(H->dev, P->aca_work + P->aca_ncoop, P->aca_nsolo, false, S.aca_part, S.aca_bar, S.flags, s));
  if (P->aca_nwarp > 0) CK(launch_aca_warp(H->dev, P->aca_work + P->aca_ncoop + P->aca_nsolo, P->aca_nwarp, s));
  return FIFA_OK;
}

fifa_status hmat_assemble_batched(fifa_ctx* ctx, Plan* P, HmatDesc* H0, int nprob, void* scratch0, size_t sstride) {
  void* saved = ctx->active_scratch;
  ctx->active_scratch = scratch0;
  Scratch S = carve(ctx, P);
  ctx->active_scratch = saved;
  cudaStream_t s = ctx->stream;
  CK(launch_prep_hmat(H0, P->nnodes, s, nprob));
  CK(launch_leaf_assemble(H0, P->nleaf, s, nprob));
  if (P->aca_ncoop > 0) {
    if ((int64_t)P->aca_ncoop * nprob <= ctx->aca_coresident) {  // every problem's groups co-resident at once
      CK(cudaMemset2DAsync(S.aca_bar, sstride, 0, sizeof(unsigned int) * P->aca_ncoop, nprob, s));
      CK(cudaMemset2DAsync(S.flags, sstride, 0, sizeof(int), nprob, s));
      CK(launch_aca(H0, P->aca_work, P->aca_ncoop, true, S.aca_part, S.aca_bar, S.flags, s, nprob, sstride));
    } else {
      for (int q = 0; q < nprob; ++q) {  // one grouped launch per problem, each filling the GPU
        const size_t off = (size_t)q * sstride;
        unsigned int* bar = (unsigned int*)((char*)S.aca_bar + off);
        int* flags = (int*)((char*)S.flags + off);
        CK(cudaMemsetAsync(bar, 0, sizeof(unsigned int) * P->aca_ncoop, s));
        CK(cudaMemsetAsync(flags, 0, sizeof(int), s));
        CK(launch_aca(H0 + q, P->aca_work, P->aca_ncoop, true, (ArgMax*)((char*)S.aca_part + off), bar, flags, s));
      }
    }
  }
  if (P->aca_nsolo > 0)
    CK(launch_aca(H0, P->aca_work + P->aca_ncoop, P->aca_nsolo, false, S.aca_part, S.aca_bar, S.flags, s, nprob,
                  sstride));
  if (P->aca_nwarp > 0) CK(launch_aca_warp(H0, P->aca_work + P->aca_ncoop + P->aca_nsolo, P->aca_nwarp, s, nprob));
  return FIFA_OK;
}

static double kernel_const(int kind, double rho) { return kind == 0 ? 0.5 / (rho * rho) : sqrt(5.0) / rho; }

extern "C" fifa_status fifa_assemble(fifa_ctx* ctx, const double* x_dev, int64_t n, const fifa_hyper* hyper,
                                     fifa_hmat** out) {
  if (!ctx || !x_dev || !hyper || !out || n < 1) return FIFA_ERR_INVALID_ARG;
  *out = nullptr;
  if (hyper->kernel != 0 && hyper->kernel != 1) return FIFA_ERR_INVALID_ARG;
  if (!(hyper->rho > 0.0) || !(hyper->nugget >= 0.0) || !isfinite(hyper->rho)) return FIFA_ERR_INVALID_ARG;
  if (n > (int64_t)1 << 30) return FIFA_ERR_UNSUPPORTED;
  // sortedness / finiteness check (synchronous)
  CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int), ctx->stream));
  CK(launch_check_sorted(x_dev, n, ctx->flags, ctx->stream));
  CK(cudaMemcpyAsync(ctx->host_flags, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->host_flags[0] & 2) return FIFA_ERR_INVALID_ARG;
  if (ctx->host_flags[0] & 1) return FIFA_ERR_UNSORTED;
  fifa_status st = FIFA_OK;
  Plan* P = get_plan(ctx, n, &st);
  if (!P) return st;
  fifa_hmat* H = nullptr;
  st = hmat_alloc(ctx, P, hyper->kernel, &H);
  if (st != FIFA_OK) return st;
  H->host.x = x_dev;
  H->host.rho = hyper->rho;
  H->host.kc = kernel_const(hyper->kernel, hyper->rho);
  H->host.nugget = hyper->nugget;
  st = upload_desc(ctx, H);
  if (st == FIFA_OK) st = hmat_assemble_enqueue(ctx, H);
  if (st != FIFA_OK) {
    fifa_destroy_hmat(ctx, H);
    return st;
  }
  *out = H;
  return FIFA_OK;
}

extern "C" fifa_status fifa_shift_scale(fifa_ctx* ctx, const fifa_hmat* C, double s, fifa_hmat** M) {
  if (!ctx || !C || !M || !isfinite(s)) return FIFA_ERR_INVALID_ARG;
  if (C->host.shift != 0.0 || C->host.scale != 1.0) return FIFA_ERR_INVALID_ARG;
  fifa_hmat* H = new (std::nothrow) fifa_hmat();
  if (!H) return FIFA_ERR_OOM;
  H->plan = C->plan;
  H->host = C->host;
  H->host.scale = s;
  H->host.shift = 1.0;
  H->owns = false;
  H->base = C;
  H->dev = (HmatDesc*)ctx->arena.alloc(sizeof(HmatDesc));
  if (!H->dev) {
    delete H;
    return FIFA_ERR_OOM;
  }
  fifa_status st = upload_desc(ctx, H);
  if (st != FIFA_OK) {
    fifa_destroy_hmat(ctx, H);
    return st;
  }
  *M = H;
  return FIFA_OK;
}

extern "C" fifa_status fifa_add_diagonal(fifa_ctx* ctx, const fifa_hmat* C, double s, const double* diag_dev,
                                         fifa_hmat** P) {
  if (!ctx || !C || !P || !diag_dev || !isfinite(s)) return FIFA_ERR_INVALID_ARG;
  if (C->host.shift != 0.0 || C->host.scale != 1.0 || C->host.diag) return FIFA_ERR_INVALID_ARG;
  fifa_hmat* H = new (std::nothrow) fifa_hmat();
  if (!H) return FIFA_ERR_OOM;
  H->plan = C->plan;
  H->host = C->host;
  H->host.scale = s;
  H->host.shift = 0.0;
  H->host.diag = diag_dev;
  H->owns = false;
  H->base = C;
  H->dev = (HmatDesc*)ctx->arena.alloc(sizeof(HmatDesc));
  if (!H->dev) {
    delete H;
    return FIFA_ERR_OOM;
  }
  fifa_status st = upload_desc(ctx, H);
  if (st != FIFA_OK) {
    fifa_destroy_hmat(ctx, H);
    return st;
  }
  *P = H;
  return FIFA_OK;
}

extern "C" void fifa_destroy_hmat(fifa_ctx* ctx, fifa_hmat* H) {
  if (!ctx || !H) return;
  cudaStreamSynchronize(ctx->stream);
  if (H->owns) {
    ctx->arena.release(H->host.leaves);
    ctx->arena.release(H->host.bases);
    ctx->arena.release(H->host.rank);
    ctx->arena.release(H->host.row_piv);
    ctx->arena.release(H->host.col_piv);
    ctx->arena.release(H->host.status);
  }
  ctx->arena.release(H->dev);
  delete H;
}

// ---------------------------------------------------------------------------
// Factor
// ---------------------------------------------------------------------------
fifa_status fact_alloc(fifa_ctx* ctx, Plan* P, int with32, fifa_fact** out) {
  fifa_fact* F = new (std::nothrow) fifa_fact();
  if (!F) return FIFA_ERR_OOM;
  F->plan = P;
  const int cap = ctx->opts.rank_cap;
  const size_t nn = std::max(1, P->nnodes);
  FactDesc& d = F->host;
  memset(&d, 0, sizeof(d));
  d.n = P->n;
  d.L = P->L;
  d.nleaf = P->nleaf;
  d.Bm = P->Bm;
  d.cap = cap;
  d.prec = 0;
  d.bnd = P->bnd_dev;
  d.skip = nullptr;
  d.spin = ctx->opts.wait_polls > 0 ? (unsigned int)ctx->opts.wait_polls : 0u;
  d.Lleaf = ctx->arena.alloc(sizeof(double) * (size_t)P->nleaf * P->Bm * P->Bm);
  d.Ldinv = ctx->arena.alloc(sizeof(double) * (size_t)P->nleaf * P->Bm);
  d.Q = ctx->arena.alloc(sizeof(double) * (size_t)std::max(1, P->L) * cap * P->n);
  d.Zf = (double*)ctx->arena.alloc(sizeof(double) * nn * 4 * cap * cap);
  d.Zi = (double*)ctx->arena.alloc(sizeof(double) * nn * 4 * cap * cap);
  d.rank = (int*)ctx->arena.alloc(sizeof(int) * nn);
  d.ld_parts = (double*)ctx->arena.alloc(sizeof(double) * (P->nleaf + nn));
  d.logdet = (double*)ctx->arena.alloc(sizeof(double));
  d.status = (int*)ctx->arena.alloc(sizeof(int));
  F->dev = (FactDesc*)ctx->arena.alloc(sizeof(FactDesc));
  if (!d.Lleaf || !d.Ldinv || !d.Q || !d.Zf || !d.Zi || !d.rank || !d.ld_parts || !d.logdet || !d.status || !F->dev) {
    fifa_destroy_fact(ctx, F);
    return FIFA_ERR_OOM;
  }
  if (with32) {
    F->has32 = true;
    FactDesc& h = F->host32;
    h = d;  // Zf, Zi, ranks, log-determinant and status are the FP64 factor's
    h.prec = 1;
    h.skip = nullptr;
    h.Lleaf = ctx->arena.alloc(sizeof(float) * (size_t)P->nleaf * P->Bm * P->Bm);
    h.Ldinv = ctx->arena.alloc(sizeof(float) * (size_t)P->nleaf * P->Bm);
    h.Q = ctx->arena.alloc(sizeof(float) * (size_t)std::max(1, P->L) * cap * P->n);
    F->dev32 = (FactDesc*)ctx->arena.alloc(sizeof(FactDesc));
    if (!h.Lleaf || !h.Ldinv || !h.Q || !F->dev32) {
      fifa_destroy_fact(ctx, F);
      return FIFA_ERR_OOM;
    }
    CK(cudaMemcpyAsync(F->dev32, &F->host32, sizeof(FactDesc), cudaMemcpyHostToDevice, ctx->stream));
  }
  CK(cudaMemcpyAsync(F->dev, &F->host, sizeof(FactDesc), cudaMemcpyHostToDevice, ctx->stream));
  *out = F;
  return FIFA_OK;
}

fifa_status fact_set_skip(fifa_ctx* ctx, fifa_fact* F, const int* skip_dev) {
  F->host.skip = skip_dev;
  CK(cudaMemcpyAsync(F->dev, &F->host, sizeof(FactDesc), cudaMemcpyHostToDevice, ctx->stream));
  return FIFA_OK;
}

// Enqueue the factorization of the (possibly view) matrix described by Hdev.
fifa_status fact_enqueue(fifa_ctx* ctx, fifa_fact* F, const HmatDesc* Hdev) {
  fifa_status st = fact_enqueue_part(ctx, F, Hdev, 0);
  return st == FIFA_OK ? fact_enqueue_part(ctx, F, Hdev, 1) : st;
}

// The deepest level whose level kernels split no node over a CTA group: levels
// >= it run with independent CTAs (groups only ever take the top levels).
int fact_ungrouped_from(const Plan* P) {
  int l = P->L;
  while (l > 0) {
    const int q = l - 1;
    if (std::max({P->lvl_G[0][q], P->lvl_G[1][q], P->lvl_G[2][q]}) > 1) break;
    l = q;
  }
  return l;
}

// part 0: descriptor reset, leaves and the levels from the deepest up to
// fact_ungrouped_from (independent CTAs only); part 1: the grouped levels
// above, the log-determinant and the FP32 copy.  Part 1 after part 0.
fifa_status fact_enqueue_part(fifa_ctx* ctx, fifa_fact* F, const HmatDesc* Hdev, int part) {
  Plan* P = F->plan;
  fifa_status st = ensure_scratch(ctx, P);
  if (st != FIFA_OK) return st;
  Scratch S = carve(ctx, P);
  cudaStream_t s = ctx->stream;
  const int prec = F->host.prec, cap = ctx->opts.rank_cap;
  const int lsplit = fact_ungrouped_from(P);
  if (part == 0) {
    CK(launch_prep_fact(F->dev, Hdev, P->nnodes, s));
    CK(launch_leaf_factor(Hdev, F->dev, prec, P->nleaf, P->Bm, P->L, cap, s));
  }
  const int lhi = part == 0 ? P->L - 1 : lsplit - 1, llo = part == 0 ? lsplit : 0;
  for (int l = lhi; l >= llo; --l) {
    const int Gb[LEVEL_BUCKETS] = {P->lvl_G[0][l], P->lvl_G[1][l], P->lvl_G[2][l]};
    if (*std::max_element(Gb, Gb + LEVEL_BUCKETS) > 1) {  // every rank bucket has its own barrier set
      CK(cudaMemsetAsync(S.lvl_bar, 0, sizeof(unsigned int) * LEVEL_BUCKETS * P->lvl_ctas_max, s));
      CK(cudaMemsetAsync(S.flags, 0, sizeof(int), s));
    }
    const int side_max = (int)(((n_of(P) + ((int64_t)1 << l) - 1) >> l) + 1) / 2;
    CK(launch_level(F->dev, prec, l, 1 << l, Gb, cap, S.lvl_part, S.lvl_bar, P->lvl_ctas_max, S.flags, side_max, s));
  }
  if (part == 0) return FIFA_OK;
  CK(launch_logdet_reduce(F->dev, s));
  if (F->has32) CK(launch_demote(F->dev, F->dev32, P->n, s));
  return FIFA_OK;
}

// Factor nprob matrices of one plan in one launch per step and tree level:
// F0[q] from H0[q] (contiguous descriptor arrays), problem q's scratch at
// scratch0 + q * sstride bytes.  Groups shrink to fit all problems' CTAs.
fifa_status fact_enqueue_batched(fifa_ctx* ctx, Plan* P, FactDesc* F0, const HmatDesc* H0, int nprob,
                                 void* scratch0, size_t sstride, const FactDesc* F32_0) {
  const int prec = 0;
  void* saved = ctx->active_scratch;
  ctx->active_scratch = scratch0;
  Scratch S = carve(ctx, P);
  ctx->active_scratch = saved;
  cudaStream_t s = ctx->stream;
  const int cap = ctx->opts.rank_cap;
  CK(launch_prep_fact(F0, H0, P->nnodes, s, nprob));
  CK(launch_leaf_factor(H0, F0, prec, P->nleaf, P->Bm, P->L, cap, s, nprob));
  for (int l = P->L - 1; l >= 0; --l) {
    int Gb[LEVEL_BUCKETS];
    for (int b = 0; b < LEVEL_BUCKETS; ++b) Gb[b] = std::max(1, P->lvl_G[b][l] / nprob);
    if (*std::max_element(Gb, Gb + LEVEL_BUCKETS) > 1) {
      CK(cudaMemset2DAsync(S.lvl_bar, sstride, 0, sizeof(unsigned int) * LEVEL_BUCKETS * P->lvl_ctas_max, nprob, s));
      CK(cudaMemset2DAsync(S.flags, sstride, 0, sizeof(int), nprob, s));
    }
    const int side_max = (int)(((n_of(P) + ((int64_t)1 << l) - 1) >> l) + 1) / 2;
    CK(launch_level(F0, prec, l, 1 << l, Gb, cap, S.lvl_part, S.lvl_bar, P->lvl_ctas_max, S.flags, side_max, s, nprob,
                    sstride));
  }
  CK(launch_logdet_reduce(F0, s, nprob));
  if (F32_0) CK(launch_demote(F0, F32_0, P->n, s, nprob));
  return FIFA_OK;
}

extern "C" fifa_status fifa_factor(fifa_ctx* ctx, const fifa_hmat* A, fifa_fact** out) {
  if (!ctx || !A || !out) return FIFA_ERR_INVALID_ARG;
  *out = nullptr;
  const int with32 = (ctx->opts.prec == FIFA_MIXED && (A->host.shift != 0.0 || A->host.diag)) ? 1 : 0;
  fifa_fact* F = nullptr;
  fifa_status st = fact_alloc(ctx, A->plan, with32, &F);
  if (st != FIFA_OK) return st;
  F->src = A;
  st = fact_enqueue(ctx, F, A->dev);
  if (st != FIFA_OK) {
    fifa_destroy_fact(ctx, F);
    return st;
  }
  *out = F;
  return FIFA_OK;
}

extern "C" void fifa_destroy_fact(fifa_ctx* ctx, fifa_fact* F) {
  if (!ctx || !F) return;
  cudaStreamSynchronize(ctx->stream);
  FactDesc& d = F->host;
  ctx->arena.release(d.Lleaf);
  ctx->arena.release(d.Ldinv);
  ctx->arena.release(d.Q);
  ctx->arena.release(d.Zf);
  ctx->arena.release(d.Zi);
  ctx->arena.release(d.rank);
  ctx->arena.release(d.ld_parts);
  ctx->arena.release(d.logdet);
  ctx->arena.release(d.status);
  ctx->arena.release(F->dev);
  if (F->has32) {
    ctx->arena.release(F->host32.Lleaf);
    ctx->arena.release(F->host32.Ldinv);
    ctx->arena.release(F->host32.Q);
    ctx->arena.release(F->dev32);
  }
  delete F;
}

extern "C" fifa_status fifa_logdet(fifa_ctx* ctx, const fifa_fact* F, double* out_host) {
  if (!ctx || !F || !out_host) return FIFA_ERR_INVALID_ARG;
  double* hb = (double*)ctx->host_flags;
  CK(cudaMemcpyAsync(hb, F->host.logdet, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(ctx->host_flags + 4, F->host.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *out_host = hb[0];
  return dev_status_to_api(ctx->host_flags[4]);
}

// ---------------------------------------------------------------------------
// Sweeps, solve, matvec
// ---------------------------------------------------------------------------
bool sweep_batch_config(fifa_ctx* ctx, const Plan* P, int nprob, int* ls, int* rows) {
  if (P->fs_ls < 0 || nprob < 1) return false;
  for (int k = P->fs_ls; k >= 0; --k) {
    int r = 0;
    for (int i = 0; i < (1 << k); ++i) r = std::max(r, P->bnd_host[bnd_off(k) + i + 1] - P->bnd_host[bnd_off(k) + i]);
    if ((int64_t)(sweep_fused_coresident(0, r, ctx->opts.rank_cap) / coresident_share(ctx->opts)) >=
        ((int64_t)nprob << k)) {
      *ls = k;
      *rows = r;
      return true;
    }
  }
  return false;
}

fifa_status sweep_enqueue_batched(fifa_ctx* ctx, Plan* P, const FactDesc* F0, double* const* vlist, int nprob,
                                  int mode, int ls, int rows, void* scratch0, size_t sstride) {
  void* saved = ctx->active_scratch;
  ctx->active_scratch = scratch0;
  Scratch S = carve(ctx, P);
  ctx->active_scratch = saved;
  cudaStream_t s = ctx->stream;
  CK(cudaMemset2DAsync(S.fs_bar, sstride, 0, sizeof(unsigned int), nprob, s));
  CK(cudaMemset2DAsync(S.flags, sstride, 0, sizeof(int), nprob, s));
  CK(launch_sweep_fused_batched(F0, ls, rows, vlist, nprob, mode, S.fs_part, S.fs_bar, S.flags, sstride, s));
  return FIFA_OK;
}

fifa_status sweep_enqueue_desc(fifa_ctx* ctx, Plan* P, const FactDesc* Fdev, int prec, int mode, double* v, int nrhs,
                               const int* active) {
  Scratch S = carve(ctx, P);
  cudaStream_t s = ctx->stream;
  if (P->fs_ls >= 0) {
    CK(cudaMemsetAsync(S.fs_bar, 0, sizeof(unsigned int), s));
    CK(cudaMemsetAsync(S.flags, 0, sizeof(int), s));
    CK(launch_sweep_fused(Fdev, prec, P->fs_ls, P->fs_rows, ctx->opts.rank_cap, v, nrhs, mode, S.fs_part, S.fs_bar,
                          S.flags, s, active));
    return FIFA_OK;
  }
  auto level = [&](int l, int zsel, int zt) -> cudaError_t {
    return launch_sweep_level(Fdev, prec, l, 1 << l, P->sweep_G[l], v, nrhs, S.sweep_part, zsel, zt, s, active);
  };
  auto one = [&](int md) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    if (md == 0) {
      for (int l = 0; l < P->L && e == cudaSuccess; ++l) e = level(l, 0, 0);
      if (e == cudaSuccess) e = launch_sweep_leaf(Fdev, prec, P->nleaf, v, nrhs, 0, s, active);
    } else if (md == 1) {
      e = launch_sweep_leaf(Fdev, prec, P->nleaf, v, nrhs, 1, s, active);
      for (int l = P->L - 1; l >= 0 && e == cudaSuccess; --l) e = level(l, 1, 0);
    } else if (md == 2) {
      e = launch_sweep_leaf(Fdev, prec, P->nleaf, v, nrhs, 2, s, active);
      for (int l = P->L - 1; l >= 0 && e == cudaSuccess; --l) e = level(l, 0, 1);
    } else {
      for (int l = 0; l < P->L && e == cudaSuccess; ++l) e = level(l, 1, 1);
      if (e == cudaSuccess) e = launch_sweep_leaf(Fdev, prec, P->nleaf, v, nrhs, 3, s, active);
    }
    return e;
  };
  if (mode == 4) {
    CK(one(1));
    CK(one(3));
  } else {
    CK(one(mode));
  }
  return FIFA_OK;
}

// W^-1 v of an FP64 factor in two parts around its grouped top levels: part 0
// (leaves and the levels the fused sweep keeps inside a CTA) needs only the
// factor's levels from fact_ungrouped_from down, part 1 the rest.  Possible
// when the fused sweep's local levels lie in that range.
bool sweep_inverse_split_ok(const Plan* P) { return P->fs_ls >= 0 && P->fs_ls >= fact_ungrouped_from(P); }

fifa_status sweep_inverse_part_enqueue(fifa_ctx* ctx, const fifa_fact* F, double* v, int part) {
  Plan* P = F->plan;
  if (!sweep_inverse_split_ok(P) || F->host.prec != 0) return FIFA_ERR_INVALID_ARG;
  return sweep_enqueue_desc(ctx, P, F->dev, 0, part == 0 ? 5 : 6, v, 1);
}

fifa_status sweep_enqueue(fifa_ctx* ctx, const fifa_fact* F, int trans, int inverse, double* v, int nrhs) {
  const int mode = trans ? (inverse ? 3 : 2) : (inverse ? 1 : 0);
  return sweep_enqueue_desc(ctx, F->plan, F->dev, F->host.prec, mode, v, nrhs);
}

extern "C" fifa_status fifa_apply_W(fifa_ctx* ctx, const fifa_fact* F, int trans, int inverse, const double* in_dev,
                                    double* out_dev, int nrhs) {
  if (!ctx || !F || !in_dev || !out_dev || nrhs < 1 || nrhs > SWEEP_RHS_MAX) return FIFA_ERR_INVALID_ARG;
  fifa_status st = ensure_scratch(ctx, F->plan);
  if (st != FIFA_OK) return st;
  if (in_dev != out_dev)
    CK(cudaMemcpyAsync(out_dev, in_dev, sizeof(double) * F->plan->n * nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
  return sweep_enqueue(ctx, F, trans ? 1 : 0, inverse ? 1 : 0, out_dev, nrhs);
}

extern "C" fifa_status fifa_apply_precond(fifa_ctx* ctx, const fifa_fact* F, const double* in_dev, double* out_dev,
                                          int nrhs) {
  if (!ctx || !F || !F->has32 || !in_dev || !out_dev || nrhs < 1 || nrhs > SWEEP_RHS_MAX) return FIFA_ERR_INVALID_ARG;
  fifa_status st = ensure_scratch(ctx, F->plan);
  if (st != FIFA_OK) return st;
  if (in_dev != out_dev)
    CK(cudaMemcpyAsync(out_dev, in_dev, sizeof(double) * F->plan->n * nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
  return sweep_enqueue_desc(ctx, F->plan, F->dev32, 1, 4, out_dev, nrhs);
}

fifa_status matvec_enqueue(fifa_ctx* ctx, const fifa_hmat* A, const double* in, double* out, int nrhs,
                           const int* active) {
  Plan* P = A->plan;
  Scratch S = carve(ctx, P);
  if (P->mv_ls >= 0) {
    CK(cudaMemsetAsync(S.mv_bar, 0, sizeof(unsigned int), ctx->stream));
    CK(cudaMemsetAsync(S.flags, 0, sizeof(int), ctx->stream));
    CK(launch_mv_fused(A->dev, P->mv_ls, P->mv_rows, in, nrhs, out, S.mv_fpart, S.mv_bar, S.flags, ctx->stream,
                       active));
    return FIFA_OK;
  }
  CK(launch_matvec(A->dev, P->nleaf, P->L, in, nrhs, S.mv_part, S.mv_proj, out, ctx->stream, active));
  return FIFA_OK;
}

extern "C" fifa_status fifa_matvec(fifa_ctx* ctx, const fifa_hmat* A, const double* in_dev, double* out_dev, int nrhs) {
  if (!ctx || !A || !in_dev || !out_dev || in_dev == out_dev || nrhs < 1 || nrhs > SWEEP_RHS_MAX)
    return FIFA_ERR_INVALID_ARG;
  fifa_status st = ensure_scratch(ctx, A->plan);
  if (st != FIFA_OK) return st;
  return matvec_enqueue(ctx, A, in_dev, out_dev, nrhs);
}

// x = A^-1 b.  FP64 factor: W^-T W^-1 b (two sweeps, or one fused launch).
// Mixed factor: conjugate gradients on the FP64 operator (op, default the
// factored matrix) preconditioned by W32 W32^T, the FP32 copy of the factor
// applied in FP32 arithmetic: x0 = P^-1 b, then refine_max captured
// iterations; once every system meets ||r|| <= refine_tol ||b|| the remaining
// iterations' launches return at once.  work holds 4 n nrhs doubles (r, z, p,
// q); b must not alias x for a mixed factor.
fifa_status solve_enqueue(fifa_ctx* ctx, const fifa_fact* F, const double* b, double* x, int nrhs, double* work,
                          double* res_dev, int* iters_dev, const fifa_hmat* op, bool true_res) {
  Plan* P = F->plan;
  const int64_t n = P->n;
  const int64_t nn = n * nrhs;
  cudaStream_t s = ctx->stream;
  if (x != b) CK(cudaMemcpyAsync(x, b, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  if (!F->has32) return sweep_enqueue_desc(ctx, P, F->dev, 0, 4, x, nrhs);
  if (!op) op = F->src;
  if (!op || x == b) return FIFA_ERR_INVALID_ARG;
  Scratch S = carve(ctx, P);
  double* part = S.pcg;
  double* st = S.pcg + PCG_OFF_STATE;  // two parity slots of PCG_RHS_MAX * PCG_SLOT doubles
  int* ints = (int*)(S.pcg + PCG_OFF_INTS);
  int* act = ints;        // act[2]
  int* iters = ints + 2;  // iterations taken
  int* act_sw = ints + 3; // this step's preconditioner needed
  double* r = work;
  double* z = work + nn;
  double* p = work + 2 * nn;
  double* q = work + 3 * nn;
  const double tol = ctx->opts.refine_tol > 0.0 ? ctx->opts.refine_tol : 1e-12;
  const double tol2 = tol * tol;
  fifa_status e = sweep_enqueue_desc(ctx, P, F->dev32, 1, 4, x, nrhs);  // x0 = P^-1 b
  if (e != FIFA_OK) return e;
  if ((e = matvec_enqueue(ctx, op, x, r, nrhs)) != FIFA_OK) return e;
  CK(launch_pcg_residual0(b, r, z, n, nrhs, part, s));  // r = b - A x0, z = r
  if ((e = sweep_enqueue_desc(ctx, P, F->dev32, 1, 4, z, nrhs)) != FIFA_OK) return e;
  CK(launch_pcg_start(r, z, p, n, nrhs, part, st, act, iters, tol2, s));
  const int slot = PCG_RHS_MAX * PCG_SLOT;
  for (int it = 0; it < ctx->opts.refine_max; ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    if ((e = matvec_enqueue(ctx, op, p, q, nrhs, act + cur)) != FIFA_OK) return e;
    CK(launch_pcg_pq(p, q, n, nrhs, part, act + cur, s));
    CK(launch_pcg_update(x, r, z, p, q, n, nrhs, st + cur * slot, part, act + cur, act_sw, tol2, s));
    if ((e = sweep_enqueue_desc(ctx, P, F->dev32, 1, 4, z, nrhs, act_sw)) != FIFA_OK) return e;
    CK(launch_pcg_direction(r, p, z, n, nrhs, st + cur * slot, st + nxt * slot, act + cur, act + nxt, iters, part,
                            tol2, s));
  }
  if (res_dev || iters_dev) {
    if (true_res) {  // ||b - A x|| / ||b|| with one more FP64 product
      if ((e = matvec_enqueue(ctx, op, x, q, nrhs)) != FIFA_OK) return e;
      CK(launch_pcg_true_residual(b, q, n, nrhs, part, res_dev, iters, iters_dev, s));
    } else {  // the iteration's own (recursive) residual
      CK(launch_pcg_recursive_residual(st + (ctx->opts.refine_max & 1) * slot, nrhs, res_dev, iters, iters_dev, s));
    }
  }
  return FIFA_OK;
}

extern "C" fifa_status fifa_solve(fifa_ctx* ctx, const fifa_fact* F, const double* b_dev, double* x_dev, int nrhs) {
  if (!ctx || !F || !b_dev || !x_dev || nrhs < 1 || nrhs > SWEEP_RHS_MAX) return FIFA_ERR_INVALID_ARG;
  fifa_status st = ensure_scratch(ctx, F->plan);
  if (st != FIFA_OK) return st;
  Scratch S = carve(ctx, F->plan);
  const int64_t n = F->plan->n;
  const double* b = b_dev;
  if (b_dev == x_dev && F->has32) {  // the iteration needs the original right-hand side
    CK(cudaMemcpyAsync(S.vec + 8 * n, b_dev, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
    b = S.vec + 8 * n;
  }
  return solve_enqueue(ctx, F, b, x_dev, nrhs, S.vec);
}

// ---------------------------------------------------------------------------
// Algorithm 1
// ---------------------------------------------------------------------------
fifa_status sample_prior_enqueue(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, double tau2, double sigma2,
                                 uint64_t seed, uint64_t sid, const uint64_t* iter_dev, uint64_t iter_host,
                                 const double* scal_dev) {
  Plan* P = C->plan;
  const int64_t n = P->n;
  Scratch S = carve(ctx, P);
  cudaStream_t s = ctx->stream;
  double* a = S.vec;           // n
  double* b = S.vec + n;       // n
  double* Ca = S.vec + 2 * n;  // n
  double* rhs = S.vec + 3 * n; // 2n : [Z, y/sigma2] -> [w, r]
  CK(launch_normals(seed, 0, iter_dev, iter_host, sid, a, n, s));
  CK(launch_normals(seed, 1, iter_dev, iter_host, sid, b, n, s));
  fifa_status st = matvec_enqueue(ctx, C, a, Ca, 1);
  if (st != FIFA_OK) return st;
  st = sweep_enqueue(ctx, WC, 0, 0, b, 1);
  if (st != FIFA_OK) return st;
  // rhs0 = (tau2/sigma) Ca + tau Wb
  CK(launch_alg1_rhs_part(Ca, b, nullptr, rhs, n, tau2, sigma2, scal_dev, 0, s));
  return FIFA_OK;
}

fifa_status sample_data_enqueue(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WM, const double* y, double tau2,
                                double sigma2, double* f, double* mean, const double* scal_dev, double* res_dev,
                                int* iters_dev, const fifa_hmat* op) {
  Plan* P = C->plan;
  const int64_t n = P->n;
  Scratch S = carve(ctx, P);
  cudaStream_t s = ctx->stream;
  double* rhs = S.vec + 3 * n;    // 2n : [Z, y/sigma2] -> [w, r]
  double* Cr = S.vec + 5 * n;     // n
  double* bsave = S.vec + 6 * n;  // 2n (iteration right-hand sides)
  double* work = S.vec + 8 * n;   // 8n (conjugate-gradient vectors)
  // rhs1 = y / sigma2
  CK(launch_alg1_rhs_part(nullptr, nullptr, y, rhs, n, tau2, sigma2, scal_dev, 1, s));
  fifa_status st;
  if (WM->has32) {
    CK(cudaMemcpyAsync(bsave, rhs, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, s));
    st = solve_enqueue(ctx, WM, bsave, rhs, 2, work, res_dev, iters_dev, op, false);
  } else {
    st = solve_enqueue(ctx, WM, rhs, rhs, 2, work);
  }
  if (st != FIFA_OK) return st;
  st = matvec_enqueue(ctx, C, rhs + n, Cr, 1);
  if (st != FIFA_OK) return st;
  CK(launch_alg1_finish(rhs, Cr, f, mean, n, tau2, scal_dev, s));
  return FIFA_OK;
}

fifa_status sample_enqueue(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, const fifa_fact* WM, const double* y,
                           double tau2, double sigma2, uint64_t seed, uint64_t sid, const uint64_t* iter_dev,
                           uint64_t iter_host, double* f, double* mean, const double* scal_dev, double* res_dev,
                           int* iters_dev, const fifa_hmat* op) {
  fifa_status st = sample_prior_enqueue(ctx, C, WC, tau2, sigma2, seed, sid, iter_dev, iter_host, scal_dev);
  if (st != FIFA_OK) return st;
  return sample_data_enqueue(ctx, C, WM, y, tau2, sigma2, f, mean, scal_dev, res_dev, iters_dev, op);
}

bool mv_batch_config(fifa_ctx* ctx, const Plan* P, int nprob, int* ls, int* rows) {
  (void)ctx;
  if (P->mv_ls < 0 || nprob < 1) return false;
  for (int k = P->mv_ls; k >= 0; --k) {
    int r = 0;
    for (int i = 0; i < (1 << k); ++i) r = std::max(r, P->bnd_host[bnd_off(k) + i + 1] - P->bnd_host[bnd_off(k) + i]);
    if (r > MV_FUSED_ROWS_MAX) return false;
    if ((int64_t)(mv_fused_coresident(r) / coresident_share(ctx->opts)) >= ((int64_t)nprob << k)) {
      *ls = k;
      *rows = r;
      return true;
    }
  }
  return false;
}

fifa_status sample_prior_batched(fifa_ctx* ctx, Plan* P, const HmatDesc* C0, const FactDesc* WC0, const Alg1Prior* P_dev,
                                 const double* const* a_list, double* const* b_list, double* const* Ca_list, int nprob,
                                 uint64_t seed, int sweep_ls, int sweep_rows, int mv_ls, int mv_rows, void* scratch0,
                                 size_t sstride, const fifa_hmat* const* C_each, const fifa_fact* const* WC_each) {
  const int64_t n = P->n;
  cudaStream_t s = ctx->stream;
  CK(launch_alg1_prior_normals(seed, P_dev, nprob, n, s));
  void* saved = ctx->active_scratch;
  ctx->active_scratch = scratch0;
  Scratch S = carve(ctx, P);
  ctx->active_scratch = saved;
  fifa_status st = FIFA_OK;
  if (mv_ls >= 0) {  // C~ a for every block in one launch
    CK(cudaMemset2DAsync(S.mv_bar, sstride, 0, sizeof(unsigned int), nprob, s));
    CK(cudaMemset2DAsync(S.flags, sstride, 0, sizeof(int), nprob, s));
    CK(launch_mv_fused_batched(C0, mv_ls, mv_rows, a_list, Ca_list, nprob, S.mv_fpart, S.mv_bar, S.flags, sstride, s));
  }
  if (sweep_ls >= 0)  // W_C b for every block in one launch
    st = sweep_enqueue_batched(ctx, P, WC0, b_list, nprob, 0, sweep_ls, sweep_rows, scratch0, sstride);
  // blocks without a shared launch: one product / sweep each, on their own scratch
  for (int q = 0; q < nprob && st == FIFA_OK && (mv_ls < 0 || sweep_ls < 0); ++q) {
    ctx->active_scratch = (char*)scratch0 + (size_t)q * sstride;
    Scratch Sq = carve(ctx, P);
    if (mv_ls < 0) st = matvec_enqueue(ctx, C_each[q], Sq.vec, Sq.vec + 2 * n, 1);
    if (st == FIFA_OK && sweep_ls < 0) st = sweep_enqueue(ctx, WC_each[q], 0, 0, Sq.vec + n, 1);
  }
  ctx->active_scratch = saved;
  if (st != FIFA_OK) return st;
  CK(launch_alg1_prior_rhs(P_dev, nprob, n, s));
  return FIFA_OK;
}

// Algorithm 1.h (Appendix "Heteroskedastic noise derivation"), noise precisions d.
fifa_status sample_hetero_enqueue(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, const fifa_fact* WP,
                                  const double* y, double tau2, const double* d, uint64_t seed, uint64_t sid,
                                  const uint64_t* iter_dev, uint64_t iter_host, double* f, double* R,
                                  double* res_dev, int* iters_dev) {
  Plan* P = C->plan;
  const int64_t n = P->n;
  Scratch S = carve(ctx, P);
  cudaStream_t s = ctx->stream;
  double* a = S.vec;              // n: a0, then a = sqrt(d) a0
  double* b = S.vec + n;          // n: b, then W_C b
  double* Ca = S.vec + 2 * n;     // n
  double* rhs = S.vec + 3 * n;    // 2n: [Z, y] -> [Z*, P~^-1 y]
  double* Cr = S.vec + 5 * n;     // n
  double* bsave = S.vec + 6 * n;  // 2n
  double* work = S.vec + 8 * n;   // 8n
  CK(launch_normals(seed, 0, iter_dev, iter_host, sid, a, n, s));
  CK(launch_normals(seed, 1, iter_dev, iter_host, sid, b, n, s));
  CK(launch_alg1h_scale(d, a, n, s));
  fifa_status st = matvec_enqueue(ctx, C, a, Ca, 1);
  if (st != FIFA_OK) return st;
  if ((st = sweep_enqueue(ctx, WC, 0, 0, b, 1)) != FIFA_OK) return st;
  CK(launch_alg1h_rhs(Ca, b, y, rhs, n, tau2, s));
  if (WP->has32) {
    CK(cudaMemcpyAsync(bsave, rhs, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, s));
    st = solve_enqueue(ctx, WP, bsave, rhs, 2, work, res_dev, iters_dev);
  } else {
    st = solve_enqueue(ctx, WP, rhs, rhs, 2, work);
  }
  if (st != FIFA_OK) return st;
  if ((st = matvec_enqueue(ctx, C, rhs + n, Cr, 1)) != FIFA_OK) return st;
  CK(launch_alg1h_finish(rhs, Cr, d, f, R, n, tau2, s));
  return FIFA_OK;
}

extern "C" fifa_status fifa_sample_hetero(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, const fifa_fact* WP,
                                          const double* y_dev, double tau2, const double* d_dev, uint64_t seed,
                                          uint64_t stream_id, uint64_t iter, double* f_dev, double* R_dev) {
  if (!ctx || !C || !WC || !WP || !y_dev || !d_dev || !f_dev || !(tau2 > 0.0)) return FIFA_ERR_INVALID_ARG;
  if (C->plan != WC->plan || C->plan != WP->plan || C->host.diag || C->host.shift != 0.0) return FIFA_ERR_INVALID_ARG;
  fifa_status st = ensure_scratch(ctx, C->plan);
  if (st != FIFA_OK) return st;
  return sample_hetero_enqueue(ctx, C, WC, WP, y_dev, tau2, d_dev, seed, stream_id, nullptr, iter, f_dev, R_dev);
}

extern "C" fifa_status fifa_sample(fifa_ctx* ctx, const fifa_hmat* C, const fifa_fact* WC, const fifa_fact* WM,
                                   const double* y_dev, double tau2, double sigma2, uint64_t seed, uint64_t stream_id,
                                   uint64_t iter, double* f_dev, double* mean_dev) {
  if (!ctx || !C || !WC || !WM || !y_dev || !f_dev || !(tau2 > 0.0) || !(sigma2 > 0.0)) return FIFA_ERR_INVALID_ARG;
  if (C->plan != WC->plan || C->plan != WM->plan) return FIFA_ERR_INVALID_ARG;
  fifa_status st = ensure_scratch(ctx, C->plan);
  if (st != FIFA_OK) return st;
  return sample_enqueue(ctx, C, WC, WM, y_dev, tau2, sigma2, seed, stream_id, nullptr, iter, f_dev, mean_dev, nullptr);
}

// ---------------------------------------------------------------------------
// Introspection
// ---------------------------------------------------------------------------
extern "C" fifa_status fifa_hmat_dims(const fifa_hmat* H, int64_t* n, int* levels, int* nleaf, int* leaf_max,
                                      int* rank_cap) {
  if (!H) return FIFA_ERR_INVALID_ARG;
  if (n) *n = H->plan->n;
  if (levels) *levels = H->plan->L;
  if (nleaf) *nleaf = H->plan->nleaf;
  if (leaf_max) *leaf_max = H->plan->Bm;
  if (rank_cap) *rank_cap = H->host.cap;
  return FIFA_OK;
}

extern "C" fifa_status fifa_hmat_level_rows(fifa_ctx* ctx, const fifa_hmat* H, int level, int64_t row0,
                                            int64_t nrows, double* out_host) {
  if (!ctx || !H || !out_host) return FIFA_ERR_INVALID_ARG;
  Plan* P = H->plan;
  if (level < 0 || level >= P->L || row0 < 0 || nrows < 1 || row0 + nrows > P->n) return FIFA_ERR_INVALID_ARG;
  const int cap = H->host.cap;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy2D(out_host, sizeof(double) * (size_t)nrows, H->host.bases + ((size_t)level * cap) * P->n + row0,
                  sizeof(double) * (size_t)P->n, sizeof(double) * (size_t)nrows, (size_t)cap, cudaMemcpyDeviceToHost));
  return FIFA_OK;
}

extern "C" fifa_status fifa_hmat_export(fifa_ctx* ctx, const fifa_hmat* H, int* ranks_host, int* row_piv_host,
                                        int* col_piv_host, double* bases_host, double* leaves_host) {
  if (!ctx || !H) return FIFA_ERR_INVALID_ARG;
  Plan* P = H->plan;
  const int cap = H->host.cap;
  cudaStream_t s = ctx->stream;
  CK(cudaStreamSynchronize(s));
  if (ranks_host && P->nnodes) CK(cudaMemcpy(ranks_host, H->host.rank, sizeof(int) * P->nnodes, cudaMemcpyDeviceToHost));
  if (row_piv_host && P->nnodes)
    CK(cudaMemcpy(row_piv_host, H->host.row_piv, sizeof(int) * P->nnodes * cap, cudaMemcpyDeviceToHost));
  if (col_piv_host && P->nnodes)
    CK(cudaMemcpy(col_piv_host, H->host.col_piv, sizeof(int) * P->nnodes * cap, cudaMemcpyDeviceToHost));
  if (bases_host && P->L)
    CK(cudaMemcpy(bases_host, H->host.bases, sizeof(double) * (size_t)P->L * cap * P->n, cudaMemcpyDeviceToHost));
  if (leaves_host)
    CK(cudaMemcpy(leaves_host, H->host.leaves, sizeof(double) * (size_t)P->nleaf * P->Bm * P->Bm, cudaMemcpyDeviceToHost));
  int hs = 0;
  CK(cudaMemcpy(&hs, H->host.status, sizeof(int), cudaMemcpyDeviceToHost));
  return dev_status_to_api(hs);
}

extern "C" fifa_status fifa_fact_export(fifa_ctx* ctx, const fifa_fact* F, double* bases_host, double* leaves_host,
                                        double* Zf_host, double* Zi_host) {
  if (!ctx || !F) return FIFA_ERR_INVALID_ARG;
  Plan* P = F->plan;
  const int cap = F->host.cap;
  CK(cudaStreamSynchronize(ctx->stream));
  const size_t nb = (size_t)P->L * cap * P->n, nl = (size_t)P->nleaf * P->Bm * P->Bm;
  auto fetch = [&](double* dst, const void* src, size_t cnt) -> cudaError_t {
    if (!dst || cnt == 0) return cudaSuccess;
    if (F->host.prec == 0) return cudaMemcpy(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost);
    std::vector<float> tmp(cnt);
    cudaError_t e = cudaMemcpy(tmp.data(), src, sizeof(float) * cnt, cudaMemcpyDeviceToHost);
    for (size_t i = 0; i < cnt; ++i) dst[i] = tmp[i];
    return e;
  };
  CK(fetch(bases_host, F->host.Q, nb));
  CK(fetch(leaves_host, F->host.Lleaf, nl));
  if (leaves_host)  // the device copy mirrors L^T into the upper triangle; export L alone
    for (size_t lf = 0; lf < (size_t)P->nleaf; ++lf)
      for (int k = 1; k < P->Bm; ++k)
        for (int j = 0; j < k; ++j) leaves_host[(lf * P->Bm + k) * P->Bm + j] = 0.0;
  const size_t nz = (size_t)std::max(1, P->nnodes) * 4 * cap * cap;
  if (Zf_host && P->nnodes) CK(cudaMemcpy(Zf_host, F->host.Zf, sizeof(double) * nz, cudaMemcpyDeviceToHost));
  if (Zi_host && P->nnodes) CK(cudaMemcpy(Zi_host, F->host.Zi, sizeof(double) * nz, cudaMemcpyDeviceToHost));
  int hs = 0;
  CK(cudaMemcpy(&hs, F->host.status, sizeof(int), cudaMemcpyDeviceToHost));
  return dev_status_to_api(hs);
}

extern "C" fifa_status fifa_det_exp(fifa_ctx* ctx, const double* in_dev, double* out_dev, int64_t n) {
  if (!ctx || !in_dev || !out_dev || n < 0) return FIFA_ERR_INVALID_ARG;
  if (n == 0) return FIFA_OK;
  CK(launch_det_exp(in_dev, out_dev, n, ctx->stream));
  return FIFA_OK;
}

extern "C" fifa_status fifa_normals(fifa_ctx* ctx, uint64_t seed, uint32_t tag, uint64_t iter, uint64_t stream_id,
                                    double* out_dev, int64_t n) {
  if (!ctx || !out_dev || n < 0) return FIFA_ERR_INVALID_ARG;
  if (n == 0) return FIFA_OK;
  CK(launch_normals(seed, tag, nullptr, iter, stream_id, out_dev, n, ctx->stream));
  return FIFA_OK;
}

extern "C" fifa_status fifa_philox(fifa_ctx* ctx, uint64_t seed, const uint32_t* ctr_dev, uint32_t* out_dev,
                                   int64_t count) {
  if (!ctx || !ctr_dev || !out_dev || count < 0) return FIFA_ERR_INVALID_ARG;
  if (count == 0) return FIFA_OK;
  CK(launch_philox(seed, ctr_dev, out_dev, count, ctx->stream));
  return FIFA_OK;
}

extern "C" fifa_status fifa_probe_fp64_fma(fifa_ctx* ctx, int iters, double* tflops_host, double* ms_host) {
  if (!ctx || iters < 1 || !tflops_host) return FIFA_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  const int blocks = ctx->num_sms * 8;  // 8 CTAs of 256 threads per SM: 64 warps, full occupancy
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return FIFA_ERR_CUDA;
  }
  fifa_status st = FIFA_OK;
  float ms = 0.0f;
  cudaError_t e = launch_dfma_probe((double*)ctx->flags, 1000, blocks, s);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = launch_dfma_probe((double*)ctx->flags, iters, blocks, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e != cudaSuccess) {
    ctx->last_cuda = e;
    st = FIFA_ERR_CUDA;
  } else {
    const double flops = 2.0 * 8.0 * (double)iters * 256.0 * (double)blocks;
    *tflops_host = flops / ((double)ms * 1e-3) / 1e12;
    if (ms_host) *ms_host = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

extern "C" const char* fifa_last_cuda_error(const fifa_ctx* ctx) {
  return ctx ? cudaGetErrorString(ctx->last_cuda) : "no context";
}

extern "C" const char* fifa_status_str(fifa_status s) {
  switch (s) {
    case FIFA_OK: return "ok";
    case FIFA_ERR_INVALID_ARG: return "invalid argument";
    case FIFA_ERR_UNSORTED: return "inputs are not sorted";
    case FIFA_ERR_NOT_SPD: return "matrix is not positive definite";
    case FIFA_ERR_RANK_CAP: return "ACA rank cap reached before the tolerance";
    case FIFA_ERR_OOM: return "device arena exhausted";
    case FIFA_ERR_CUDA: return "CUDA runtime error";
    case FIFA_ERR_TIMEOUT: return "bounded device wait timed out";
    case FIFA_ERR_UNSUPPORTED: return "unsupported size";
  }
  return "unknown status";
}
