// Serving: independent 1-D GP regression requests run as Gibbs chains with
// continuous batching on one GPU.
//
// The server owns one device pool (the HBM budget) and `slots` workers, each a
// host thread with its own non-blocking CUDA stream and library context.  A
// request is admitted as soon as a worker that may run it is idle and the pool
// can hold its chain (the exact arena footprint from the plan, plus its result
// buffers); among the requests a worker may run, the oldest goes first.
// Admitted requests run concurrently, their kernels overlapping on the GPU.
//
// Narrow workers use independent CTAs (no CTA groups that wait on each other).
// With wide_min_n > 0, the first wide_workers workers are wide: they run
// exactly the requests with n >= wide_min_n, with CTA groups and fused
// cooperative sweeps, each launch sized to 1 / wide_workers of the CTAs the GPU
// holds at once.  Only the wide streams hold kernels whose CTAs wait on each
// other, at most one such launch each, and together they fit on the GPU; every
// other kernel's CTAs finish without waiting, so the waiting launches always
// become co-resident.  Which worker type runs a request depends only on its n,
// and every wide worker uses the same sizes, so its arithmetic, and its
// result, is the same alone and in any mix.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/fifa.h"
#include "fifa_api_internal.h"
#include "fifa_chain.h"
#include "fifa_chain_impl.h"

namespace {

struct Req {
  uint64_t id = 0;
  std::vector<double> x, y;
  fifa_request r{};
  bool wide = false;
  size_t bytes = 0;
  char* mem = nullptr;
  std::vector<double> mean, draws;
  fifa_result res{};
  bool done = false;
};

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

struct fifa_server {
  fifa_server_opts o{};
  int device = 0;
  char* pool = nullptr;
  Arena arena;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::map<uint64_t, Req*> reqs;
  std::vector<std::thread> workers;
  bool stop = false;
  uint64_t next_id = 1;
  int in_flight = 0, peak_in_flight = 0;
  size_t peak_bytes = 0;
  uint64_t iterations_done = 0, completed = 0;
  std::chrono::steady_clock::time_point t0;
};

// Device bytes of one request: the chain's arena (fifa_chain_bytes), the
// device copies of x and y, the mean accumulator and the draws.
static fifa_status request_bytes(const fifa_opts& o, const fifa_request& r, size_t* out) {
  size_t chain = 0;
  fifa_status st = fifa_chain_bytes(&o, r.n, &chain);
  if (st != FIFA_OK) return st;
  const size_t vec = round256(sizeof(double) * (size_t)r.n);
  *out = std::max<size_t>(chain + 3 * vec + round256(sizeof(double) * (size_t)r.n * r.ndraws), 1 << 20);
  return FIFA_OK;
}

static fifa_status run_request(fifa_server* S, fifa_ctx** pctx, cudaStream_t stream, Req* q) {
  fifa_opts o = S->o.opts;
  o.independent_ctas = q->wide ? 0 : 1;
  o.coresident_share = q->wide ? S->o.wide_workers : 0;  // the wide workers' launches fit side by side
  fifa_status st;
  if (!*pctx) {
    st = fifa_create(pctx, &o, stream, q->mem, q->bytes);
    if (st != FIFA_OK) return st;
  } else {
    st = ctx_rebind_arena(*pctx, q->mem, q->bytes);
    if (st != FIFA_OK) return st;
  }
  fifa_ctx* ctx = *pctx;
  const int64_t n = q->r.n;
  double* xd = (double*)ctx->arena.alloc(sizeof(double) * n);
  double* yd = (double*)ctx->arena.alloc(sizeof(double) * n);
  double* macc = (double*)ctx->arena.alloc(sizeof(double) * n);
  double* draws = q->r.ndraws ? (double*)ctx->arena.alloc(sizeof(double) * n * q->r.ndraws) : nullptr;
  if (!xd || !yd || !macc || (q->r.ndraws && !draws)) return FIFA_ERR_OOM;
  if (cudaMemcpyAsync(xd, q->x.data(), sizeof(double) * n, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemcpyAsync(yd, q->y.data(), sizeof(double) * n, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return FIFA_ERR_CUDA;
  fifa_chain* ch = nullptr;
  st = fifa_chain_create(ctx, xd, yd, n, &q->r.init, &q->r.prior, q->r.seed, q->r.chain_id, &ch);
  if (st != FIFA_OK) return st;
  st = chain_run_collect(ctx, ch, q->r.iters, q->r.burn, q->r.ndraws, macc, draws);
  ChainDev c;
  memset(&c, 0, sizeof(c));
  if (st == FIFA_OK) st = chain_state(ctx, ch, &c);
  if (st == FIFA_OK) {
    q->mean.resize(n);
    q->draws.resize((size_t)n * q->r.ndraws);
    if (cudaMemcpyAsync(q->mean.data(), macc, sizeof(double) * n, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        (q->r.ndraws && cudaMemcpyAsync(q->draws.data(), draws, sizeof(double) * n * q->r.ndraws,
                                        cudaMemcpyDeviceToHost, stream) != cudaSuccess) ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      st = FIFA_ERR_CUDA;
    const double kept = (double)(q->r.iters - q->r.burn);
    for (auto& v : q->mean) v /= kept;
    q->res.last.kernel = c.kind;
    q->res.last.tau2 = c.tau2;
    q->res.last.rho = c.rho;
    q->res.last.sigma2 = c.sigma2;
    q->res.last.nugget = q->r.init.nugget;
    q->res.accept_rate = (double)c.n_accept / (double)q->r.iters;
  }
  fifa_destroy_chain(ctx, ch);
  return st;
}

static void worker_main(fifa_server* S, bool wide) {
  cudaSetDevice(S->device);
  cudaStream_t stream = nullptr;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) stream = nullptr;
  fifa_ctx* ctx = nullptr;
  for (;;) {
    Req* q = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) break;
        // the oldest queued request this worker may run
        auto it = S->queue.begin();
        while (it != S->queue.end() && (*it)->wide != wide) ++it;
        if (it != S->queue.end()) {
          Req* h = *it;
          h->mem = (char*)S->arena.alloc(h->bytes);
          if (h->mem) {
            q = h;
            S->queue.erase(it);
            break;
          }
          if (S->in_flight == 0) {  // the pool is empty and still too small: cannot ever run
            S->queue.erase(it);
            h->res.status = FIFA_ERR_OOM;
            h->res.t_start = h->res.t_done = now_s(S->t0);
            h->done = true;
            S->cv_done.notify_all();
            continue;
          }
        }
        S->cv_work.wait(lk);
      }
      if (!q) break;
      ++S->in_flight;
      S->peak_in_flight = std::max(S->peak_in_flight, S->in_flight);
      S->peak_bytes = std::max(S->peak_bytes, S->arena.in_use);
      q->res.t_start = now_s(S->t0);
    }
    fifa_status st = stream ? run_request(S, &ctx, stream, q) : FIFA_ERR_CUDA;
    if (ctx) cudaStreamSynchronize(stream);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->arena.release(q->mem);
      q->mem = nullptr;
      q->res.status = st;
      q->res.t_done = now_s(S->t0);
      q->done = true;
      --S->in_flight;
      ++S->completed;
      if (st == FIFA_OK) S->iterations_done += (uint64_t)q->r.iters;
      S->cv_done.notify_all();
      S->cv_work.notify_all();  // memory came back: the head of the queue may fit now
    }
  }
  if (ctx) fifa_destroy_ctx(ctx);
  if (stream) cudaStreamDestroy(stream);
}

extern "C" fifa_status fifa_server_create(const fifa_server_opts* o, fifa_server** out) {
  if (!o || !out || o->slots < 1 || o->slots > 256 || o->hbm_budget < (16u << 20) || o->wide_min_n < 0 ||
      (o->wide_min_n > 0 && o->slots < 2) || o->wide_workers < 0 ||
      (o->wide_min_n > 0 && std::max(1, o->wide_workers) >= o->slots) || o->wide_workers > 64)
    return FIFA_ERR_INVALID_ARG;
  *out = nullptr;
  fifa_opts fo = o->opts;
  fo.independent_ctas = 1;  // per request: 0 for the wide workers' requests
  fo.coresident_share = 0;
  size_t probe = 0;
  fifa_status st = fifa_chain_bytes(&fo, 1024, &probe);  // validates the options
  if (st != FIFA_OK) return st;
  fifa_server* S = new (std::nothrow) fifa_server();
  if (!S) return FIFA_ERR_OOM;
  S->o = *o;
  S->o.opts = fo;
  S->o.wide_workers = o->wide_min_n > 0 ? std::max(1, o->wide_workers) : 0;
  S->t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&S->device);
  void* p = nullptr;
  if (cudaMalloc(&p, o->hbm_budget) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return FIFA_ERR_OOM;
  }
  S->pool = (char*)p;
  S->arena.base = S->pool;
  S->arena.size = o->hbm_budget & ~(size_t)255;
  S->arena.free_[0] = S->arena.size;
  for (int k = 0; k < o->slots; ++k) S->workers.emplace_back(worker_main, S, k < S->o.wide_workers);
  *out = S;
  return FIFA_OK;
}

extern "C" fifa_status fifa_server_submit(fifa_server* S, const fifa_request* r, uint64_t* id_out) {
  if (!S || !r || !id_out || !r->x_host || !r->y_host || r->n < 2 || r->iters < 1 || r->burn < 0 ||
      r->burn >= r->iters || r->ndraws < 0 || r->ndraws > r->iters - r->burn)
    return FIFA_ERR_INVALID_ARG;
  for (int64_t i = 0; i < r->n; ++i) {
    if (!isfinite(r->x_host[i]) || !isfinite(r->y_host[i])) return FIFA_ERR_INVALID_ARG;
    if (i > 0 && r->x_host[i] < r->x_host[i - 1]) return FIFA_ERR_UNSORTED;
  }
  Req* q = new (std::nothrow) Req();
  if (!q) return FIFA_ERR_OOM;
  q->r = *r;
  q->wide = S->o.wide_min_n > 0 && r->n >= S->o.wide_min_n;
  fifa_opts ro = S->o.opts;
  ro.independent_ctas = q->wide ? 0 : 1;
  ro.coresident_share = q->wide ? S->o.wide_workers : 0;
  fifa_status st = request_bytes(ro, *r, &q->bytes);
  if (st != FIFA_OK || q->bytes > S->arena.size) {
    delete q;
    return st != FIFA_OK ? st : FIFA_ERR_OOM;
  }
  q->x.assign(r->x_host, r->x_host + r->n);
  q->y.assign(r->y_host, r->y_host + r->n);
  q->r.x_host = nullptr;
  q->r.y_host = nullptr;
  std::lock_guard<std::mutex> lk(S->mu);
  q->id = S->next_id++;
  q->res.t_submit = now_s(S->t0);
  q->res.bytes = q->bytes;
  S->reqs[q->id] = q;
  S->queue.push_back(q);
  S->cv_work.notify_all();  // only some workers may run it (wide / narrow): wake them all
  *id_out = q->id;
  return FIFA_OK;
}

extern "C" fifa_status fifa_server_wait(fifa_server* S, uint64_t id, double* mean_host, double* draws_host,
                                        fifa_result* res) {
  if (!S) return FIFA_ERR_INVALID_ARG;
  Req* q = nullptr;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return FIFA_ERR_INVALID_ARG;
    q = it->second;
    S->cv_done.wait(lk, [&] { return q->done; });
    S->reqs.erase(it);
  }
  if (res) *res = q->res;
  if (q->res.status == FIFA_OK) {
    if (mean_host) memcpy(mean_host, q->mean.data(), sizeof(double) * q->mean.size());
    if (draws_host && !q->draws.empty()) memcpy(draws_host, q->draws.data(), sizeof(double) * q->draws.size());
  }
  const fifa_status st = (fifa_status)q->res.status;
  delete q;
  return st;
}

extern "C" fifa_status fifa_server_poll(fifa_server* S, uint64_t id, int* done_out) {
  if (!S || !done_out) return FIFA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return FIFA_ERR_INVALID_ARG;
  *done_out = it->second->done ? 1 : 0;
  return FIFA_OK;
}

extern "C" fifa_status fifa_server_stats(fifa_server* S, fifa_server_counters* out) {
  if (!S || !out) return FIFA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  out->now = now_s(S->t0);
  out->queued = (int)S->queue.size();
  out->in_flight = S->in_flight;
  out->peak_in_flight = S->peak_in_flight;
  out->bytes_in_use = S->arena.in_use;
  out->peak_bytes = S->peak_bytes;
  out->completed = S->completed;
  out->iterations_done = S->iterations_done;
  return FIFA_OK;
}

extern "C" void fifa_server_destroy(fifa_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
  }
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->reqs) delete kv.second;
  if (S->pool) cudaFree(S->pool);
  delete S;
}
