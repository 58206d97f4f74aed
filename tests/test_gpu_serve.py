"""Serving (fifa_server_*) and the chain footprint (fifa_chain_bytes) on the GPU.

* fifa_chain_bytes is exact: a context whose arena has exactly that many
  bytes creates and runs the chain, one 256-byte granule less does not.
* A request's posterior mean and draws match the oracle's Gibbs chain (mean
  to 1e-8 as for the single chain, draws to 100 x max(1e-10, 8 kappa u)).
* Continuous batching: every request's result is bit-for-bit the same alone
  (one slot, nothing else submitted) and in a mix of concurrent requests of
  different sizes and kernels, and the mix really ran requests concurrently.
* Admission never lets the requests in flight exceed the HBM budget.
"""
import math
import time

import numpy as np
import pytest

from oracle import hodlr, sampler
from paper_2006_06537_gb300.inputs import request_data, uniform_sine
from tests.gpu_util import build_lib, dev, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402

B, EPS, CAP = 64, 1e-12, 32


def _opts(prec=fifa.FIFA_FP64, leaf=B, eps=EPS, overlap=0):
    return fifa.fifa_opts(leaf, eps, CAP, prec, 1e-12, 3, 1, 0, 0, overlap)


def _prior(mu=math.log(0.1)):
    return fifa.fifa_prior(1.0, 1.0, 1.0, 1.0, mu, 1.0, 0.2)


@pytest.mark.parametrize("indep", [1, 0])
@pytest.mark.parametrize("n", [3000, 40000])
def test_chain_bytes_is_exact(n, indep):
    x, y = uniform_sine(n, 2)
    o = fifa.fifa_opts(B, 1e-10, CAP, fifa.FIFA_FP64, 1e-12, 3, indep)
    need = fifa.fifa_chain_bytes(o, n)
    vy = float(np.var(y))
    hy = fifa.fifa_hyper(0, vy, 0.1, 0.5 * vy, 1e-6)
    for size, ok in ((need, True), (need - 256, False)):
        if size < (1 << 20):
            continue
        ctx = fifa.Context(leaf_size=B, aca_tol=1e-10, rank_cap=CAP, arena_bytes=size, independent_ctas=indep)
        xd, yd = dev(x, torch), dev(y, torch)
        if ok:
            ch = fifa.fifa_chain_create(ctx.h, xd, yd, n, hy, _prior(), 0, 0)
            fifa.fifa_gibbs_step(ctx.h, ch, 2)
            fifa.fifa_destroy_chain(ctx.h, ch)
        else:
            with pytest.raises(fifa.FifaError) as e:
                fifa.fifa_chain_create(ctx.h, xd, yd, n, hy, _prior(), 0, 0)
            assert e.value.code == fifa.FIFA_ERR_OOM
        ctx.close()


def _run(server, reqs):
    ids = [fifa.fifa_server_submit(server, *r[:2], r[2], r[3], r[4], r[5], r[6], r[7], r[8]) for r in reqs]
    out = []
    for r, rid in zip(reqs, ids):
        n, nd = len(r[0]), r[8]
        mean = np.empty(n)
        draws = np.empty((nd, n))
        st, res = fifa.fifa_server_wait(server, rid, mean, draws)
        out.append((mean, draws, res))
    return out


def test_server_request_matches_oracle():
    n, iters, burn, nd = 2048, 6, 2, 2
    x, y = uniform_sine(n, 0)
    vy = float(np.var(y))
    srv = fifa.fifa_server_create(_opts(), 1 << 30, 2)
    # non-blocking poll until the request is done, then collect it
    rid = fifa.fifa_server_submit(srv, x, y, fifa.fifa_hyper(0, vy, 0.1, 0.5 * vy, 1e-6), _prior(), 0, 0, iters, burn,
                                  nd)
    deadline = time.monotonic() + 600
    while not fifa.fifa_server_poll(srv, rid):
        assert time.monotonic() < deadline
        time.sleep(0.01)
    mean, draws = np.empty(n), np.empty((nd, n))
    st, res = fifa.fifa_server_wait(srv, rid, mean, draws)
    with pytest.raises(fifa.FifaError) as e:  # collected: the id is gone
        fifa.fifa_server_poll(srv, rid)
    assert e.value.code == fifa.FIFA_ERR_INVALID_ARG
    fifa.fifa_server_destroy(srv)
    assert res.status == fifa.FIFA_OK
    assert res.t_submit <= res.t_start <= res.t_done
    opts = sampler.Opts(B=B, eps=EPS, cap=CAP, kind=0, nugget=1e-6)
    st = sampler.init_state(x, y, 0.1, opts)
    kappa = np.linalg.cond(hodlr.dense(st.HC))
    tol = max(1e-10, 8 * kappa * 1.1e-16)
    pr = sampler.Prior(logrho_mu=math.log(0.1))
    acc = np.zeros(n)
    want = []
    for t in range(iters):
        sampler.gibbs_step(st, x, y, pr, opts, seed=0, chain=0)
        if t >= burn:
            acc += st.mean
        if t in (burn + (iters - burn) // 2 - 1, iters - 1):
            want.append(st.f.copy())
    assert rel(mean, acc / (iters - burn)) <= 1e-8
    for j in range(nd):
        assert rel(draws[j], want[j]) <= 100 * tol
    assert res.last.rho == pytest.approx(math.exp(st.eta), rel=1e-12)


def _mix(count=10, seed=11):
    g = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(2 ** g.uniform(10, 16))
        kind = int(g.integers(0, 2))
        x, y = request_data(dict(id=100 + i, n=n, kind=kind))
        vy = float(np.var(y))
        hy = fifa.fifa_hyper(kind, vy, 0.1, 0.5 * vy, 1e-6)
        reqs.append((x, y, hy, _prior(), 5, i, 12, 4, 3))
    return reqs


WIDE = 1 << 14  # requests with n >= WIDE run on the wide worker (CTA groups, fused sweeps)


@pytest.mark.parametrize("wide_workers,overlap", [(1, 0), (2, 0), (2, 1)])
def test_server_result_same_alone_and_in_mix(wide_workers, overlap):
    # with two wide workers, two requests' grouped launches (each sized to half
    # the GPU) run side by side; a request's result must not depend on it.
    # overlap: every request's proposal runs on a branch stream beside its draw
    # (fifa_opts.overlap_proposal), which must not change a bit either
    reqs = _mix()
    assert sum(len(r[0]) >= WIDE for r in reqs) >= 2 and any(len(r[0]) < WIDE for r in reqs)
    srv = fifa.fifa_server_create(_opts(eps=1e-10, overlap=overlap), 8 << 30, 6, WIDE, wide_workers)
    mixed = _run(srv, reqs)
    stats = fifa.fifa_server_stats(srv)
    fifa.fifa_server_destroy(srv)
    assert stats.completed == len(reqs)
    assert all(m[2].status == fifa.FIFA_OK for m in mixed)
    assert stats.peak_in_flight > 1  # requests really overlapped
    for k in (0, len(reqs) // 2, int(np.argmax([len(r[0]) for r in reqs]))):
        srv = fifa.fifa_server_create(_opts(eps=1e-10, overlap=0), 8 << 30, 1 + wide_workers, WIDE, wide_workers)
        (mean, draws, res), = _run(srv, [reqs[k]])
        fifa.fifa_server_destroy(srv)
        assert res.status == fifa.FIFA_OK and mixed[k][2].status == fifa.FIFA_OK
        assert np.array_equal(mean, mixed[k][0]), k
        assert np.array_equal(draws, mixed[k][1]), k
        assert res.last.rho == mixed[k][2].last.rho


def test_server_admission_respects_budget():
    reqs = _mix(count=8, seed=3)
    per = [fifa.fifa_chain_bytes(_opts(eps=1e-10), len(r[0])) for r in reqs]
    budget = max(3 * max(per), 64 << 20)
    srv = fifa.fifa_server_create(_opts(eps=1e-10), budget, 8)
    out = _run(srv, reqs)
    stats = fifa.fifa_server_stats(srv)
    assert all(o[2].status == fifa.FIFA_OK for o in out)
    assert stats.peak_bytes <= budget
    assert stats.bytes_in_use == 0 and stats.in_flight == 0 and stats.queued == 0
    # a request that can never fit is refused at submission
    big = np.linspace(0, 1, 1 << 20)
    with pytest.raises(fifa.FifaError) as e:
        fifa.fifa_server_submit(srv, big, np.sin(big), reqs[0][2], _prior(), 0, 0, 4, 1, 1)
    assert e.value.code == fifa.FIFA_ERR_OOM
    # unsorted inputs are refused at submission
    x, y = reqs[0][0].copy(), reqs[0][1]
    x[[3, 4]] = x[[4, 3]]
    with pytest.raises(fifa.FifaError) as e:
        fifa.fifa_server_submit(srv, x, y, reqs[0][2], _prior(), 0, 0, 4, 1, 1)
    assert e.value.code == fifa.FIFA_ERR_UNSORTED
    fifa.fifa_server_destroy(srv)
