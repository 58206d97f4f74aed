"""Gibbs chain on the GPU (fifa_chain_create / fifa_gibbs_step) against the
oracle's Gibbs iteration from the same state, seed and Philox streams.

Tolerances: the posterior mean (no factor of C~ involved) 1e-10; quantities
that pass through W_C (the draw f, ||y - f||^2, q = f^T C~^-1 f, hence sigma2,
tau2, log alpha) max(1e-10, 8 kappa(C~) u), kappa from the oracle's dense
C~.  Accept / reject decisions must agree unless |log u - log alpha| is
inside that tolerance.
"""
import math

import numpy as np
import pytest

from oracle import hodlr, rng, sampler
from paper_2006_06537_gb300.inputs import uniform_sine
from tests.gpu_util import build_lib, dev, host, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402

N, B, EPS, RHO0 = 2048, 64, 1e-12, 0.1


def _prior():
    return sampler.Prior(a_tau2=1.0, b_tau2=1.0, a_sigma2=1.0, b_sigma2=1.0, logrho_mu=math.log(0.1), logrho_sd=1.0,
                         prop_sd=0.2)


def _gpu_chain(x, y, nugget, prec=fifa.FIFA_FP64, sigma2=None, tau2=None, refine_max=8, prior=None):
    # a stream of its own, so the iteration runs as a captured graph (the
    # legacy default stream cannot be captured)
    ctx = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=32, prec=prec, refine_max=refine_max, refine_tol=1e-13,
                       arena_bytes=1 << 30, stream=torch.cuda.Stream())
    vy = float(np.var(y))
    s2 = 0.5 * vy if sigma2 is None else sigma2
    t2 = vy if tau2 is None else tau2
    p = _prior() if prior is None else prior
    pr = fifa.fifa_prior(p.a_tau2, p.b_tau2, p.a_sigma2, p.b_sigma2, p.logrho_mu, p.logrho_sd, p.prop_sd)
    xd, yd = dev(x, torch), dev(y, torch)
    torch.cuda.synchronize()
    ch = fifa.fifa_chain_create(ctx.h, xd, yd, len(x), fifa.fifa_hyper(0, t2, RHO0, s2, nugget), pr, 0, 0)
    return ctx, ch


def _oracle_chain(x, y, nugget, iters):
    opts = sampler.Opts(B=B, eps=EPS, cap=32, kind=0, nugget=nugget)
    st = sampler.init_state(x, y, RHO0, opts)
    for _ in range(iters):
        sampler.gibbs_step(st, x, y, _prior(), opts, seed=0, chain=0)
    return st


@pytest.mark.parametrize("nugget", [1e-6, 1e-8])
def test_chain_matches_oracle(nugget):
    x, y = uniform_sine(N, 0)
    iters = 6
    ctx, ch = _gpu_chain(x, y, nugget)
    tr = np.zeros((iters, fifa.FIFA_TRACE_FIELDS))
    fifa.fifa_gibbs_step(ctx.h, ch, iters, tr)
    f = torch.empty(N, dtype=torch.float64, device="cuda")
    mean = torch.empty_like(f)
    hyp = fifa.fifa_chain_get(ctx.h, ch, f, mean)
    st = _oracle_chain(x, y, nugget, iters)
    kappa = np.linalg.cond(hodlr.dense(st.HC))
    tol = max(1e-10, 8 * kappa * 1.1e-16)
    for t, o in zip(tr, st.trace):
        assert int(t[0]) == o["it"]
        assert abs(t[1] - o["sigma2"]) <= 10 * tol * o["sigma2"]
        assert abs(t[2] - o["tau2"]) <= 10 * tol * o["tau2"]
        assert abs(t[8] - o["rss"]) <= 10 * tol * o["rss"]
        assert abs(t[7] - o["q"]) <= 10 * tol * o["q"]
        # log alpha is a difference of two log-determinants and two quadratic forms of
        # ill-conditioned matrices: absolute error ~ tol * (|logdet| + q / tau2)
        la_tol = 8 * tol * (abs(t[6]) + abs(t[7]) / t[2]) + 1e-9
        assert abs(t[5] - o["log_alpha"]) <= la_tol, (t[5], o["log_alpha"], la_tol)
        lu = math.log(rng.scalar_uniform(0, 0, rng.TAG_MH_UNIF, o["it"], 0))
        if (t[5] - lu) * (o["log_alpha"] - lu) > 0:  # both sides on the same side of log u
            assert bool(t[4]) == o["accept"]
    assert hyp.rho == pytest.approx(math.exp(st.eta), rel=1e-12)
    assert rel(host(mean), st.mean) <= 1e-8
    assert rel(host(f), st.f) <= 100 * tol
    assert fifa.fifa_chain_kernel_nodes(ch) > 0  # the graph path ran


def test_mixed_chain_refines_to_fp64_tolerance():
    x, y = uniform_sine(N, 0)
    iters = 4
    ctx, ch = _gpu_chain(x, y, 1e-6, prec=fifa.FIFA_MIXED)
    tr = np.zeros((iters, fifa.FIFA_TRACE_FIELDS))
    fifa.fifa_gibbs_step(ctx.h, ch, iters, tr)
    mean = torch.empty(N, dtype=torch.float64, device="cuda")
    fifa.fifa_chain_get(ctx.h, ch, None, mean)
    st = _oracle_chain(x, y, 1e-6, iters)
    assert np.all(tr[:, 9] <= 1e-10), tr[:, 9]  # true relative residual of the M~ solves
    assert tr[0, 11] == 1.0                     # the first iteration factors M~
    assert np.all(tr[:, 12] <= 8)
    for t, o in zip(tr, st.trace):
        assert abs(t[1] - o["sigma2"]) <= 1e-8 * o["sigma2"]
        assert bool(t[4]) == o["accept"]
        if o["accept"] and t[0] + 1 < iters:    # a new length-scale: M~ is refactored next
            assert tr[int(t[0]) + 1, 11] == 1.0
    assert rel(host(mean), st.mean) <= 1e-8


def test_mixed_chain_reuses_its_factor_and_tracks_the_fp64_chain():
    # fixed length-scale (a zero-step proposal is accepted without changing C~)
    # and variances started near the posterior: s = tau2 / sigma2 moves by well
    # under 5% per iteration, so the kept FP64 factor of M~ preconditions the
    # later iterations' solves; the chain must still follow the FP64 chain
    x, y = uniform_sine(N, 0)
    iters = 8
    p = _prior()
    p.prop_sd = 0.0
    cm, chm = _gpu_chain(x, y, 1e-6, prec=fifa.FIFA_MIXED, sigma2=0.01, tau2=0.5, prior=p)
    c6, ch6 = _gpu_chain(x, y, 1e-6, sigma2=0.01, tau2=0.5, prior=p)
    tm = np.zeros((iters, fifa.FIFA_TRACE_FIELDS))
    t6 = np.zeros((iters, fifa.FIFA_TRACE_FIELDS))
    fifa.fifa_gibbs_step(cm.h, chm, iters, tm)
    fifa.fifa_gibbs_step(c6.h, ch6, iters, t6)
    assert tm[0, 11] == 1.0 and np.any(tm[1:, 11] == 0.0), tm[:, 11]
    assert np.all(t6[:, 11] == 1.0) and np.all(t6[:, 12] == 0.0)  # FP64: refactored every iteration
    kept = tm[:, 11] == 0.0
    assert np.all(tm[kept, 12] >= 1) and np.all(tm[:, 12] <= 8)
    assert np.all(tm[:, 9] <= 1e-10), tm[:, 9]
    for a, b in zip(tm, t6):
        assert abs(a[1] - b[1]) <= 1e-9 * b[1] and abs(a[2] - b[2]) <= 1e-9 * b[2]
        assert abs(a[8] - b[8]) <= 1e-9 * b[8]
    f_m, f_6 = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(2))
    m_m, m_6 = torch.empty_like(f_m), torch.empty_like(f_m)
    fifa.fifa_chain_get(cm.h, chm, f_m, m_m)
    fifa.fifa_chain_get(c6.h, ch6, f_6, m_6)
    assert rel(host(f_m), host(f_6)) <= 1e-8
    assert rel(host(m_m), host(m_6)) <= 1e-9


def test_graph_replay_is_deterministic_and_chunking_invariant():
    x, y = uniform_sine(512, 1)
    a_ctx, a = _gpu_chain(x, y, 1e-6)
    b_ctx, b = _gpu_chain(x, y, 1e-6)
    ta = np.zeros((8, fifa.FIFA_TRACE_FIELDS))
    fifa.fifa_gibbs_step(a_ctx.h, a, 8, ta)
    tb = np.zeros((8, fifa.FIFA_TRACE_FIELDS))
    for k in range(8):
        fifa.fifa_gibbs_step(b_ctx.h, b, 1, tb[k:k + 1])
    assert np.array_equal(ta, tb)
