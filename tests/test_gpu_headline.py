"""Gibbs iterations of the clustered headline recipe against the oracle.

The recipe the benchmark times at n = 2^20 (8 narrow clusters, y = sin 2 pi x +
N(0, 0.05^2), squared exponential, rho0 = 0.01, leaf 32, ACA tolerance 1e-10,
rank cap 32, nugget 1e-6), here at n = 2^17 so the oracle's iterations take
seconds.  Three iterations of the FP64 chain and of the mixed chain (kept FP64
factor of M~, FP32 preconditioner, FP64-residual conjugate gradients) are
compared with the oracle's iterations from the same state and Philox streams.

Tolerances: the posterior mean 1e-8 against the oracle; every quantity that
passes through a factor of C~ (the draw f, ||y - f||^2, q, sigma2, tau2, log
alpha) max(1e-10, 8 kappa u) with kappa estimated as lambda_max(C~) / nugget
(lambda_max by power iteration with the oracle's product; the nugget bounds
the small eigenvalues of C + nugget I, which the compression moves by far
less here).  Mixed against FP64 on the GPU: f within 1e-8 (the mixed path's
stated tolerance) and the mean within 1e-9.
"""
import math

import numpy as np
import pytest

from oracle import hodlr, rng, sampler
from paper_2006_06537_gb300.inputs import clustered
from tests.gpu_util import build_lib, dev, host, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402

N, B, EPS, CAP, RHO0, NUG, NOISE = 1 << 17, 32, 1e-10, 32, 0.01, 1e-6, 0.05
ITERS = 3


def _prior():
    return sampler.Prior(a_tau2=1.0, b_tau2=1.0, a_sigma2=1.0, b_sigma2=1.0, logrho_mu=math.log(RHO0), logrho_sd=1.0,
                         prop_sd=0.2)


@pytest.fixture(scope="module")
def oracle_run():
    x, y = clustered(N, 2, noise=NOISE)
    opts = sampler.Opts(B=B, eps=EPS, cap=CAP, kind=0, nugget=NUG)
    st = sampler.init_state(x, y, RHO0, opts)
    v = np.random.default_rng(0).standard_normal(N)
    lam = 0.0
    for _ in range(25):  # power iteration: lambda_max of C~(rho0)
        w = hodlr.matvec(st.HC, v)
        lam = float(np.linalg.norm(w))
        v = w / lam
    traces, fs, means = [], [], []
    for _ in range(ITERS):
        sampler.gibbs_step(st, x, y, _prior(), opts, seed=0, chain=0)
        fs.append(st.f.copy())
        means.append(st.mean.copy())
    return x, y, st.trace, fs, means, lam / NUG


def _gpu_run(x, y, prec):
    stream = torch.cuda.Stream()
    ctx = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=CAP, prec=prec, refine_max=8, refine_tol=1e-13,
                       arena_bytes=6 << 30, stream=stream)
    vy = float(np.var(y))
    p = _prior()
    pr = fifa.fifa_prior(p.a_tau2, p.b_tau2, p.a_sigma2, p.b_sigma2, p.logrho_mu, p.logrho_sd, p.prop_sd)
    xd, yd = dev(x, torch), dev(y, torch)
    torch.cuda.synchronize()
    ch = fifa.fifa_chain_create(ctx.h, xd, yd, N, fifa.fifa_hyper(0, vy, RHO0, 0.5 * vy, NUG), pr, 0, 0)
    trs, fs, means = [], [], []
    for _ in range(ITERS):
        tr = np.zeros((1, fifa.FIFA_TRACE_FIELDS))
        fifa.fifa_gibbs_step(ctx.h, ch, 1, tr)
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        m = torch.empty_like(f)
        fifa.fifa_chain_get(ctx.h, ch, f, m)
        trs.append(tr[0])
        fs.append(host(f))
        means.append(host(m))
    fifa.fifa_destroy_chain(ctx.h, ch)
    ctx.close()
    return np.array(trs), fs, means


def _check_against_oracle(tr, fs, means, o_trace, o_fs, o_means, kappa):
    tol = max(1e-10, 8 * kappa * 1.1e-16)
    for t, o in zip(tr, o_trace):
        assert int(t[0]) == o["it"]
        assert abs(t[1] - o["sigma2"]) <= 10 * tol * o["sigma2"], (t[1], o["sigma2"])
        assert abs(t[2] - o["tau2"]) <= 10 * tol * o["tau2"], (t[2], o["tau2"])
        assert abs(t[8] - o["rss"]) <= 10 * tol * o["rss"]
        assert abs(t[7] - o["q"]) <= 10 * tol * o["q"]
        la_tol = 8 * tol * (abs(t[6]) + abs(t[7]) / t[2]) + 1e-9
        if math.isfinite(o["log_alpha"]):
            assert abs(t[5] - o["log_alpha"]) <= la_tol, (t[5], o["log_alpha"], la_tol)
        lu = math.log(rng.scalar_uniform(0, 0, rng.TAG_MH_UNIF, o["it"], 0))
        if (t[5] - lu) * (o["log_alpha"] - lu) > 0:
            assert bool(t[4]) == o["accept"]
    for f, m, of, om in zip(fs, means, o_fs, o_means):
        assert rel(m, om) <= 1e-8
        assert rel(f, of) <= 100 * tol


def test_fp64_headline_recipe_iterations_match_oracle(oracle_run):
    x, y, o_trace, o_fs, o_means, kappa = oracle_run
    tr, fs, means = _gpu_run(x, y, fifa.FIFA_FP64)
    assert np.all(tr[:, 11] == 1.0)  # FP64: M~ factored every iteration
    _check_against_oracle(tr, fs, means, o_trace, o_fs, o_means, kappa)


def test_mixed_headline_recipe_iterations_match_oracle_and_fp64(oracle_run):
    x, y, o_trace, o_fs, o_means, kappa = oracle_run
    tm, fm, mm = _gpu_run(x, y, fifa.FIFA_MIXED)
    t6, f6, m6 = _gpu_run(x, y, fifa.FIFA_FP64)
    assert tm[0, 11] == 1.0
    assert np.all(tm[:, 9] <= 1e-8), tm[:, 9]  # true relative residual of the M~ solves
    _check_against_oracle(tm, fm, mm, o_trace, o_fs, o_means, kappa)
    for a, b, c, d in zip(fm, f6, mm, m6):
        assert rel(a, b) <= 1e-8
        assert rel(c, d) <= 1e-9
