"""Additive d-block model on the GPU (fifa_additive_create / fifa_additive_sweep)
against the oracle's block-Gibbs sweep from the same state, seed and Philox
streams (block k: stream id k, shared sigma2: stream id d).

Tolerances as for the single chain: quantities that pass through a factor W_C
of some block's C~ agree to max(1e-10, 8 kappa u), kappa the largest condition
number over the blocks' dense C~; the trace scalars to 10x that, the latent
components to 100x.
"""
import math

import numpy as np
import pytest

from oracle import hodlr, sampler
from paper_2006_06537_gb300.inputs import additive4
from tests.gpu_util import build_lib, dev, host, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402

B, EPS, RHO0, NUG = 64, 1e-12, 0.1, 1e-6


def _prior():
    return sampler.Prior(a_tau2=1.0, b_tau2=1.0, a_sigma2=1.0, b_sigma2=1.0, logrho_mu=math.log(0.1), logrho_sd=1.0,
                         prop_sd=0.2)


def _gpu_model(X, y, seed, indep=0):
    n, d = X.shape
    # a stream of its own: the sweep graph cannot be captured on the legacy default stream;
    # with independent CTAs the blocks' factorizations and hyper steps run as concurrent branches
    ctx = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=32, prec=fifa.FIFA_FP64, arena_bytes=1 << 30,
                       stream=torch.cuda.Stream(), independent_ctas=indep)
    vy = float(np.var(y))
    p = _prior()
    pr = fifa.fifa_prior(p.a_tau2, p.b_tau2, p.a_sigma2, p.b_sigma2, p.logrho_mu, p.logrho_sd, p.prop_sd)
    Xd, yd = dev(X.T, torch), dev(y, torch)
    torch.cuda.synchronize()
    m = fifa.fifa_additive_create(ctx.h, Xd, yd, n, d,
                                  fifa.fifa_hyper(0, vy / d, RHO0, 0.5 * vy, NUG), pr, seed)
    return ctx, m


@pytest.mark.parametrize("indep", [0, 1])
@pytest.mark.parametrize("n,d,sweeps", [(1024, 4, 3), (1500, 2, 4)])
def test_additive_matches_oracle(n, d, sweeps, indep):
    X, y = additive4(n, seed=5)
    X = np.ascontiguousarray(X[:, :d])
    seed = 7
    ctx, m = _gpu_model(X, y, seed, indep)
    tr = np.zeros((sweeps, fifa.fifa_additive_trace_fields(d)))
    fifa.fifa_additive_sweep(ctx.h, m, sweeps, tr)
    F = torch.empty((d, n), dtype=torch.float64, device="cuda")
    s2, hyp = fifa.fifa_additive_get(ctx.h, m, d, F)

    opts = sampler.Opts(B=B, eps=EPS, cap=32, kind=0, nugget=NUG)
    st = sampler.additive_init(X, y, RHO0, opts)
    kappa = max(np.linalg.cond(hodlr.dense(b["HC"])) for b in st.blocks)
    for _ in range(sweeps):
        sampler.additive_sweep(st, y, _prior(), opts, seed=seed)
    tol = max(1e-10, 8 * kappa * 1.1e-16)

    for t, o in zip(tr, st.trace):
        assert int(t[0]) == o["it"]
        assert int(t[3]) == 0
        assert t[4] == 0.0  # FP64 path: no refinement
        assert abs(t[1] - o["sigma2"]) <= 10 * tol * o["sigma2"]
        assert abs(t[2] - o["rss"]) <= 10 * tol * o["rss"]
        for k in range(d):
            assert abs(t[5 + k] - o["tau2"][k]) <= 10 * tol * o["tau2"][k]
            assert t[5 + d + k] == pytest.approx(o["rho"][k], rel=1e-12)
            assert bool(t[5 + 2 * d + k]) == o["accept"][k]
    assert s2 == pytest.approx(st.sigma2, rel=10 * tol)
    for k in range(d):
        assert hyp[k].rho == pytest.approx(math.exp(st.blocks[k]["eta"]), rel=1e-12)
        assert hyp[k].tau2 == pytest.approx(st.blocks[k]["tau2"], rel=10 * tol)
    assert rel(host(F), st.F.T) <= 100 * tol
    assert fifa.fifa_additive_kernel_nodes(m) > 0
    fifa.fifa_destroy_additive(ctx.h, m)


def test_additive_rejects_bad_arguments():
    X, y = additive4(256, seed=1)
    ctx = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=32, prec=fifa.FIFA_FP64, arena_bytes=1 << 28)
    p = _prior()
    pr = fifa.fifa_prior(p.a_tau2, p.b_tau2, p.a_sigma2, p.b_sigma2, p.logrho_mu, p.logrho_sd, p.prop_sd)
    hy = fifa.fifa_hyper(0, 1.0, RHO0, 0.5, NUG)
    Xd, yd = dev(X.T, torch), dev(y, torch)
    for d in (0, fifa.FIFA_ADDITIVE_MAX_D + 1):
        with pytest.raises(fifa.FifaError) as e:
            fifa.fifa_additive_create(ctx.h, Xd, yd, 256, d, hy, pr, 0)
        assert e.value.code == fifa.FIFA_ERR_INVALID_ARG
    Xn = X.T.copy()
    Xn[2, 17] = np.nan
    with pytest.raises(fifa.FifaError) as e:
        fifa.fifa_additive_create(ctx.h, dev(Xn, torch), yd, 256, 4, hy, pr, 0)
    assert e.value.code == fifa.FIFA_ERR_INVALID_ARG
