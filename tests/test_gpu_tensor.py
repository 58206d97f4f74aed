"""The tensor-product model of Sec. 4.2 on the GPU (fifa_tensor_*) against the
oracle's sweep (oracle/tensor.py) from the same state and Philox streams.

Each block draws f_h - 1 by Algorithm 1.h; beta and sigma2 follow their
conditionals and every length-scale its Metropolis step.  Quantities that pass
through a factor of C~ (the draws, hence beta, sigma2, the Metropolis
ratios) are compared within max(1e-10, 8 kappa u) scaled as in the 1-D chain
tests, kappa the largest dense condition number of the blocks' C~; the
Metropolis decisions must agree unless log u sits within that tolerance of
log alpha.
"""
import math

import numpy as np
import pytest

from oracle import hodlr, sampler, tensor
from paper_2006_06537_gb300.inputs import tensor2
from tests.gpu_util import build_lib, dev, host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402

N, D, B, EPS, RHO0, NUG = 1024, 2, 32, 1e-12, 0.2, 1e-6


def _prior():
    return sampler.Prior(a_tau2=1.0, b_tau2=1.0, a_sigma2=1.0, b_sigma2=1.0, logrho_mu=math.log(RHO0),
                         logrho_sd=1.0, prop_sd=0.2)


def test_tensor_sweeps_match_oracle():
    X, y = tensor2(N)
    sweeps, seed = 3, 5
    s2 = 0.5 * float(np.var(y))
    opts = sampler.Opts(B=B, eps=EPS, cap=32, kind=0, nugget=NUG)
    st = tensor.tensor_init(X, y, RHO0, opts, sigma2=s2, beta=1.0)
    kappa = max(np.linalg.cond(hodlr.dense(b["HC"])) for b in st.blocks)
    bp = tensor.BetaPrior(mu=1.0, sd=1.0)
    for _ in range(sweeps):
        tensor.tensor_sweep(st, y, _prior(), bp, opts, seed)
    ctx = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=32, arena_bytes=1 << 30, stream=torch.cuda.Stream())
    p = _prior()
    pr = fifa.fifa_prior(p.a_tau2, p.b_tau2, p.a_sigma2, p.b_sigma2, p.logrho_mu, p.logrho_sd, p.prop_sd)
    Xd = dev(np.ascontiguousarray(X.T), torch)
    m = fifa.fifa_tensor_create(ctx.h, Xd, dev(y, torch), N, D, fifa.fifa_hyper(0, 1.0, RHO0, s2, NUG), pr, 1.0, 1.0,
                                1.0, seed)
    tr = np.zeros((sweeps, fifa.fifa_tensor_trace_fields(D)))
    fifa.fifa_tensor_sweep(ctx.h, m, sweeps, tr)
    F = torch.empty((D, N), dtype=torch.float64, device="cuda")
    beta, sigma2, blocks = fifa.fifa_tensor_get(ctx.h, m, D, F)
    tol = max(1e-10, 8 * kappa * 1.1e-16)
    for t, o in zip(tr, st.trace):
        assert int(t[0]) == o["it"]
        assert abs(t[1] - o["beta"]) <= 100 * tol * abs(o["beta"]), (t[1], o["beta"])
        assert abs(t[2] - o["sigma2"]) <= 100 * tol * o["sigma2"], (t[2], o["sigma2"])
        assert abs(t[3] - o["rss"]) <= 100 * tol * o["rss"]
        assert t[4] == 0.0
        for h in range(D):
            if bool(t[5 + D + h]) == o["accept"][h]:
                assert t[5 + h] == pytest.approx(o["rho"][h], rel=1e-12)
    assert beta == pytest.approx(st.beta, rel=100 * tol)
    Fo = st.F.T
    assert np.linalg.norm(host(F) - Fo) <= 1000 * tol * np.linalg.norm(Fo)
    fifa.fifa_destroy_tensor(ctx.h, m)
    ctx.close()
