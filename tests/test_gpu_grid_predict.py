"""Two next rows on the GPU against their oracles:

* the length-scale on a discrete grid (Eq. posterior_gibs4; oracle/rhogrid.py):
  fifa_grid_create / fifa_grid_draw against rhogrid.grid_step on the same
  grid, f, tau2 and Philox uniform;
* the function posterior at new inputs (Eq. gp_posterior_newx;
  oracle/predict.py): fifa_predict against predict.predict.

Tolerances: every quantity here passes through C~^-1, so it is determined to
kappa(C~) u by two backward-stable FP64 computations (kappa computed densely):
log-weights within 8 kappa u (|logdet| + q / tau2), means and variances within
8 kappa u relative to their scale.  The grid index must agree unless the
uniform falls within that tolerance of a cumulative boundary.
"""
import math

import numpy as np
import pytest

from oracle import detmath, factor, hodlr, predict, rhogrid, rng
from paper_2006_06537_gb300.inputs import uniform_sine
from tests.gpu_util import build_lib, dev, host, oracle_hmat

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402

N, B, EPS = 2048, 64, 1e-12


def test_grid_draw_matches_oracle():
    # grid values 1% apart and a moderate nugget: probabilities spread over the
    # grid (not a point mass), kappa(C~) ~ 5e5
    x, y = uniform_sine(N, 6)
    nug, tau2 = 1e-3, 1.0
    rhos = [0.1 * (1 + 0.01 * k) for k in range(-2, 3)]
    lp = np.log(np.array([0.1, 0.2, 0.4, 0.2, 0.1]))
    f = np.sin(2 * math.pi * x)
    ctx = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=32, arena_bytes=1 << 30)
    g = fifa.fifa_grid_create(ctx.h, dev(x, torch), N, 0, nug, rhos, lp)
    Hs = [oracle_hmat(x, B, 0, r, nug, EPS, 32) for r in rhos]
    fs = [factor.factorize(H) for H in Hs]
    logdets, quads = rhogrid.grid_terms(fs, f)
    kappa = max(np.linalg.cond(hodlr.dense(H)) for H in Hs)
    tol = max(1e-10, 8 * kappa * 1.1e-16)
    spread = 0
    for it in range(6):
        seed, sid = 11, 2
        idx, probs = fifa.fifa_grid_draw(ctx.h, g, dev(f, torch), tau2, seed, sid, it, G=len(rhos))
        u = rng.scalar_uniform(0, seed, rng.TAG_MH_UNIF, it, sid)
        oidx, oprobs = rhogrid.grid_step(fs, f, tau2, u, lp)
        spread = max(spread, 1.0 - oprobs.max())
        lw_tol = 8 * tol * (np.abs(logdets) + quads / tau2).max() + 1e-12
        assert np.all(np.abs(probs - oprobs) <= 2 * lw_tol * np.maximum(probs, oprobs) + 1e-300), (probs, oprobs)
        cdf = np.cumsum(oprobs)
        if np.min(np.abs(cdf - u)) > 4 * lw_tol:
            assert idx == oidx
        tau2 *= 1.3  # different weights every draw
    assert spread > 0.1  # the draws were not decided by a point mass
    # the grid's factors are the library's ordinary ones: the grid point's log-determinant
    C2, W2 = fifa.fifa_grid_get(g, 2)
    ld, _ = fifa.fifa_logdet(ctx.h, W2)
    assert abs(ld - fs[2].logdet) <= 1e-10 * abs(fs[2].logdet)
    fifa.fifa_destroy_grid(ctx.h, g)
    ctx.close()


@pytest.mark.parametrize("kind,rho", [(0, 0.1), (1, 0.08)])
def test_predict_matches_oracle(kind, rho):
    x, y = uniform_sine(N, 7)
    nug, tau2 = 1e-4, 0.8
    f = np.sin(2 * math.pi * x)
    g = np.random.default_rng(3)
    xs = np.concatenate([g.uniform(-0.2, 1.2, 30), x[[0, 500, 2047]], [0.5, 3.0]])
    ctx = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=32, arena_bytes=1 << 30)
    xd = dev(x, torch)
    C = fifa.fifa_assemble(ctx.h, xd, N, fifa.fifa_hyper(kind, tau2, rho, 1.0, nug))
    W = fifa.fifa_factor(ctx.h, C)
    mu = torch.empty(len(xs), dtype=torch.float64, device="cuda")
    var = torch.empty_like(mu)
    fifa.fifa_predict(ctx.h, C, W, xd, dev(f, torch), dev(xs, torch), len(xs), tau2, mu, var)
    torch.cuda.synchronize()
    H = oracle_hmat(x, B, kind, rho, nug, EPS, 32)
    om, ov = predict.predict(H, x, xs, f, tau2, kind, detmath.kernel_const(kind, rho))
    kappa = np.linalg.cond(hodlr.dense(H))
    tol = max(1e-10, 8 * kappa * 1.1e-16)
    assert np.linalg.norm(host(mu) - om) <= tol * np.linalg.norm(om)
    assert np.all(np.abs(host(var) - ov) <= tol * tau2 * 10)
    assert host(var)[-1] == pytest.approx(tau2, rel=1e-12)  # far from every input: the prior variance
    ctx.close()
