"""The Matern-5/2 configuration at n = 131072 (x ~ U[0,1], f a Matern-5/2 draw
with rho = 0.05, y = f + N(0, 0.2^2), leaf 128, ACA tolerance 1e-10), pinned
against the exact O(n) state-space route (oracle/statespace.py: Kalman filter
innovations and a Bryson-Frazier smoother), with no dense O(n^3) work:

  log det M~ against log det(M) = log det(tau2 C + sigma2 I) - n log sigma2,
  the posterior mean tau2 C~ M~^-1 y / sigma2 against E[f | y],

for the FP64 factor and solves, and for the mixed ones (FP64 factor applied in
FP32 as the preconditioner of FP64-residual conjugate gradients).

Tolerances come from the compression alone (M = s C + I with C the exact
kernel plus nugget, M~ its HODLR form, E = M~ - M with entries below s eps):
  |log det M~ - log det M| <= |tr(M^-1 E)| <= ||M^-1||_F ||E||_F <= sqrt(n) n s eps
  ||mean~ - mean|| = ||M~^-1 E M^-1 y|| <= n s eps ||y||     (||M^-1||, ||M~^-1|| <= 1)
plus FP64 rounding; mixed against FP64 on the GPU: 1e-8.
"""
import math

import numpy as np
import pytest

from oracle import statespace
from paper_2006_06537_gb300.inputs import matern_draw
from tests.gpu_util import build_lib, dev, host, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402

N, B, EPS, RHO, NOISE, NUG, TAU2 = 131072, 128, 1e-10, 0.05, 0.2, 1e-6, 1.0


@pytest.fixture(scope="module")
def exact():
    x, y, f = matern_draw(N, 1, rho=RHO, var=1.0, noise=NOISE)
    sigma2 = NOISE ** 2
    # y = f_K + (white nugget part of f) + e: the Kalman model's noise is sigma2 + tau2 nugget
    ld, quad, mk = statespace.kalman(x, y, RHO, TAU2, sigma2 + TAU2 * NUG)
    a = (y - mk) / (sigma2 + TAU2 * NUG)      # (tau2 C + sigma2 I)^-1 y
    mean = mk + TAU2 * NUG * a                 # tau2 C (tau2 C + sigma2 I)^-1 y
    return x, y, ld - N * math.log(sigma2), mean


@pytest.mark.parametrize("prec", [fifa.FIFA_FP64, fifa.FIFA_MIXED])
def test_matern_logdet_and_posterior_mean_against_state_space(exact, prec):
    x, y, ld_exact, mean_exact = exact
    s = TAU2 / NOISE ** 2
    ctx = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=32, prec=prec, refine_max=8, refine_tol=1e-13,
                       arena_bytes=4 << 30)
    xd, yd = dev(x, torch), dev(y, torch)
    C = fifa.fifa_assemble(ctx.h, xd, N, fifa.fifa_hyper(fifa.FIFA_KERNEL_MATERN52, TAU2, RHO, NOISE ** 2, NUG))
    WC = fifa.fifa_factor(ctx.h, C)
    M = fifa.fifa_shift_scale(ctx.h, C, s)
    WM = fifa.fifa_factor(ctx.h, M)
    ld, code = fifa.fifa_logdet(ctx.h, WM)
    assert code == fifa.FIFA_OK
    tol_ld = 2.0 * math.sqrt(N) * N * s * EPS + 1e-12 * abs(ld_exact)
    assert abs(ld - ld_exact) <= tol_ld, (ld, ld_exact, tol_ld)
    f = torch.empty(N, dtype=torch.float64, device="cuda")
    mean = torch.empty_like(f)
    fifa.fifa_sample(ctx.h, C, WC, WM, yd, TAU2, NOISE ** 2, 0, 0, 0, f, mean)
    torch.cuda.synchronize()
    err = float(np.linalg.norm(host(mean) - mean_exact))
    assert err <= N * s * EPS * np.linalg.norm(y) + 1e-10 * np.linalg.norm(mean_exact), err
    if prec == fifa.FIFA_MIXED:  # the mixed solves reproduce the FP64 ones
        ctx64 = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=32, arena_bytes=4 << 30)
        C6 = fifa.fifa_assemble(ctx64.h, xd, N, fifa.fifa_hyper(fifa.FIFA_KERNEL_MATERN52, TAU2, RHO, NOISE ** 2, NUG))
        W6 = fifa.fifa_factor(ctx64.h, C6)
        M6 = fifa.fifa_factor(ctx64.h, fifa.fifa_shift_scale(ctx64.h, C6, s))
        f6, m6 = torch.empty_like(f), torch.empty_like(f)
        fifa.fifa_sample(ctx64.h, C6, W6, M6, yd, TAU2, NOISE ** 2, 0, 0, 0, f6, m6)
        torch.cuda.synchronize()
        assert rel(host(mean), host(m6)) <= 1e-8
        assert rel(host(f), host(f6)) <= 1e-8
        ctx64.close()
    ctx.close()
