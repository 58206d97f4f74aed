"""KL divergence between the exact posterior of f and the one the GPU's
H-matrices define (Sec. 4.1.3, Theorem 4.1; the Gaussian KL of its proof).

P = N(mu_P, Sigma_P): the exact posterior for K = tau2 (C + nugget I) (dense).
Q = N(mu_Q, Sigma_Q): the law Algorithm 1 samples (Lemma 1), Sigma_Q = K~ M~^-1,
mu_Q = Sigma_Q y / sigma2, with K~ = tau2 C~ rebuilt densely from the GPU's
exported leaves and ACA bases, M~ = K~ / sigma2 + I.

Checks: KL >= 0; its log-determinant part is within Theorem 4.1's first term
2 n^2 e_max (e_max = max |K~ - K|, |M~ - M|, the proof's max-norm error); the KL
falls as the ACA tolerance falls; and the GPU's K~ meets the tolerance in the
max norm (the premise of the theorem).
"""
import math

import numpy as np
import pytest

from oracle import dense
from paper_2006_06537_gb300.inputs import uniform_sine
from tests.gpu_util import build_lib, dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402

N, B, RHO, NUG, TAU2, SIGMA2 = 2048, 64, 0.1, 1e-6, 0.5, 0.01


def gpu_dense_ctilde(x, eps):
    """C~ assembled on the GPU, exported, and written out densely."""
    ctx = fifa.Context(leaf_size=B, aca_tol=eps, rank_cap=32, arena_bytes=1 << 28)
    H = fifa.fifa_assemble(ctx.h, dev(x, torch), N, fifa.fifa_hyper(0, 1.0, RHO, 1.0, NUG))
    ex = fifa.fifa_hmat_export(ctx.h, H)
    ctx.close()
    L, cap, Bm = ex["L"], ex["cap"], ex["Bm"]
    bounds = [[0, N]]
    for _ in range(L):
        bounds = [b for s, e in bounds for b in ([s, s + (e - s) // 2], [s + (e - s) // 2, e])]
    Ct = np.zeros((N, N))
    for i, (s, e) in enumerate(bounds):
        m = e - s
        Ct[s:e, s:e] = ex["leaves"][i, :m, :m].T  # leaves are column-major
    nodes = [[0, N]]
    for lvl in range(L):
        for i, (s, e) in enumerate(nodes):
            h = s + (e - s) // 2
            r = ex["ranks"][(1 << lvl) - 1 + i]
            U = ex["bases"][lvl, :r, s:h].T
            V = ex["bases"][lvl, :r, h:e].T
            Ct[s:h, h:e] = U @ V.T
            Ct[h:e, s:h] = V @ U.T
        nodes = [b for s, e in nodes for b in ([s, s + (e - s) // 2], [s + (e - s) // 2, e])]
    return Ct


def kl_report(x, y, eps):
    d = x[:, None] - x[None, :]
    K = TAU2 * (np.exp(-d * d / (2 * RHO * RHO)) + NUG * np.eye(N))
    Kt = TAU2 * gpu_dense_ctilde(x, eps)
    mu_p, S_p = dense.posterior(K, y, SIGMA2)
    Mt = Kt / SIGMA2 + np.eye(N)
    S_q = Kt @ np.linalg.inv(Mt)
    S_q = 0.5 * (S_q + S_q.T)
    mu_q = S_q @ y / SIGMA2
    kl, parts = dense.kl_gauss(mu_p, S_p, mu_q, S_q)
    e_max = max(np.abs(Kt - K).max(), np.abs(Mt - (K / SIGMA2 + np.eye(N))).max())
    return kl, parts, e_max


def test_kl_of_gpu_hmatrix_posterior_to_exact():
    x, y = uniform_sine(N, 0)
    kls = []
    for eps in (1e-6, 1e-9, 1e-12):
        kl, parts, e_max = kl_report(x, y, eps)
        assert e_max <= 8 * (TAU2 / SIGMA2) * eps + 1e-12  # the max-norm premise (M~ carries s = tau2 / sigma2)
        assert kl >= -1e-9
        assert abs(parts["logdet"]) <= 2 * N * N * e_max
        kls.append(kl)
    assert kls[0] > kls[1] > kls[2] or kls[2] < 1e-9
    assert kls[2] < 1e-6
