"""Algorithm 1.h (heteroskedastic noise) on the GPU against the oracle
(oracle/hetero.py) from the same Philox normals.

P~ = tau2 C~ + D^-1 is a per-row-diagonal view of C~ (fifa_add_diagonal); its
factor, the two solves and the products run in the library.  Tolerances as for
Algorithm 1: R = K~ P~^-1 y (no factor of C~ involved) 1e-10; the draw, which
carries W_C b, max(1e-10, 8 kappa(C~) u) with kappa computed densely.  The
mixed factor of P~ (FP32 copy as preconditioner, FP64 residuals) must give the
same results within 1e-8 of the FP64 ones.
"""
import numpy as np
import pytest

from oracle import factor, hetero, hodlr, rng
from paper_2006_06537_gb300.inputs import uniform_sine
from tests.gpu_util import build_lib, dev, host, oracle_hmat, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402

N, B, EPS, RHO, NUG, TAU2 = 2048, 64, 1e-12, 0.1, 1e-6, 0.7


def _precisions(x):
    # noise standard deviation varying smoothly over [0.05, 0.2]: d = 1 / sd^2
    sd = 0.05 + 0.15 * (0.5 + 0.5 * np.sin(6.0 * x))
    return 1.0 / (sd * sd)


def _gpu(x, y, d, prec):
    ctx = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=32, prec=prec, refine_max=8, refine_tol=1e-13,
                       arena_bytes=1 << 30)
    C = fifa.fifa_assemble(ctx.h, dev(x, torch), N, fifa.fifa_hyper(0, TAU2, RHO, 1.0, NUG))
    WC = fifa.fifa_factor(ctx.h, C)
    dd = dev(d, torch)
    dinv = dev(1.0 / d, torch)
    P = fifa.fifa_add_diagonal(ctx.h, C, TAU2, dinv)
    WP = fifa.fifa_factor(ctx.h, P)
    f = torch.empty(N, dtype=torch.float64, device="cuda")
    R = torch.empty_like(f)
    fifa.fifa_sample_hetero(ctx.h, C, WC, WP, dev(y, torch), TAU2, dd, 0, 3, 7, f, R)
    ld, code = fifa.fifa_logdet(ctx.h, WP)
    torch.cuda.synchronize()
    out = host(f), host(R), ld, code
    ctx.close()
    return out


def test_hetero_draw_matches_oracle_fp64_and_mixed():
    x, y = uniform_sine(N, 4)
    d = _precisions(x)
    Co = oracle_hmat(x, B, 0, RHO, NUG, EPS, 32)
    FCo = factor.factorize(Co)
    a0 = rng.normals(N, 0, rng.TAG_A, 7, 3)
    b0 = rng.normals(N, 0, rng.TAG_B, 7, 3)
    fo, Ro = hetero.draw_f_hetero(Co, FCo, y, TAU2, d, a0, b0)
    Po = factor.factorize(hetero.add_diagonal(Co, TAU2, 1.0 / d))
    kappa = np.linalg.cond(hodlr.dense(Co))
    tol = max(1e-10, 8 * kappa * 1.1e-16)
    f6, R6, ld6, code6 = _gpu(x, y, d, fifa.FIFA_FP64)
    assert code6 == fifa.FIFA_OK
    assert rel(R6, Ro) <= 1e-10
    assert rel(f6, fo) <= tol
    assert abs(ld6 - Po.logdet) <= 1e-10 * abs(Po.logdet)
    fm, Rm, ldm, codem = _gpu(x, y, d, fifa.FIFA_MIXED)
    assert codem == fifa.FIFA_OK
    assert rel(Rm, R6) <= 1e-8 and rel(fm, f6) <= 1e-8
    assert ldm == ld6  # the mixed factor is the FP64 one plus its FP32 copy


def test_hetero_equal_precisions_reduce_to_algorithm_1():
    # d_i = 1 / sigma2 for all i: Algorithm 1.h is Algorithm 1 with the same normals
    x, y = uniform_sine(N, 5)
    sigma2 = 0.02
    d = np.full(N, 1.0 / sigma2)
    f_h, R_h, _, _ = _gpu(x, y, d, fifa.FIFA_FP64)
    ctx = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=32, arena_bytes=1 << 30)
    C = fifa.fifa_assemble(ctx.h, dev(x, torch), N, fifa.fifa_hyper(0, TAU2, RHO, sigma2, NUG))
    WC = fifa.fifa_factor(ctx.h, C)
    WM = fifa.fifa_factor(ctx.h, fifa.fifa_shift_scale(ctx.h, C, TAU2 / sigma2))
    f = torch.empty(N, dtype=torch.float64, device="cuda")
    mean = torch.empty_like(f)
    fifa.fifa_sample(ctx.h, C, WC, WM, dev(y, torch), TAU2, sigma2, 0, 3, 7, f, mean)
    torch.cuda.synchronize()
    assert rel(R_h, host(mean)) <= 1e-10
    assert rel(f_h, host(f)) <= 1e-9
    ctx.close()
