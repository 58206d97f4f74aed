"""GPU parity against the CPU oracle, through the C ABI.

Bit-exact: the deterministic exponential, the Philox words, ACA ranks, pivots,
bases and dense leaves (integer decisions taken from identical FP64 operation
sequences).  Tolerance (relative 2-norm): 1e-10 for products, solves of the
shifted M~, posterior means and log-determinants; for results that pass
through a factor W of an ill-conditioned C~ (W b, W^-1 b, the Algorithm 1
draw) the bound is max(1e-10, 8 kappa(A) u): a Cholesky-type factor is only
determined to kappa(A) u by two backward-stable FP64 computations that round
differently (Higham, Accuracy and Stability, Thm 10.8), so no tighter
pointwise agreement exists between any two correct implementations.
"""
import math

import numpy as np
import pytest

from oracle import detmath, factor, hodlr, rng, sampler
from paper_2006_06537_gb300.inputs import clustered, matern_draw, uniform_sine
from tests.gpu_util import build_lib, dev, host, oracle_bases, oracle_hmat, rel, used_mask

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402


def make_ctx(B=64, eps=1e-12, cap=32, prec=fifa.FIFA_FP64, refine_max=3, indep=0):
    return fifa.Context(leaf_size=B, aca_tol=eps, rank_cap=cap, prec=prec, refine_max=refine_max,
                        arena_bytes=1 << 30, independent_ctas=indep)


def test_det_exp_bitwise():
    ctx = make_ctx()
    g = np.random.default_rng(0)
    # inputs whose x 32/ln2 is exactly a half-integer: the range reduction's
    # rounding ties (to even) must agree too
    inv = float.fromhex("0x1.71547652b82fep+5")
    m = np.arange(-32000, 0, 7, dtype=np.float64)
    xt = (m + 0.5) / inv
    ties = xt[(xt * inv) == (m + 0.5)]
    assert len(ties) > 100
    x = np.concatenate([-g.uniform(0, 708, 200000), -g.uniform(0, 1, 50000), ties, [0.0, -708.0, -708.5, -1e-300]])
    xd = dev(x, torch)
    out = torch.empty_like(xd)
    fifa.fifa_det_exp(ctx.h, xd, out, len(x))
    torch.cuda.synchronize()
    assert np.array_equal(host(out).view(np.uint64), detmath.det_exp(x).view(np.uint64))


def test_philox_bitwise_and_normals():
    ctx = make_ctx()
    g = np.random.default_rng(1)
    ctr = g.integers(0, 2 ** 32, (5000, 4), dtype=np.uint64)
    seed = 0x123456789ABCDEF
    cd = torch.as_tensor(ctr.astype(np.uint32).view(np.int32)).cuda()
    out = torch.empty_like(cd)
    fifa.fifa_philox(ctx.h, seed, cd, out, len(ctr))
    torch.cuda.synchronize()
    got = host(out).view(np.uint32).astype(np.uint64)
    ref = rng.philox4x32_10(ctr, rng.key_of(seed))
    assert np.array_equal(got, ref)
    z = torch.empty(10001, dtype=torch.float64, device="cuda")
    fifa.fifa_normals(ctx.h, seed, rng.TAG_B, 7, 3, z, 10001)
    torch.cuda.synchronize()
    zr = rng.normals(10001, seed, rng.TAG_B, 7, 3)
    assert np.max(np.abs(host(z) - zr)) <= 1e-13


ASSEMBLY_CASES = [
    # n, B, kind, rho, nugget, eps, data
    (2048, 64, 0, 0.1, 1e-8, 1e-12, "sine"),      # first workload: n = 2048, B = 64, eps = 1e-12
    (1000, 37, 1, 0.05, 1e-8, 1e-10, "sine"),     # ragged leaves, Matern-5/2
    (20000, 64, 0, 0.01, 1e-8, 1e-10, "cluster"), # grouped (multi-CTA) ACA at the top levels
    (1, 64, 0, 0.1, 1e-8, 1e-12, "sine"),         # single point
    (65, 64, 1, 0.3, 1e-6, 1e-12, "sine"),        # one split, leaves 32 / 33
]


def _data(n, kind):
    if kind == "cluster":
        return clustered(n, 2)
    return uniform_sine(n, 0)


@pytest.mark.parametrize("case", ASSEMBLY_CASES)
def test_assembly_bit_exact(case):
    n, B, kind, rho, nug, eps, data = case
    x, y = _data(n, data)
    ctx = make_ctx(B=B, eps=eps)
    H = fifa.fifa_assemble(ctx.h, dev(x, torch), n, fifa.fifa_hyper(kind, 1.0, rho, 1.0, nug))
    ex = fifa.fifa_hmat_export(ctx.h, H)
    Ho = oracle_hmat(x, B, kind, rho, nug, eps, 32)
    t = Ho.tree
    assert ex["L"] == t.L and ex["nleaf"] == 2 ** t.L
    for lvl in range(t.L):
        for i in range(1 << lvl):
            nid = (1 << lvl) - 1 + i
            r = Ho.rank(lvl, i)
            assert ex["ranks"][nid] == r, (lvl, i)
            assert list(ex["row_piv"][nid, :r]) == Ho.row_piv[(lvl, i)]
            assert list(ex["col_piv"][nid, :r]) == Ho.col_piv[(lvl, i)]
    mask = used_mask(ex["ranks"], t, 32)
    ob = oracle_bases(Ho, n, 32)
    assert np.array_equal(ex["bases"][mask].view(np.uint64), ob[mask].view(np.uint64))
    for li, ((s, e), D) in enumerate(zip(t.leaves(), Ho.leaves)):
        m = e - s
        assert np.array_equal(ex["leaves"][li, :m, :m].T.copy().view(np.uint64), D.view(np.uint64))


def _factor_setup(n, B, kind, rho, nug, eps, s_shift=None, prec=fifa.FIFA_FP64, data="sine", indep=0):
    x, y = _data(n, data)
    ctx = make_ctx(B=B, eps=eps, prec=prec, refine_max=4, indep=indep)
    xd = dev(x, torch)
    H = fifa.fifa_assemble(ctx.h, xd, n, fifa.fifa_hyper(kind, 1.0, rho, 1.0, nug))
    Ho = oracle_hmat(x, B, kind, rho, nug, eps, 32)
    A, Ao = H, Ho
    if s_shift is not None:
        A = fifa.fifa_shift_scale(ctx.h, H, s_shift)
        Ao = hodlr.shift_scale(Ho, s_shift)
    F = fifa.fifa_factor(ctx.h, A)
    Fo = factor.factorize(Ao)
    return ctx, x, y, xd, H, Ho, A, Ao, F, Fo


FACTOR_CASES = [
    (2048, 64, 0, 0.1, 1e-6, 1e-12, None, "sine"),
    (1000, 37, 1, 0.05, 1e-6, 1e-10, None, "sine"),
    (2048, 64, 0, 0.1, 1e-8, 1e-12, 250.0, "sine"),   # M~ = s C~ + I of the first workload
    (20000, 64, 0, 0.01, 1e-8, 1e-10, 400.0, "cluster"),
    (65, 64, 1, 0.3, 1e-6, 1e-12, None, "sine"),
    (1, 64, 0, 0.1, 1e-6, 1e-12, None, "sine"),        # a single point: one 1 x 1 leaf, no level
    (2, 64, 0, 0.1, 1e-6, 1e-12, 3.0, "sine"),         # two points, shifted view
]


@pytest.mark.parametrize("indep", [0, 1])  # 0: grouped CTAs and the fused sweep; 1: independent CTAs, per-level sweeps
@pytest.mark.parametrize("case", FACTOR_CASES)
def test_factor_apply_solve_parity(case, indep):
    n, B, kind, rho, nug, eps, sh, data = case
    ctx, x, y, xd, H, Ho, A, Ao, F, Fo = _factor_setup(n, B, kind, rho, nug, eps, sh, data=data, indep=indep)
    ld, code = fifa.fifa_logdet(ctx.h, F)
    assert code == fifa.FIFA_OK
    # logdet: both sides backward stable; bound 1e-10 relative plus n * u * cond(W)^2 slack
    assert abs(ld - Fo.logdet) <= 1e-10 * abs(Fo.logdet) + 1e-6
    if n <= 4096:
        kappa = np.linalg.cond(hodlr.dense(Ao))
    else:
        # M~ = s C~ + I with C~ positive semidefinite and entrywise nonnegative
        # (SE): lambda_min >= 1 and lambda_max <= 1 + s ||C~||_inf, the row sums
        # of C~ (plus the compression error, n eps per row)
        assert sh is not None and kind == 0
        kappa = 1.0 + sh * (hodlr.matvec(Ho, np.ones(n)).max() + n * eps)
    wtol = max(1e-10, 8 * kappa * 1.1e-16)
    g = np.random.default_rng(9)
    v = g.standard_normal((2, n))
    vd = dev(v, torch)  # two column-major right-hand sides
    out = torch.empty_like(vd)
    for trans in (0, 1):
        for inv in (0, 1):
            fifa.fifa_apply_W(ctx.h, F, trans, inv, vd, out, 2)
            torch.cuda.synchronize()
            ref = factor.apply_W(Fo, v.T, trans=bool(trans), inverse=bool(inv)).T
            assert rel(host(out), ref) <= wtol, (trans, inv, rel(host(out), ref), wtol)
            out1 = torch.empty(n, dtype=torch.float64, device="cuda")  # one right-hand side
            fifa.fifa_apply_W(ctx.h, F, trans, inv, vd[1], out1, 1)
            torch.cuda.synchronize()
            assert rel(host(out1), ref[1]) <= wtol
    fifa.fifa_solve(ctx.h, F, vd, out, 2)
    torch.cuda.synchronize()
    ref = factor.solve(Fo, v.T).T
    assert rel(host(out), ref) <= wtol  # forward error of a solve is also kappa u
    fifa.fifa_matvec(ctx.h, A, vd, out, 2)
    torch.cuda.synchronize()
    ref = hodlr.matvec(Ao, v.T).T
    assert rel(host(out), ref) <= 1e-13


@pytest.mark.parametrize("nugget", [1e-3, 1e-8])
def test_sample_parity(nugget):
    """Algorithm 1 through fifa_sample vs the oracle's draw with the same Philox normals
    (first workload shape: n = 2048, B = 64, eps = 1e-12, SE)."""
    n, B = 2048, 64
    x, y = uniform_sine(n, 0)
    tau2, sigma2, rho = 0.9, 0.012, 0.1
    ctx = make_ctx(B=B, eps=1e-12)
    xd, yd = dev(x, torch), dev(y, torch)
    C = fifa.fifa_assemble(ctx.h, xd, n, fifa.fifa_hyper(0, tau2, rho, sigma2, nugget))
    WC = fifa.fifa_factor(ctx.h, C)
    M = fifa.fifa_shift_scale(ctx.h, C, tau2 / sigma2)
    WM = fifa.fifa_factor(ctx.h, M)
    f = torch.empty(n, dtype=torch.float64, device="cuda")
    mean = torch.empty_like(f)
    fifa.fifa_sample(ctx.h, C, WC, WM, yd, tau2, sigma2, 0, 0, 5, f, mean)
    torch.cuda.synchronize()
    Co = oracle_hmat(x, B, 0, rho, nugget, 1e-12, 32)
    FCo = factor.factorize(Co)
    FMo = factor.factorize(hodlr.shift_scale(Co, tau2 / sigma2))
    a = rng.normals(n, 0, rng.TAG_A, 5, 0)
    b = rng.normals(n, 0, rng.TAG_B, 5, 0)
    fo, mo = sampler.draw_f(Co, FCo, FMo, y, tau2, sigma2, a, b)
    kappa = np.linalg.cond(hodlr.dense(Co))
    assert rel(host(mean), mo) <= 1e-10
    assert rel(host(f), fo) <= max(1e-10, 8 * kappa * 1.1e-16)


def test_mixed_precision_solve_refines_to_fp64():
    n, B = 2048, 64
    s = 250.0
    ctx, x, y, xd, H, Ho, A, Ao, F, Fo = _factor_setup(n, B, 0, 0.1, 1e-8, 1e-12, s, prec=fifa.FIFA_MIXED)
    v = np.random.default_rng(4).standard_normal((2, n))
    vd = dev(v, torch)
    out = torch.empty_like(vd)
    fifa.fifa_solve(ctx.h, F, vd, out, 2)
    torch.cuda.synchronize()
    ref = factor.solve(Fo, v.T).T
    assert rel(host(out), ref) <= 1e-10
    # a mixed factor is an FP64 factor with an FP32 copy: its log-determinant is FP64
    ld, code = fifa.fifa_logdet(ctx.h, F)
    assert abs(ld - Fo.logdet) <= 1e-10 * abs(Fo.logdet)


def test_fp32_preconditioner_solve_within_its_precision():
    # the mixed factor's FP32 copy, applied in FP32 arithmetic, solves M~ to
    # about sqrt(kappa) u32 (W's condition number times the FP32 unit roundoff)
    # -- and no better: it really is FP32 work
    n, B = 2048, 64
    s = 250.0
    ctx, x, y, xd, H, Ho, A, Ao, F, Fo = _factor_setup(n, B, 0, 0.1, 1e-8, 1e-12, s, prec=fifa.FIFA_MIXED)
    v = np.random.default_rng(5).standard_normal((2, n))
    vd = dev(v, torch)
    out = torch.empty_like(vd)
    fifa.fifa_apply_precond(ctx.h, F, vd, out, 2)
    torch.cuda.synchronize()
    ref = factor.solve(Fo, v.T).T
    kappa = np.linalg.cond(hodlr.dense(Ao))
    err = rel(host(out), ref)
    assert 1e-10 < err <= 64 * math.sqrt(kappa) * 2.0 ** -24, (err, kappa)


def test_rejects_bad_inputs():
    ctx = make_ctx()
    x = np.array([0.3, 0.1, 0.5])
    with pytest.raises(fifa.FifaError) as e:
        fifa.fifa_assemble(ctx.h, dev(x, torch), 3, fifa.fifa_hyper(0, 1.0, 0.1, 1.0, 1e-8))
    assert e.value.code == fifa.FIFA_ERR_UNSORTED
    x = np.array([0.1, float("nan"), 0.5])
    with pytest.raises(fifa.FifaError) as e:
        fifa.fifa_assemble(ctx.h, dev(x, torch), 3, fifa.fifa_hyper(0, 1.0, 0.1, 1.0, 1e-8))
    assert e.value.code in (fifa.FIFA_ERR_INVALID_ARG, fifa.FIFA_ERR_UNSORTED)
    with pytest.raises(fifa.FifaError) as e:
        fifa.fifa_assemble(ctx.h, dev(np.array([0.1, 0.2]), torch), 2, fifa.fifa_hyper(0, 1.0, -1.0, 1.0, 1e-8))
    assert e.value.code == fifa.FIFA_ERR_INVALID_ARG


def test_not_spd_reported():
    # a negative nugget large enough to destroy positive definiteness of the leaves
    x, y = uniform_sine(256, 3)
    ctx = make_ctx(B=32, eps=1e-8)
    C = fifa.fifa_assemble(ctx.h, dev(x, torch), 256, fifa.fifa_hyper(0, 1.0, 0.2, 1.0, 0.0))
    M = fifa.fifa_shift_scale(ctx.h, C, -5.0)  # -5 C + I is indefinite
    F = fifa.fifa_factor(ctx.h, M)
    _, code = fifa.fifa_logdet(ctx.h, F, allow=(fifa.FIFA_ERR_NOT_SPD,))
    assert code == fifa.FIFA_ERR_NOT_SPD
