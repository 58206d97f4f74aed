"""Pins for the oracle's tree, ACA, HODLR assembly, factorization and solves.

Checks against brute force on small n (dense kernel matrices, numpy
Cholesky / slogdet / solve), exact low-rank matrices, the special case B >= n
that reduces to a plain dense Cholesky, and the ranks printed in the paper's
SI worked example.
"""
import json
import os

import numpy as np
import pytest

from oracle import aca, detmath, factor, hodlr, tree
from paper_2006_06537_gb300.inputs import uniform_sine

GOLD = os.path.join(os.path.dirname(__file__), "golden", "si_worked_example.json")


@pytest.mark.parametrize("n,B", [(1, 1), (7, 2), (100, 64), (2048, 64), (1000, 37), (129, 64)])
def test_tree_partition(n, B):
    t = tree.Tree(n, B)
    sizes = [e - s for s, e in t.leaves()]
    assert sum(sizes) == n and max(sizes) <= B and max(sizes) - min(sizes) <= 1
    assert len(sizes) == 2 ** t.L
    if t.L > 0:
        assert -(-n // 2 ** (t.L - 1)) > B  # L is minimal
    for lvl in range(t.L + 1):
        b = t.bounds[lvl]
        assert b[0] == 0 and b[-1] == n and np.all(np.diff(b) >= 0)


def test_aca_recovers_exact_low_rank():
    g = np.random.default_rng(3)
    G, Hm = g.standard_normal((90, 4)), g.standard_normal((70, 4))
    A = G @ Hm.T
    U, V, rows, cols, hit = aca.aca_entries(lambda i: A[i], lambda j: A[:, j], 90, 70, 1e-10, 20)
    assert U.shape[1] == 4 and not hit
    assert np.abs(U @ V.T - A).max() < 1e-12 * np.abs(A).max()
    assert rows[0] == 89 and len(set(rows)) == 4 and len(set(cols)) == 4


@pytest.mark.parametrize("kind", [detmath.KERNEL_SE, detmath.KERNEL_MATERN52])
@pytest.mark.parametrize("eps", [1e-6, 1e-10, 1e-12])
def test_aca_max_norm_error(kind, eps):
    g = np.random.default_rng(4)
    xr = np.sort(g.uniform(0.0, 0.5, 300))
    xc = np.sort(g.uniform(0.5, 1.0, 260))
    c = detmath.kernel_const(kind, 0.1)
    U, V, rows, cols, hit = aca.aca_block(kind, c, xr, xc, eps, 128)
    A = detmath.kernel_entries(kind, c, xr[:, None], xc[None, :])
    assert not hit
    assert np.abs(A - U @ V.T).max() <= 10 * eps


def test_aca_separated_clusters_rank_zero():
    xr = np.linspace(0.0, 0.01, 50)
    xc = np.linspace(0.9, 1.0, 40)
    c = detmath.kernel_const(detmath.KERNEL_SE, 0.01)
    U, V, *_ = aca.aca_block(detmath.KERNEL_SE, c, xr, xc, 1e-10, 32)
    assert U.shape[1] == 0


def _svd_rank(B, tol):
    U, s, Vt = np.linalg.svd(B)
    for r in range(len(s) + 1):
        if np.abs(B - (U[:, :r] * s[:r]) @ Vt[:r]).max() <= tol:
            return r


def test_si_worked_example_ranks():
    gold = json.load(open(GOLD))
    x = np.sort(np.random.default_rng(0).uniform(0, 1, 200))
    c = 4.0  # exp(-4 (x-x')^2) is the SE form with c = 1/(2 rho^2) = 4
    H = hodlr.assemble(x, 50, detmath.KERNEL_SE, c, 0.0, 1e-8, 64)
    assert H.tree.L == 2
    A = hodlr.dense_kernel(x, detmath.KERNEL_SE, c, 0.0)
    assert _svd_rank(A[:100, 100:], 1e-8) == gold["rank_level0_block_tol_1e-8"]
    assert _svd_rank(A[:50, 50:100], 1e-8) == gold["rank_level1_blocks_tol_1e-8"]
    r0 = H.rank(0, 0)
    assert gold["rank_level0_block_tol_1e-8"] <= r0 <= gold["rank_level0_block_tol_1e-8"] + 3
    for i in range(2):
        assert gold["rank_level1_blocks_tol_1e-8"] <= H.rank(1, i) <= gold["rank_level1_blocks_tol_1e-8"] + 3
    assert abs(_svd_rank(A[:100, 100:], 1e-12) - gold["rank_n200_half_block_tol_1e-12_svd"]) <= 1
    x2 = np.sort(np.random.default_rng(0).uniform(0, 1, 2000))
    A2 = hodlr.dense_kernel(x2, detmath.KERNEL_SE, c, 0.0)
    assert abs(_svd_rank(A2[:1000, 1000:], 1e-12) - gold["rank_n2000_half_block_tol_1e-12_svd"]) <= 1


def _setup(n=512, B=32, kind=detmath.KERNEL_SE, rho=0.1, nugget=1e-6, eps=1e-12):
    x, y = uniform_sine(n, 0)
    c = detmath.kernel_const(kind, rho)
    H = hodlr.assemble(x, B, kind, c, nugget, eps, 64)
    return x, y, c, H


@pytest.mark.parametrize("kind", [detmath.KERNEL_SE, detmath.KERNEL_MATERN52])
def test_assembly_max_norm(kind):
    x, y, c, H = _setup(kind=kind, eps=1e-10)
    A = hodlr.dense_kernel(x, kind, c, 1e-6)
    assert np.abs(hodlr.dense(H) - A).max() <= 10 * 1e-10


def test_matvec_and_shift_scale():
    x, y, c, H = _setup()
    A = hodlr.dense(H)
    v = np.random.default_rng(5).standard_normal((len(x), 3))
    np.testing.assert_allclose(hodlr.matvec(H, v), A @ v, rtol=0, atol=1e-12 * np.abs(A @ v).max())
    s = 37.5
    M = hodlr.shift_scale(H, s)
    # an off-diagonal entry is a rank-r dot product, formed as (s U) V^T in the
    # view and s (U V^T) here: the two roundings differ by up to ~r ulps of the
    # largest entry (dot-product error bound gamma_r), plus the scale and shift
    rmax = max(H.rank(l, i) for l in range(H.tree.L) for i in range(1 << l)) if H.tree.L else 0
    np.testing.assert_allclose(hodlr.dense(M), s * A + np.eye(len(x)), rtol=0,
                               atol=(rmax + 4) * np.spacing(s * np.abs(A).max()))


def test_single_leaf_reduces_to_dense_cholesky():
    x, y = uniform_sine(50, 1)
    c = detmath.kernel_const(0, 0.2)
    H = hodlr.assemble(x, 64, 0, c, 1e-6, 1e-12, 64)
    assert H.tree.L == 0
    F = factor.factorize(H)
    A = hodlr.dense_kernel(x, 0, c, 1e-6)
    assert np.array_equal(F.Lleaf[0], np.linalg.cholesky(A))
    L = np.linalg.cholesky(A)
    assert F.logdet == pytest.approx(2.0 * np.log(np.diag(L)).sum(), rel=1e-15)
    assert abs(F.logdet - np.linalg.slogdet(A)[1]) <= 1e-15 * np.linalg.cond(A) * len(x)


@pytest.mark.parametrize("kind", [detmath.KERNEL_SE, detmath.KERNEL_MATERN52])
def test_factor_brute_force(kind):
    x, y, c, H = _setup(kind=kind)
    A = hodlr.dense(H)
    n = len(x)
    F = factor.factorize(H)
    W = factor.apply_W(F, np.eye(n))
    assert np.abs(W @ W.T - A).max() <= 1e-13 * np.abs(A).max()
    Winv = factor.apply_W(F, np.eye(n), inverse=True)
    np.testing.assert_allclose(Winv @ W, np.eye(n), atol=1e-9)
    np.testing.assert_allclose(factor.apply_W(F, np.eye(n), trans=True), W.T, atol=1e-13)
    np.testing.assert_allclose(factor.apply_W(F, np.eye(n), trans=True, inverse=True), Winv.T, atol=1e-9 * np.abs(Winv).max())
    sign, ld = np.linalg.slogdet(A)
    assert sign > 0
    kappa = np.linalg.cond(A)
    assert abs(F.logdet - ld) <= 1e-13 * kappa * n
    b = np.random.default_rng(6).standard_normal(n)
    xs = factor.solve(F, b)
    assert np.linalg.norm(A @ xs - b) <= 1e-15 * kappa * n * np.linalg.norm(b)


def test_factor_of_shifted_matrix_is_accurate():
    x, y, c, H = _setup(nugget=1e-8)
    s = 100.0
    M = hodlr.shift_scale(H, s)
    A = hodlr.dense(M)
    F = factor.factorize(M)
    b = np.random.default_rng(7).standard_normal(len(x))
    xs = factor.solve(F, b)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(xs - ref) <= 1e-10 * np.linalg.norm(ref)
    assert F.logdet == pytest.approx(np.linalg.slogdet(A)[1], rel=1e-12)


def test_not_spd_is_reported():
    x, y = uniform_sine(128, 2)
    c = detmath.kernel_const(0, 0.5)
    H = hodlr.assemble(x, 16, 0, c, 0.0, 1e-3, 64)  # no nugget, coarse tolerance
    H.leaves[0][0, 0] = -1.0
    with pytest.raises(factor.NotSPD):
        factor.factorize(H)
