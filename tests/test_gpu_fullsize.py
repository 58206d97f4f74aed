"""Parity at the headline size: n = 2^20 clustered inputs (the recipe and seed
the benchmark uses), leaf 32, eps 1e-10, rank cap 32, nugget 1e-6, rho 0.01:
the plan and launches the benchmark times.  The oracle cannot build or factor
the whole H-matrix at this size, so it checks outputs it can compute one by
one, and the factor is checked through identities that hold at any size.

* ACA (Sec. 3.2; partial pivoting as in the proof of Lemma 1) of sampled
  off-diagonal blocks at every level (the first, middle and last node):
  ranks, pivots and U / V bit for bit against the oracle's ACA of the same
  block; sampled dense leaves bit for bit.
* H-matrix product at sampled rows (the first, middle and last leaf): the
  oracle's row of C~ (its leaf block and the ancestor blocks above) times x,
  within the first-order bound n u sum_k |C~_pk| |x_k| of a sum of n products.
* The factor W of C~ (SI, after Ambikasaran et al., Thm 3.1): W W^T x = C~ x
  and C~ (C~^-1 b) = b in the normwise backward sense,
  ||residual|| <= 1e-13 (||C~|| ||vector|| + ||rhs||), with ||C~||_2 bounded
  by the largest row sum of C~ plus n eps (about 1.6e5 here, not n).  1e-13 is about
  2 L B u, twice the first-order growth of a backward-stable HODLR Cholesky
  with L = 15 levels and leaves of 32 rows.
* The log-determinant against the oracle's assembly and factorization of the
  whole H-matrix (the one full-size oracle computation, about a minute).
"""
import numpy as np
import pytest

from oracle import detmath
from oracle.aca import aca_block
from oracle.tree import Tree
from paper_2006_06537_gb300.inputs import clustered
from tests.gpu_util import build_lib, dev, host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402

N, B, EPS, CAP, NUG, RHO = 1 << 20, 32, 1e-10, 32, 1e-6, 0.01
U64 = np.finfo(np.float64).eps / 2


@pytest.fixture(scope="module")
def full():
    x, _ = clustered(N, 2)
    stream = torch.cuda.Stream()
    ctx = fifa.Context(leaf_size=B, aca_tol=EPS, rank_cap=CAP, prec=fifa.FIFA_FP64, arena_bytes=16 << 30,
                       stream=stream)
    xd = dev(x, torch)
    torch.cuda.synchronize()
    H = fifa.fifa_assemble(ctx.h, xd, N, fifa.fifa_hyper(0, 1.0, RHO, 1.0, NUG))
    ex = fifa.fifa_hmat_export(ctx.h, H, bases=False, leaves=True)
    t = Tree(N, B)
    c = detmath.kernel_const(0, RHO)
    blocks = {}

    def block(lvl, i):  # the oracle's ACA of one off-diagonal block, cached
        if (lvl, i) not in blocks:
            s, h, e = t.node(lvl, i)
            blocks[(lvl, i)] = aca_block(0, c, x[s:h], x[h:e], EPS, CAP)
        return blocks[(lvl, i)]

    yield dict(x=x, xd=xd, ctx=ctx, H=H, ex=ex, t=t, c=c, block=block, stream=stream)
    ctx.close()


def _sampled_nodes(lvl):
    return sorted({0, (1 << lvl) >> 1, (1 << lvl) - 1})


def test_fullsize_aca_blocks_and_leaves_bit_exact(full):
    ctx, H, ex, t, x = full["ctx"], full["H"], full["ex"], full["t"], full["x"]
    assert ex["L"] == t.L == 15 and ex["status"] == fifa.FIFA_OK
    for lvl in range(t.L):
        for i in _sampled_nodes(lvl):
            U, V, rows, cols, hit = full["block"](lvl, i)
            nid = (1 << lvl) - 1 + i
            r = U.shape[1]
            assert ex["ranks"][nid] == r and not hit, (lvl, i)
            assert list(ex["row_piv"][nid, :r]) == list(rows), (lvl, i)
            assert list(ex["col_piv"][nid, :r]) == list(cols), (lvl, i)
            s, h, e = t.node(lvl, i)
            got = fifa.fifa_hmat_level_rows(ctx.h, H, lvl, s, e - s)
            assert np.array_equal(got[:r, :h - s].T.copy().view(np.uint64), U.view(np.uint64)), (lvl, i)
            assert np.array_equal(got[:r, h - s:].T.copy().view(np.uint64), V.view(np.uint64)), (lvl, i)
    leaves = t.leaves()
    for li in (0, len(leaves) // 2, len(leaves) - 1):
        s, e = leaves[li]
        xi = x[s:e]
        D = detmath.kernel_entries(0, full["c"], xi[:, None], xi[None, :])
        D[np.diag_indices(e - s)] += NUG
        assert np.array_equal(ex["leaves"][li, :e - s, :e - s].T.copy().view(np.uint64), D.view(np.uint64))


def test_fullsize_matvec_sampled_rows(full):
    ctx, H, t, x = full["ctx"], full["H"], full["t"], full["x"]
    g = np.random.default_rng(20)
    v = g.standard_normal(N)
    vd = dev(v, torch)
    yd = torch.empty_like(vd)
    with torch.cuda.stream(full["stream"]):
        fifa.fifa_matvec(ctx.h, H, vd, yd, 1)
    torch.cuda.synchronize()
    y = host(yd)
    leaves = t.leaves()
    for li in (0, len(leaves) // 2, len(leaves) - 1):
        s0, e0 = leaves[li]
        xi = x[s0:e0]
        D = detmath.kernel_entries(0, full["c"], xi[:, None], xi[None, :])
        D[np.diag_indices(e0 - s0)] += NUG
        for p in (s0, (s0 + e0) // 2, e0 - 1):
            want = D[p - s0] @ v[s0:e0]
            mag = np.abs(D[p - s0]) @ np.abs(v[s0:e0])
            for lvl in range(t.L):
                i = li >> (t.L - lvl)
                U, V, _, _, _ = full["block"](lvl, i)
                s, h, e = t.node(lvl, i)
                if p < h:  # row of the upper block U V^T, partner columns [h, e)
                    want += U[p - s] @ (V.T @ v[h:e])
                    mag += np.abs(U[p - s]) @ (np.abs(V).T @ np.abs(v[h:e]))
                else:  # row of the lower block V U^T, partner columns [s, h)
                    want += V[p - h] @ (U.T @ v[s:h])
                    mag += np.abs(V[p - h]) @ (np.abs(U).T @ np.abs(v[s:h]))
            assert abs(y[p] - want) <= N * U64 * mag, (p, y[p], want)


def test_fullsize_factor_identities(full):
    ctx, H = full["ctx"], full["H"]
    F = fifa.fifa_factor(ctx.h, H)
    g = np.random.default_rng(21)
    xv = dev(g.standard_normal(N), torch)
    a, wwt, cx, z = (torch.empty_like(xv) for _ in range(4))
    with torch.cuda.stream(full["stream"]):
        fifa.fifa_apply_W(ctx.h, F, 1, 0, xv, a)   # W^T x
        fifa.fifa_apply_W(ctx.h, F, 0, 0, a, wwt)  # W W^T x
        fifa.fifa_matvec(ctx.h, H, xv, cx, 1)      # C~ x
        fifa.fifa_solve(ctx.h, F, cx, z)           # C~^-1 (C~ x)
    torch.cuda.synchronize()
    # ||C~||_2 <= ||C~||_inf: the largest row sum, here C~ 1 (the SE kernel and
    # the nugget are nonnegative; each ACA block is within eps of its kernel
    # block entrywise, so a row sum of |C~| exceeds the one of C~ by at most n eps)
    ones = torch.ones_like(xv)
    rs = torch.empty_like(xv)
    with torch.cuda.stream(full["stream"]):
        fifa.fifa_matvec(ctx.h, H, ones, rs, 1)
    torch.cuda.synchronize()
    norm_c = float(host(rs).max()) + N * EPS
    assert norm_c < 0.5 * N  # eight clusters: far below the n of the crude bound
    x_h, wwt_h, cx_h, z_h = host(xv), host(wwt), host(cx), host(z)
    nx, ncx = np.linalg.norm(x_h), np.linalg.norm(cx_h)
    eta_w = np.linalg.norm(wwt_h - cx_h) / (norm_c * nx)
    assert eta_w <= 1e-13, eta_w
    # C~ z = C~ x: the residual of the solve, through the library's product
    cz = torch.empty_like(xv)
    with torch.cuda.stream(full["stream"]):
        fifa.fifa_matvec(ctx.h, H, z, cz, 1)
    torch.cuda.synchronize()
    eta_s = np.linalg.norm(host(cz) - cx_h) / (norm_c * np.linalg.norm(z_h) + ncx)
    assert eta_s <= 1e-13, eta_s
    ld, code = fifa.fifa_logdet(ctx.h, F)
    assert code == fifa.FIFA_OK and np.isfinite(ld)
    fifa.fifa_destroy_fact(ctx.h, F)


def test_fullsize_logdet_matches_oracle(full):
    """The log-determinant the Metropolis step uses, against the oracle's own
    assembly and factorization of the whole H-matrix at n = 2^20 (about a
    minute of CPU time): both sides are backward-stable FP64 factorizations of
    the same C~ (its assembly is bit for bit the same) and must agree within
    the 1e-10 relative bound stated for the FP64 path.  (Measured 6.6e-11: the
    rounding of either side is amplified by C~'s condition number, about 1e11
    with the 1e-6 nugget, so the agreement is far from the unit roundoff.)"""
    from tests.gpu_util import oracle_hmat
    from oracle import factor

    ctx, H = full["ctx"], full["H"]
    F = fifa.fifa_factor(ctx.h, H)
    ld, code = fifa.fifa_logdet(ctx.h, F)
    fifa.fifa_destroy_fact(ctx.h, F)
    assert code == fifa.FIFA_OK
    Ho = oracle_hmat(full["x"], B, 0, RHO, NUG, EPS, CAP)
    Fo = factor.factorize(Ho)
    assert abs(ld - Fo.logdet) <= 1e-10 * abs(Fo.logdet), (ld, Fo.logdet)
