"""The bench line's KL report (Sec. 4.1.3, Theorem 4.1) checked on the CPU:
bench.dense_ctilde must rebuild the oracle's C~ from an export in the
library's layout (level-major bases, U on the left child's rows and V on the
right child's; column-major leaves), and bench.kl_terms must agree with the
oracle's dense posterior and Gaussian KL on the same K and K~."""
import numpy as np

import bench
from oracle import dense, hodlr
from paper_2006_06537_gb300.inputs import clustered
from tests.gpu_util import oracle_bases, oracle_hmat

N, B, RHO, NUG, EPS, CAP = 512, 32, 0.01, 1e-6, 1e-10, 32


def _export(H, n):
    """The oracle's H-matrix in fifa_hmat_export's layout."""
    L = H.tree.L
    ranks = np.zeros((1 << L) - 1 if L > 0 else 0, dtype=np.int64)
    for lvl in range(L):
        for i in range(1 << lvl):
            ranks[(1 << lvl) - 1 + i] = H.U[(lvl, i)].shape[1]
    leaves = H.tree.leaves()
    bm = max(e - s for s, e in leaves)
    lv = np.zeros((len(leaves), bm, bm))
    for i, (s, e) in enumerate(leaves):
        lv[i, :e - s, :e - s] = H.leaves[i].T  # column-major
    return {"L": L, "ranks": ranks, "bases": oracle_bases(H, n, CAP), "leaves": lv}


def test_dense_ctilde_and_kl_match_the_oracle():
    x, y = clustered(N, 2, noise=0.05)
    H = oracle_hmat(x, B, 0, RHO, NUG, EPS, CAP)
    Ct = bench.dense_ctilde(_export(H, N), N)
    Cd = hodlr.dense(H)
    assert np.max(np.abs(Ct - Cd)) <= 1e-15
    tau2, sigma2 = float(np.var(y)), 0.0025
    got = bench.kl_terms(x, y, Ct, tau2, sigma2, RHO, NUG)
    dx = x[:, None] - x[None, :]
    K = tau2 * (np.exp(-dx * dx / (2 * RHO * RHO)) + NUG * np.eye(N))
    mp, Sp = dense.posterior(K, y, sigma2)
    Kt = tau2 * Cd
    Mt = Kt / sigma2 + np.eye(N)
    Sq = Kt @ np.linalg.inv(Mt)
    Sq = 0.5 * (Sq + Sq.T)
    mq = Sq @ y / sigma2
    kl, parts = dense.kl_gauss(mp, Sp, mq, Sq)
    assert got["kl"] >= 0.0
    assert abs(got["kl"] - kl) <= 1e-6 * max(abs(kl), 1e-12) + 1e-9, (got["kl"], kl)
    assert got["e_max"] <= 2 * EPS * tau2 + 1e-15
