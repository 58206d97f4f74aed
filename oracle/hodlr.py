"""HODLR matrix of the kernel (oracle side): Sec. 3.2 and the SI example.

C~ is stored as
  * dense diagonal leaves  D_i = C(I_i, I_i) + nugget * I  (nugget: Sec. 4.1.4),
  * for every non-leaf node [s, e) with split h, the off-diagonal block
    C([s,h), [h,e)) ~= U V^T from ``aca_block`` (the lower block is its transpose).

``shift_scale`` forms M~ = s C~ + I from C~ exactly as the proof of Theorem 4.1
allows (M~ built from K~): leaves s*D_i + I, U scaled by s, V shared.  Because
the identity only touches the dense leaves, M~ - (s C~ + I) is zero entry by
entry, the precondition of Lemma 1.
"""
from __future__ import annotations

import numpy as np

from .aca import aca_block
from .detmath import kernel_entries
from .tree import Tree


class HMat:
    """tree, leaves[i], U[(l,i)], V[(l,i)], rows/cols pivots, ranks, hit_cap flags."""

    def __init__(self, tree: Tree):
        self.tree = tree
        self.leaves = []
        self.U, self.V = {}, {}
        self.row_piv, self.col_piv = {}, {}
        self.hit_cap = {}

    def rank(self, lvl, i):
        return self.U[(lvl, i)].shape[1]

    def ranks(self):
        return {key: u.shape[1] for key, u in self.U.items()}


def assemble(x, B, kind, c, nugget, eps, cap):
    """C~(rho) for sorted inputs x: leaves of the kernel plus nugget, ACA off-diagonal blocks."""
    x = np.asarray(x, dtype=np.float64)
    if np.any(np.diff(x) < 0):
        raise ValueError("inputs must be sorted")
    t = Tree(len(x), B)
    H = HMat(t)
    for s, e in t.leaves():
        xi = x[s:e]
        D = kernel_entries(kind, c, xi[:, None], xi[None, :])
        D[np.diag_indices(e - s)] += nugget
        H.leaves.append(D)
    for lvl in range(t.L):
        for i in range(1 << lvl):
            s, h, e = t.node(lvl, i)
            U, V, rows, cols, hit = aca_block(kind, c, x[s:h], x[h:e], eps, cap)
            H.U[(lvl, i)], H.V[(lvl, i)] = U, V
            H.row_piv[(lvl, i)], H.col_piv[(lvl, i)] = rows, cols
            H.hit_cap[(lvl, i)] = hit
    return H


def shift_scale(H: HMat, s: float) -> HMat:
    """M~ = s * C~ + I (leaves s*D + I, U -> s*U, V unchanged)."""
    M = HMat(H.tree)
    for D in H.leaves:
        Dm = s * D
        Dm[np.diag_indices(D.shape[0])] += 1.0
        M.leaves.append(Dm)
    for key in H.U:
        M.U[key] = s * H.U[key]
        M.V[key] = H.V[key].copy()
        M.row_piv[key], M.col_piv[key] = H.row_piv[key], H.col_piv[key]
        M.hit_cap[key] = H.hit_cap[key]
    return M


def dense(H: HMat):
    """The n x n matrix the HODLR representation stands for."""
    t = H.tree
    A = np.zeros((t.n, t.n))
    for (s, e), D in zip(t.leaves(), H.leaves):
        A[s:e, s:e] = D
    for lvl in range(t.L):
        for i in range(1 << lvl):
            s, h, e = t.node(lvl, i)
            blk = H.U[(lvl, i)] @ H.V[(lvl, i)].T
            A[s:h, h:e] = blk
            A[h:e, s:h] = blk.T
    return A


def matvec(H: HMat, x):
    """y = C~ x: leaf products plus, per node, y_top += U (V^T x_bot), y_bot += V (U^T x_top)."""
    t = H.tree
    x = np.asarray(x, dtype=np.float64)
    squeeze = x.ndim == 1
    X = x.reshape(t.n, -1)
    Y = np.zeros_like(X)
    for (s, e), D in zip(t.leaves(), H.leaves):
        Y[s:e] += D @ X[s:e]
    for lvl in range(t.L):
        for i in range(1 << lvl):
            s, h, e = t.node(lvl, i)
            U, V = H.U[(lvl, i)], H.V[(lvl, i)]
            Y[s:h] += U @ (V.T @ X[h:e])
            Y[h:e] += V @ (U.T @ X[s:h])
    return Y[:, 0] if squeeze else Y


def dense_kernel(x, kind, c, nugget):
    """Exact C + nugget I (for brute-force checks at small n)."""
    x = np.asarray(x, dtype=np.float64)
    A = kernel_entries(kind, c, x[:, None], x[None, :])
    A[np.diag_indices(len(x))] += nugget
    return A
