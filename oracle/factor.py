"""Symmetric factorization A = W W^T of a HODLR matrix (oracle side).

Follows the SI section "HODLR decomposition and factorization" (after
Ambikasaran et al. 2014, Theorem 3.1) in its stated order:

1. factor every dense diagonal leaf, A_L = blkdiag(L_i) with L_i = chol(D_i);
2. apply the inverse of that block-diagonal factor to every U and V (each
   basis row block lying in leaf i is replaced by L_i^-1 times it), so that
   A = A_L A~_L A_L^T where A~_L has identity diagonal blocks;
3. for levels l = L-1 down to 0: every node's diagonal block of the current
   matrix is I + U^ X U^T with U^ = blkdiag(U~, V~) and X = [[0, I], [I, 0]].
   With the QR factorizations U~ = Q_U R_U, V~ = Q_V R_V (R upper triangular
   with positive diagonal), Q = blkdiag(Q_U, Q_V), R = blkdiag(R_U, R_V),
       I + U^ X U^T = I + Q (R X R^T) Q^T = (I + Q Z Q^T)(I + Q Z Q^T)^T
   with I + Z = L_S = chol(I + R X R^T) (Theorem 3.1 of Ambikasaran et al.),
   so the node factor and its inverse are
       A_l(node)    = I + Q (L_S - I) Q^T,
       A_l(node)^-1 = I + Q (L_S^-1 - I) Q^T   (Q has orthonormal columns),
   and the inverse node factor is applied to the rows of every ancestor's
   basis that fall inside the node, which leaves identity blocks one level up.
   The node stores Q in place of its transformed bases.
The result is W = A_L A_{L-1} ... A_0.

Log-determinant (SI, "Determinant computation speedup"): det(A) = det(W)^2,
det of a leaf factor is the product of its diagonal and, by Sylvester's
theorem, det(I + Q Z Q^T) = det(I + Z) = det(L_S).  So
    log det A = 2 * (sum over leaves of sum log diag L_i
                     + sum over nodes of sum log diag L_S).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from .hodlr import HMat


class NotSPD(Exception):
    pass


class Factor:
    """Leaf factors L_i; per node the orthonormal bases Q_U (Ut) and Q_V (Vt)
    and the small matrices Y = L_S - I, Yinv = L_S^-1 - I."""

    def __init__(self, tree):
        self.tree = tree
        self.Lleaf = []
        self.Ut, self.Vt = {}, {}
        self.Y, self.Yinv = {}, {}
        self.logdet = 0.0


def _chol(A):
    try:
        return np.linalg.cholesky(A)
    except np.linalg.LinAlgError as exc:
        raise NotSPD(str(exc)) from exc


def _qr_pos(A):
    """Householder QR with the signs fixed so that diag(R) > 0 (the unique thin QR)."""
    Q, R = np.linalg.qr(A)
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * sgn, R * sgn[:, None]


def _basis_rows_in(F, lvl, i, s, e):
    """Views of the transformed basis rows of ancestor node (lvl, i) that lie in [s, e)."""
    a_s, a_h, _ = F.tree.node(lvl, i)
    if e <= a_h:
        return F.Ut[(lvl, i)][s - a_s:e - a_s]
    return F.Vt[(lvl, i)][s - a_h:e - a_h]


def _ancestor(tree, lvl, s):
    """Index of the node at level lvl containing row s."""
    b = tree.bounds[lvl]
    return int(np.searchsorted(b, s, side="right") - 1)


def factorize(H: HMat) -> Factor:
    t = H.tree
    F = Factor(t)
    logdet = 0.0
    # 1. leaf Cholesky factors
    for D in H.leaves:
        Li = _chol(D)
        F.Lleaf.append(Li)
        logdet += 2.0 * np.sum(np.log(np.diag(Li)))
    # 2. apply blkdiag(L_i)^-1 to every off-diagonal basis
    for key in H.U:
        F.Ut[key] = H.U[key].copy()
        F.Vt[key] = H.V[key].copy()
    for (s, e), Li in zip(t.leaves(), F.Lleaf):
        for lvl in range(t.L):
            i = _ancestor(t, lvl, s)
            rows = _basis_rows_in(F, lvl, i, s, e)
            if rows.shape[1]:
                rows[:] = solve_triangular(Li, rows, lower=True)
    # 3. levels L-1 .. 0
    for lvl in range(t.L - 1, -1, -1):
        for i in range(1 << lvl):
            s, h, e = t.node(lvl, i)
            Ub, Vb = F.Ut[(lvl, i)], F.Vt[(lvl, i)]
            r = Ub.shape[1]
            if r == 0:
                F.Y[(lvl, i)] = np.zeros((0, 0))
                F.Yinv[(lvl, i)] = np.zeros((0, 0))
                continue
            QU, RU = _qr_pos(Ub)
            QV, RV = _qr_pos(Vb)
            Cm = RU @ RV.T
            S = np.eye(2 * r)
            S[:r, r:] = Cm
            S[r:, :r] = Cm.T
            LS = _chol(S)
            logdet += 2.0 * np.sum(np.log(np.diag(LS)))
            I2 = np.eye(2 * r)
            LSinv = solve_triangular(LS, I2, lower=True)
            F.Ut[(lvl, i)], F.Vt[(lvl, i)] = QU, QV
            Ub, Vb = QU, QV
            Y, Yi = LS - I2, LSinv - I2
            F.Y[(lvl, i)], F.Yinv[(lvl, i)] = Y, Yi
            # inverse node factor applied to every ancestor basis on this node's rows
            for anc in range(lvl):
                a = _ancestor(t, anc, s)
                B = _basis_rows_in(F, anc, a, s, e)
                if B.shape[1] == 0:
                    continue
                P = np.concatenate([Ub.T @ B[:h - s], Vb.T @ B[h - s:]], axis=0)
                T = Yi @ P
                B[:h - s] += Ub @ T[:r]
                B[h - s:] += Vb @ T[r:]
    F.logdet = logdet
    return F


def _apply_node(F, lvl, i, v, Ym):
    s, h, e = F.tree.node(lvl, i)
    Ub, Vb = F.Ut[(lvl, i)], F.Vt[(lvl, i)]
    r = Ub.shape[1]
    if r == 0:
        return
    p = np.concatenate([Ub.T @ v[s:h], Vb.T @ v[h:e]], axis=0)
    t = Ym @ p
    v[s:h] += Ub @ t[:r]
    v[h:e] += Vb @ t[r:]


def apply_W(F: Factor, b, trans=False, inverse=False):
    """W b, W^T b, W^-1 b or W^-T b for W = A_L A_{L-1} ... A_0."""
    t = F.tree
    b = np.asarray(b, dtype=np.float64)
    squeeze = b.ndim == 1
    v = b.reshape(t.n, -1).copy()
    leaves = list(zip(t.leaves(), F.Lleaf))
    top_down = range(t.L)
    bottom_up = range(t.L - 1, -1, -1)
    if not trans and not inverse:
        for lvl in top_down:
            for i in range(1 << lvl):
                _apply_node(F, lvl, i, v, F.Y[(lvl, i)])
        for (s, e), Li in leaves:
            v[s:e] = Li @ v[s:e]
    elif inverse and not trans:
        for (s, e), Li in leaves:
            v[s:e] = solve_triangular(Li, v[s:e], lower=True)
        for lvl in bottom_up:
            for i in range(1 << lvl):
                _apply_node(F, lvl, i, v, F.Yinv[(lvl, i)])
    elif trans and not inverse:
        for (s, e), Li in leaves:
            v[s:e] = Li.T @ v[s:e]
        for lvl in bottom_up:
            for i in range(1 << lvl):
                _apply_node(F, lvl, i, v, F.Y[(lvl, i)].T)
    else:
        for lvl in top_down:
            for i in range(1 << lvl):
                _apply_node(F, lvl, i, v, F.Yinv[(lvl, i)].T)
        for (s, e), Li in leaves:
            v[s:e] = solve_triangular(Li, v[s:e], lower=True, trans="T")
    return v[:, 0] if squeeze else v


def solve(F: Factor, b):
    """x = A^-1 b = W^-T (W^-1 b)."""
    return apply_W(F, apply_W(F, b, inverse=True), trans=True, inverse=True)
