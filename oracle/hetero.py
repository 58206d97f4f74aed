"""Algorithm 1.h: the draw of f | y under heteroskedastic noise (oracle side;
test infrastructure only).

Appendix "Heteroskedastic noise derivation": noise e_i ~ N(0, 1/d_i), with
D = diag(d) the precisions.  With K~ = tau2 C~ (W W^T = K~, W = sqrt(tau2) W_C)
and P~ = K~ + D^-1 (the same H-matrix with D^-1 added on its diagonal):

    a ~ N(0, D), b ~ N(0, I)   (a = sqrt(d) a0 for a standard normal a0)
    Z    = K~ a + W b
    Z*   = P~^-1 Z
    Z**  = D^-1 Z*
    R    = K~ P~^-1 y
    f    = R + Z**

and, by the lemma that follows the algorithm, f ~ N(K~ P~^-1 y, K~ P~^-1 D^-1).
The standard normals a0, b are inputs.  P~ is factored by the same HODLR
factorization as C~ (Ambikasaran et al., Thm 3.1).
"""
from __future__ import annotations

import math

import numpy as np

from .factor import apply_W, factorize, solve
from .hodlr import HMat, matvec


def add_diagonal(H: HMat, s: float, diag) -> HMat:
    """s * C~ + diag(diag): leaves s*D_i + diag, U -> s*U, V unchanged."""
    diag = np.asarray(diag, dtype=np.float64)
    P = HMat(H.tree)
    for (s0, e0), D in zip(H.tree.leaves(), H.leaves):
        Dp = s * D
        Dp[np.diag_indices(e0 - s0)] += diag[s0:e0]
        P.leaves.append(Dp)
    for key in H.U:
        P.U[key] = s * H.U[key]
        P.V[key] = H.V[key].copy()
        P.row_piv[key], P.col_piv[key] = H.row_piv[key], H.col_piv[key]
        P.hit_cap[key] = H.hit_cap[key]
    return P


def draw_f_hetero(HC: HMat, FC, y, tau2: float, d, a0, b):
    """Algorithm 1.h with given standard normals a0, b. Returns (f, R = K~ P~^-1 y)."""
    d = np.asarray(d, dtype=np.float64)
    a = np.sqrt(d) * np.asarray(a0, dtype=np.float64)
    Z = tau2 * matvec(HC, a) + math.sqrt(tau2) * apply_W(FC, b)
    FP = factorize(add_diagonal(HC, tau2, 1.0 / d))
    Zs = solve(FP, Z)
    Zss = Zs / d
    R = tau2 * matvec(HC, solve(FP, np.asarray(y, dtype=np.float64)))
    return R + Zss, R
