"""Partial-pivoted cross approximation of one off-diagonal block (oracle side).

The paper compresses each off-diagonal block A = C(I, J) by "partial-pivoted
LU" (proof of Lemma 1) to a max-norm tolerance that holds by construction
(Sec. 3.2).  This is adaptive cross approximation with partial pivoting; the
steps below fix every choice the paper leaves open (start row, ties, stopping),
so that the GPU reproduces the same pivots bit for bit:

    i = m - 1                      (the row nearest the partner block)
    for k = 0, 1, ... while k < cap:
        rho_j  = A[i, j] - sum_{l<k} U[i, l] V[j, l]      for every column j
        j*     = argmax over unused columns of |rho_j|    (lowest j on ties)
        if rho_j* == 0 (or every column is used): stop
        v      = rho * (1 / rho_j*)         (one IEEE division, then products)
        u_i'   = A[i', j*] - sum_{l<k} U[i', l] V[j*, l]  for every row i'
        if max |u| <= eps: stop (this term is not kept)
        keep U[:, k] = u, V[:, k] = v; mark row i and column j* used
        i      = argmax over unused rows of |u_i'|        (lowest i on ties)
    if no unused row remains the loop ends.

Every sum above is accumulated from l = 0 upward as acc = fma(-U, V, acc):
acc - U * V with one rounding (IEEE fused multiply-add, `oracle/fmath.py`).
Since |v| <= 1 (up to one rounding of the reciprocal and one of the product,
|v| <= 1 + 2**-51) with v_j* within that of 1, max|u| * max|v| = max|u| is the
size of the new term, the max-norm estimate of the remaining error.
"""
from __future__ import annotations

import numpy as np

from .detmath import kernel_entries
from .fmath import fma


def aca_entries(row_fn, col_fn, m, p, eps, cap):
    """ACA of an m x p block given row_fn(i) -> A[i, :] and col_fn(j) -> A[:, j].

    Returns (U, V, row_pivots, col_pivots, hit_cap)."""
    rows, cols = [], []
    row_used = np.zeros(m, dtype=bool)
    col_used = np.zeros(p, dtype=bool)
    Ucols, Vcols = [], []
    i = m - 1
    hit_cap = False
    k = 0
    while m > 0 and p > 0:
        if k == cap:
            hit_cap = True
            break
        rho = np.array(row_fn(i), dtype=np.float64)
        for l in range(k):
            rho = fma(-Ucols[l][i], Vcols[l], rho)
        a = np.where(col_used, -1.0, np.abs(rho))
        j = int(np.argmax(a))  # first maximal index
        if a[j] <= 0.0:
            break
        v = rho * (1.0 / rho[j])
        u = np.array(col_fn(j), dtype=np.float64)
        for l in range(k):
            u = fma(-Ucols[l], Vcols[l][j], u)
        if np.max(np.abs(u)) <= eps:
            break
        Ucols.append(u)
        Vcols.append(v)
        rows.append(i)
        cols.append(j)
        row_used[i] = True
        col_used[j] = True
        k += 1
        b = np.where(row_used, -1.0, np.abs(u))
        inext = int(np.argmax(b))
        if b[inext] < 0.0:
            break
        i = inext
    U = np.stack(Ucols, axis=1) if k else np.zeros((m, 0))
    V = np.stack(Vcols, axis=1) if k else np.zeros((p, 0))
    return U, V, rows, cols, hit_cap


def aca_block(kind, c, x_rows, x_cols, eps, cap):
    """ACA of the kernel block A[i, j] = k(x_rows[i], x_cols[j])."""
    return aca_entries(lambda i: kernel_entries(kind, c, x_rows[i], x_cols),
                       lambda j: kernel_entries(kind, c, x_rows, x_cols[j]),
                       len(x_rows), len(x_cols), eps, cap)
