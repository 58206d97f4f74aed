"""Shared helpers for the GPU parity tests (device buffers, oracle set-up)."""
import numpy as np

from oracle import detmath, factor, hodlr


def build_lib():
    from paper_2006_06537_gb300 import build

    return build.build()


def dev(a, torch):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_hmat(x, B, kind, rho, nugget, eps, cap):
    return hodlr.assemble(x, B, kind, detmath.kernel_const(kind, rho), nugget, eps, cap)


def oracle_bases(H, n, cap):
    """The oracle's U / V in the library's level-major export layout."""
    L = H.tree.L
    out = np.zeros((max(1, L), cap, n))
    for lvl in range(L):
        for i in range(1 << lvl):
            s, h, e = H.tree.node(lvl, i)
            U, V = H.U[(lvl, i)], H.V[(lvl, i)]
            out[lvl, :U.shape[1], s:h] = U.T
            out[lvl, :V.shape[1], h:e] = V.T
    return out


def used_mask(ranks, tree, cap):
    """Boolean mask of the export layout entries that hold basis data."""
    n, L = tree.n, tree.L
    m = np.zeros((max(1, L), cap, n), bool)
    for lvl in range(L):
        for i in range(1 << lvl):
            s, h, e = tree.node(lvl, i)
            r = ranks[(1 << lvl) - 1 + i]
            m[lvl, :r, s:e] = True
    return m


def oracle_factor(H):
    return factor.factorize(H)
