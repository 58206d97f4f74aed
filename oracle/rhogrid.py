"""Length-scale on a discrete grid, Eq. (posterior_gibs4) (oracle side; test
infrastructure only).

With a uniform prior over the grid {s_1, ..., s_r} and K_h = tau2 C~(s_h),

    Pr(rho = s_h | -) = c det(K_h)^-1/2 exp(-f^T K_h^-1 f / 2),

so with the factors W_h W_h^T = C~(s_h) computed once per grid point,
log w_h = -logdet C~_h / 2 - ||W_h^-1 f||^2 / (2 tau2) + const (the common
-n log(tau2) / 2 cancels in c).  The draw takes a uniform u in [0, 1): the
smallest h whose cumulative probability exceeds u.  A non-uniform prior adds
its log weights.
"""
from __future__ import annotations

import numpy as np

from .factor import Factor, apply_W


def grid_terms(factors, f):
    """(logdet C~_h, f^T C~_h^-1 f) for every grid factor."""
    f = np.asarray(f, dtype=np.float64)
    logdets = np.array([F.logdet for F in factors])
    quads = np.array([float(np.sum(apply_W(F, f, inverse=True) ** 2)) for F in factors])
    return logdets, quads


def grid_logw(logdets, quads, tau2: float, log_prior=None):
    """Unnormalised log Pr(rho = s_h | f, tau2), up to the constant common to all h."""
    lw = -0.5 * np.asarray(logdets, dtype=np.float64) - 0.5 * np.asarray(quads, dtype=np.float64) / tau2
    if log_prior is not None:
        lw = lw + np.asarray(log_prior, dtype=np.float64)
    return lw


def grid_probs(logdets, quads, tau2: float, log_prior=None):
    """Normalised Pr(rho = s_h | f, tau2) from the per-point log-determinants and quadratic forms."""
    lw = grid_logw(logdets, quads, tau2, log_prior)
    lw = lw - np.max(lw)
    w = np.exp(lw)
    return w / np.sum(w)


def grid_draw(probs, u: float) -> int:
    """Index h = min{h : sum_{l <= h} p_l > u} for u in [0, 1)."""
    cdf = np.cumsum(np.asarray(probs, dtype=np.float64))
    h = int(np.searchsorted(cdf, u, side="right"))
    return min(h, len(cdf) - 1)


def grid_step(factors: list[Factor], f, tau2: float, u: float, log_prior=None):
    """One draw of the grid index given f, tau2 and a uniform u; returns (index, probabilities)."""
    logdets, quads = grid_terms(factors, f)
    p = grid_probs(logdets, quads, tau2, log_prior)
    return grid_draw(p, u), p
