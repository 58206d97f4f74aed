"""Exact dense Gaussian-process quantities (oracle side, small n only).

* Eq. (gp_posterior): Sigma_f = K (tau K + I)^-1 = K - K (K + tau^-1 I)^-1 K,
  mu_f = tau Sigma_f y; here tau = 1/sigma2 and K = tau2 (C + nugget I).
* Eqs. (posterior_gibs2)-(posterior_gibs3): conjugate conditionals of the two
  variances, written as inverse-gamma parameters (shape, scale).
* Log density of eta = log rho given f (Eq. (posterior_gibs4) with a normal
  prior on eta instead of the discrete grid).
* KL divergence of the proof of Theorem 4.1, Eq. (big_KL_pts1to3): for
  P = N(mu_P, S_P), Q = N(mu_Q, S_Q),
  KL(P||Q) = 1/2 [ log det S_Q / det S_P + tr(S_Q^-1 S_P) - n
                   + (mu_Q - mu_P)^T S_Q^-1 (mu_Q - mu_P) ].
"""
from __future__ import annotations

import numpy as np


def posterior(K, y, sigma2):
    """Exact (mean, covariance) of f | y for prior covariance K and noise variance sigma2."""
    n = K.shape[0]
    M = K / sigma2 + np.eye(n)
    Sigma = np.linalg.solve(M, K)  # M^-1 K = K M^-1 (the two commute)
    Sigma = 0.5 * (Sigma + Sigma.T)
    mean = Sigma @ (np.asarray(y) / sigma2)
    return mean, Sigma


def posterior_alt(K, y, sigma2):
    """Same posterior through the first form of Eq. (gp_posterior): K - K (K + sigma2 I)^-1 K."""
    n = K.shape[0]
    A = K + sigma2 * np.eye(n)
    Sigma = K - K @ np.linalg.solve(A, K)
    mean = K @ np.linalg.solve(A, np.asarray(y))
    return mean, 0.5 * (Sigma + Sigma.T)


def sigma2_conditional(y, f, a, b):
    """IG(shape, scale) of sigma2 | y, f."""
    r = np.asarray(y) - np.asarray(f)
    return a + 0.5 * len(r), b + 0.5 * float(r @ r)


def tau2_conditional(C, f, a, b):
    """IG(shape, scale) of tau2 | f for f ~ N(0, tau2 C)."""
    f = np.asarray(f)
    q = float(f @ np.linalg.solve(C, f))
    return a + 0.5 * len(f), b + 0.5 * q


def log_density_eta(C, f, tau2):
    """log N(f; 0, tau2 C) up to the constant -n/2 log(2 pi)."""
    sign, ld = np.linalg.slogdet(tau2 * C)
    if sign <= 0:
        return -np.inf
    f = np.asarray(f)
    return -0.5 * ld - 0.5 * float(f @ np.linalg.solve(tau2 * C, f))


def kl_gauss(mu_p, S_p, mu_q, S_q):
    n = len(mu_p)
    s1, ld_q = np.linalg.slogdet(S_q)
    s2, ld_p = np.linalg.slogdet(S_p)
    d = np.asarray(mu_q) - np.asarray(mu_p)
    tr = np.trace(np.linalg.solve(S_q, S_p))
    quad = float(d @ np.linalg.solve(S_q, d))
    return 0.5 * ((ld_q - ld_p) + tr - n + quad), dict(logdet=ld_q - ld_p, trace=tr - n, quad=quad)
