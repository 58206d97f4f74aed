"""Exact O(n) Gaussian-process quantities for the Matern-5/2 kernel in 1-D
(oracle side, test infrastructure): an independent pin for large n.

Not from the paper: the Matern-5/2 process on a line is the first coordinate
of a 3-state linear stochastic differential equation (Hartikainen & Sarkka,
"Kalman filtering and smoothing solutions to temporal Gaussian process
regression models", 2010),

    ds = F s dt + L dbeta,   F = [[0, 1, 0], [0, 0, 1], [-lam^3, -3 lam^2, -3 lam]],
    L = [0, 0, 1]^T,  spectral density q = (16/3) var lam^5,  lam = sqrt(5) / rho,

whose stationary covariance P_inf solves F P + P F^T + L q L^T = 0, so that
f(x) = s_0(x) has covariance var (1 + lam d + lam^2 d^2 / 3) exp(-lam d).  At
sorted inputs the states form a Markov chain with transition A = expm(F d)
and noise Q = int_0^d expm(F t) L q L^T expm(F t)^T dt (Van Loan's block
exponential, accurate for the tiny gaps of dense inputs, where
P_inf - A P_inf A^T cancels).  A Kalman filter on y = f + e, e ~ N(0, noise I)
then gives, through its innovations v_i and their variances S_i,

    log det(var C + noise I) = sum_i log S_i,   y^T (var C + noise I)^-1 y = sum_i v_i^2 / S_i,

and the modified Bryson-Frazier backward pass (no inverse of a predicted
covariance) gives the smoothed mean E[f | y] = var C (var C + noise I)^-1 y,
all in O(n) for C the unit-variance Matern-5/2 correlation matrix.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


def matern52_sde(rho: float, var: float):
    """(F, G = L q L^T, P_inf) of the Matern-5/2 state-space model."""
    lam = math.sqrt(5.0) / rho
    F = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [-lam ** 3, -3.0 * lam ** 2, -3.0 * lam]])
    G = np.zeros((3, 3))
    G[2, 2] = 16.0 / 3.0 * var * lam ** 5
    Pinf = sla.solve_continuous_lyapunov(F, -G)
    return F, G, 0.5 * (Pinf + Pinf.T)


def discretize(F, G, d):
    """(A, Q) for every gap in d (arrays of shape (len(d), 3, 3)) by Van Loan's
    method: expm([[F, G], [0, -F^T]] d) = [[A, E12], [0, A^-T]], Q = E12 A^T."""
    d = np.asarray(d, dtype=np.float64)
    blk = np.zeros((6, 6))
    blk[:3, :3] = F
    blk[:3, 3:] = G
    blk[3:, 3:] = -F.T
    Ms = d[:, None, None] * blk[None, :, :]
    try:
        E = sla.expm(Ms)
    except ValueError:  # an older scipy without stacked matrices
        E = np.stack([sla.expm(m) for m in Ms])
    A = E[:, :3, :3]
    Q = np.einsum("nij,nkj->nik", E[:, :3, 3:], A)
    return A, 0.5 * (Q + np.transpose(Q, (0, 2, 1)))


def kalman(x, y, rho: float, var: float, noise: float):
    """Kalman filter and modified Bryson-Frazier smoother for y = f + e with
    f ~ GP(0, var C_matern52(rho)) at sorted x and e ~ N(0, noise I).
    Returns (log det(var C + noise I), y^T (var C + noise I)^-1 y, E[f | y])."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = len(x)
    F, G, Pinf = matern52_sde(rho, var)
    A, Q = discretize(F, G, np.diff(x))
    mp = np.zeros((n, 3))      # predicted means and covariances
    Pp = np.zeros((n, 3, 3))
    v = np.zeros(n)            # innovations
    S = np.zeros(n)            # their variances
    K = np.zeros((n, 3))       # gains
    m = np.zeros(3)
    P = Pinf.copy()
    for i in range(n):
        if i > 0:
            m = A[i - 1] @ m
            P = A[i - 1] @ P @ A[i - 1].T + Q[i - 1]
        mp[i] = m
        Pp[i] = P
        S[i] = P[0, 0] + noise
        v[i] = y[i] - m[0]
        K[i] = P[:, 0] / S[i]
        m = m + K[i] * v[i]
        P = P - np.outer(K[i], P[0, :])
        P = 0.5 * (P + P.T)
    logdet = float(np.sum(np.log(S)))
    quad = float(np.sum(v * v / S))
    # backward pass: lam_i = H^T v_i / S_i + (I - K_i H)^T A_i^T lam_{i+1};  m_s = m_p + P_p lam
    mean = np.zeros(n)
    lam_next = np.zeros(3)  # A_i^T lam_{i+1}, zero past the last point
    for i in range(n - 1, -1, -1):
        t = lam_next - np.array([K[i] @ lam_next, 0.0, 0.0])  # (I - K H)^T u = u - H^T (K^T u)
        t[0] += v[i] / S[i]
        mean[i] = mp[i][0] + Pp[i][0] @ t
        lam_next = A[i - 1].T @ t if i > 0 else lam_next
    return logdet, quad, mean
