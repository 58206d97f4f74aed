"""Pins of the Matern-5/2 state-space oracle (oracle/statespace.py), the exact
O(n) reference used at n = 131072 where dense algebra is out of reach.

Against the kernel itself: P_inf holds the covariance function's derivatives
at zero, and the discretised chain reproduces the covariance k(d) at every
gap.  Against dense linear algebra at n = 300: the innovations' log det and
quadratic form and the smoothed mean, for a well- and an ill-conditioned noise
level.  A wrong spectral density, a transposed transition or a dropped term of
the backward pass fails one of these.
"""
import math

import numpy as np
import pytest

from oracle import statespace as ss


def _kern(d, rho, var):
    lam = math.sqrt(5.0) / rho
    d = np.abs(d)
    return var * (1.0 + lam * d + (lam * d) ** 2 / 3.0) * np.exp(-lam * d)


@pytest.mark.parametrize("rho,var", [(0.05, 1.0), (0.3, 2.5)])
def test_stationary_covariance_is_the_kernel_derivatives(rho, var):
    lam = math.sqrt(5.0) / rho
    F, G, P = ss.matern52_sde(rho, var)
    # Cov(f, f) = k(0), Cov(f', f') = -k''(0), Cov(f'', f'') = k''''(0), Cov(f, f'') = k''(0)
    k2 = -var * lam ** 2 / 3.0
    k4 = var * lam ** 4
    want = np.array([[var, 0.0, k2], [0.0, -k2, 0.0], [k2, 0.0, k4]])
    assert np.allclose(P, want, rtol=1e-10, atol=1e-10 * k4)
    assert np.abs(F @ P + P @ F.T + G).max() <= 1e-9 * np.abs(G).max()


@pytest.mark.parametrize("rho", [0.05, 0.3])
def test_discrete_chain_reproduces_the_covariance_function(rho):
    F, G, P = ss.matern52_sde(rho, 1.7)
    d = np.concatenate([[1e-7, 1e-5, 1e-3], np.linspace(0.01, 5.0, 40) * rho])
    A, Q = ss.discretize(F, G, d)
    cov = A[:, 0, :] @ P[:, 0]  # Cov(f(t + d), f(t)) = [A(d) P_inf]_00
    assert np.allclose(cov, _kern(d, rho, 1.7), rtol=1e-11, atol=1e-13)
    # the process noise keeps the chain stationary: A P A^T + Q = P (checked where it does not cancel)
    big = d > 0.1 * rho
    assert np.allclose(np.einsum("nij,jk,nlk->nil", A[big], P, A[big]) + Q[big], P[None], rtol=1e-9,
                       atol=1e-9 * np.abs(P).max())
    # and for tiny gaps Q is positive semidefinite with the analytic leading order q d^5 / 20 in its (0, 0) entry
    for k in range(3):
        assert np.linalg.eigvalsh(Q[k]).min() >= -1e-12 * np.abs(Q[k]).max()
    q = G[2, 2]
    assert Q[0, 0, 0] == pytest.approx(q * d[0] ** 5 / 20.0, rel=1e-4)


@pytest.mark.parametrize("noise", [0.04, 1e-4])
def test_kalman_matches_dense_algebra(noise):
    g = np.random.default_rng(3)
    n, rho, var = 300, 0.05, 1.3
    x = np.sort(g.uniform(0.0, 1.0, n))
    y = g.standard_normal(n)
    Cm = _kern(x[:, None] - x[None, :], rho, 1.0)
    M = var * Cm + noise * np.eye(n)
    L = np.linalg.cholesky(M)
    ld = 2.0 * np.sum(np.log(np.diag(L)))
    a = np.linalg.solve(M, y)
    kappa = np.linalg.cond(M)
    logdet, quad, mean = ss.kalman(x, y, rho, var, noise)
    tol = max(1e-12, 16 * kappa * 1.1e-16)
    assert abs(logdet - ld) <= tol * abs(ld)
    assert abs(quad - y @ a) <= tol * abs(y @ a)
    ref = var * Cm @ a
    assert np.linalg.norm(mean - ref) <= tol * np.linalg.norm(ref)
