"""Pins of oracle/hetero.py (Algorithm 1.h) by routes other than its own steps.

* equal precisions d_i = 1/sigma2: Algorithm 1.h reduces to Algorithm 1 (the
  pinned oracle draw) for the same normals (a = a0 / sigma);
* the lemma after Algorithm 1.h: the draw is affine in the normals, so its
  mean (normals zero) must be K~ P~^-1 y and its covariance, assembled from the
  draws of unit normals, must be K~ P~^-1 D^-1, both formed densely;
* add_diagonal: the dense matrix of s C~ + diag(d) entry by entry.

Tolerances: 8 kappa u relative to the magnitudes involved (kappa of the dense
P~ or M~), the bound two correct FP64 routes through an ill-conditioned solve
share.
"""
import math

import numpy as np
import pytest

from oracle import detmath, hodlr
from oracle.factor import factorize
from oracle.hetero import add_diagonal, draw_f_hetero
from oracle.sampler import draw_f
from paper_2006_06537_gb300.inputs import uniform_sine

U = np.finfo(np.float64).eps / 2


def _setup(n=96, B=16, rho=0.15, nug=1e-6, seed=5):
    x, y = uniform_sine(n, seed)
    c = detmath.kernel_const(0, rho)
    HC = hodlr.assemble(x, B, 0, c, nug, 1e-12, 32)
    return x, y, HC, factorize(HC)


def test_add_diagonal_matches_dense():
    x, y, HC, _ = _setup()
    d = np.random.default_rng(1).uniform(0.5, 2.0, len(x))
    P = add_diagonal(HC, 3.0, d)
    want = 3.0 * hodlr.dense(HC) + np.diag(d)
    np.testing.assert_allclose(hodlr.dense(P), want, rtol=1e-15, atol=1e-15)


def test_equal_precisions_reduce_to_algorithm_1():
    x, y, HC, FC = _setup()
    tau2, sigma2 = 0.8, 0.05
    n = len(x)
    g = np.random.default_rng(2)
    a0, b = g.standard_normal(n), g.standard_normal(n)
    f_h, R = draw_f_hetero(HC, FC, y, tau2, np.full(n, 1.0 / sigma2), a0, b)
    FM = factorize(hodlr.shift_scale(HC, tau2 / sigma2))
    f_1, mean_1 = draw_f(HC, FC, FM, y, tau2, sigma2, a0, b)
    kappa = np.linalg.cond(tau2 / sigma2 * hodlr.dense(HC) + np.eye(n))
    tol = 8 * kappa * U
    assert np.linalg.norm(f_h - f_1) <= tol * (np.linalg.norm(f_1) + np.linalg.norm(mean_1))
    assert np.linalg.norm(R - mean_1) <= tol * np.linalg.norm(mean_1)


def test_lemma_mean_and_covariance():
    x, y, HC, FC = _setup(n=64)
    n = len(x)
    tau2 = 1.7
    d = np.random.default_rng(3).uniform(5.0, 80.0, n)  # heteroskedastic precisions
    zero = np.zeros(n)
    mean, R = draw_f_hetero(HC, FC, y, tau2, d, zero, zero)
    K = tau2 * hodlr.dense(HC)
    P = K + np.diag(1.0 / d)
    mu = K @ np.linalg.solve(P, y)
    Sigma = K @ np.linalg.solve(P, np.diag(1.0 / d))
    tol = 8 * np.linalg.cond(P) * U
    assert np.linalg.norm(mean - mu) <= tol * np.linalg.norm(K) * np.linalg.norm(np.linalg.solve(P, y))
    assert np.array_equal(mean, R)
    # the draw is affine in (a0, b): columns of its two linear maps from unit normals
    A1 = np.empty((n, n))
    A2 = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A1[:, j] = draw_f_hetero(HC, FC, y, tau2, d, e, zero)[0] - mean
        A2[:, j] = draw_f_hetero(HC, FC, y, tau2, d, zero, e)[0] - mean
    cov = A1 @ A1.T + A2 @ A2.T
    scale = np.linalg.norm(K, 2) * np.linalg.norm(np.linalg.inv(P), 2) * np.max(1.0 / d) * math.sqrt(n)
    assert np.linalg.norm(cov - Sigma) <= tol * scale
