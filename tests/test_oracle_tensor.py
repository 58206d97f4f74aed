"""Pins of oracle/tensor.py (tensor product of 1-D GPs, Sec. 4.2).

* d = 1: the block update of f_1 is Algorithm 1 (the pinned oracle draw) on
  the data y / beta - 1 with noise variance sigma2 / beta^2 and tau2 = 1, for
  the same normals;
* d = 2, block h: the draw is affine in its normals; its mean and covariance
  equal the dense Gaussian conditional of f_h given y with the other factor
  fixed, written without any division by the products:
  y = G f_h + e, G = diag(beta prod_{k != h} f_k), f_h ~ N(1, C~_h):
  mean 1 + C~ G (G C~ G + sigma2 I)^-1 (y - G 1),
  cov C~ - C~ G (G C~ G + sigma2 I)^-1 G C~;
* beta | y: the conjugate form against the joint Gaussian of (beta, y)
  conditioned by its Schur complement;
* a short chain on a product surface recovers the noise variance.

Tolerances: 8 kappa u relative to the magnitudes involved (kappa of the
matrix that is solved with), as for the other oracle pins.
"""
import math

import numpy as np
import pytest

from oracle import hodlr
from oracle.factor import factorize
from oracle.hetero import draw_f_hetero
from oracle.sampler import Opts, Prior, draw_f
from oracle.tensor import BetaPrior, beta_conditional, block_data, products, tensor_init, tensor_sweep
from paper_2006_06537_gb300.inputs import tensor2, uniform_sine

U = np.finfo(np.float64).eps / 2
OPTS = Opts(B=16, eps=1e-12, cap=32, kind=0, nugget=1e-6)


def test_d1_block_is_algorithm_1():
    x, y = uniform_sine(96, 9)
    st = tensor_init(x[:, None], y, 0.15, OPTS, sigma2=0.02, beta=1.7)
    st.F[:, 0] = 1.0 + 0.1 * np.sin(3 * x)  # any current state: block 0 ignores its own f
    yt, dd = block_data(st, y, 0)
    b = st.blocks[0]
    n = len(x)
    g = np.random.default_rng(1)
    a0, b0 = g.standard_normal(n), g.standard_normal(n)
    f_h, _ = draw_f_hetero(b["HC"], b["FC"], yt, 1.0, dd, a0, b0)
    s2 = st.sigma2 / st.beta ** 2
    FM = factorize(hodlr.shift_scale(b["HC"], 1.0 / s2))
    ys = (y / st.beta - 1.0)[b["perm"]]
    f_1, mean_1 = draw_f(b["HC"], b["FC"], FM, ys, 1.0, s2, a0, b0)
    kappa = np.linalg.cond(hodlr.dense(b["HC"]) / s2 + np.eye(n))
    assert np.linalg.norm(f_h - f_1) <= 8 * kappa * U * (np.linalg.norm(f_1) + np.linalg.norm(mean_1))


def test_d2_block_conditional_is_the_dense_gaussian_conditional():
    X, y = tensor2(64, 2)
    st = tensor_init(X, y, 0.2, OPTS, sigma2=0.01, beta=1.3)
    st.F[:, 1] = 1.0 + 0.3 * np.cos(2 * math.pi * X[:, 1])
    h = 0
    b = st.blocks[h]
    n = len(y)
    yt, dd = block_data(st, y, h)
    zero = np.zeros(n)
    mean, _ = draw_f_hetero(b["HC"], b["FC"], yt, 1.0, dd, zero, zero)
    A1, A2 = np.empty((n, n)), np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A1[:, j] = draw_f_hetero(b["HC"], b["FC"], yt, 1.0, dd, e, zero)[0] - mean
        A2[:, j] = draw_f_hetero(b["HC"], b["FC"], yt, 1.0, dd, zero, e)[0] - mean
    cov = A1 @ A1.T + A2 @ A2.T
    # dense conditional in the sorted order of x_h, no division by the products
    perm = b["perm"]
    Gd = st.beta * st.F[perm, 1]
    C = hodlr.dense(b["HC"])
    S = Gd[:, None] * C * Gd[None, :] + st.sigma2 * np.eye(n)
    mu_ref = 1.0 + C @ (Gd * np.linalg.solve(S, y[perm] - Gd))
    cov_ref = C - C @ (Gd[:, None] * np.linalg.solve(S, Gd[:, None] * C))
    tol = 8 * max(np.linalg.cond(S), np.linalg.cond(C)) * U
    assert np.linalg.norm((1.0 + mean) - mu_ref) <= tol * np.linalg.norm(C) * np.linalg.norm(np.linalg.solve(S, y[perm]))
    assert np.linalg.norm(cov - cov_ref) <= tol * np.linalg.norm(C) * math.sqrt(n)


def test_beta_conditional_against_joint_gaussian():
    g = np.random.default_rng(4)
    n = 50
    G = 1.0 + 0.5 * g.standard_normal(n)
    y = 1.8 * G + 0.1 * g.standard_normal(n)
    pr = BetaPrior(mu=0.7, sd=1.4)
    s2 = 0.01
    m, v = beta_conditional(G, y, s2, pr)
    Syy = pr.sd ** 2 * np.outer(G, G) + s2 * np.eye(n)
    sby = pr.sd ** 2 * G
    m_ref = pr.mu + sby @ np.linalg.solve(Syy, y - pr.mu * G)
    v_ref = pr.sd ** 2 - sby @ np.linalg.solve(Syy, sby)
    tol = 8 * np.linalg.cond(Syy) * U
    assert abs(m - m_ref) <= tol * (abs(m_ref) + 1)
    assert abs(v - v_ref) <= tol * pr.sd ** 2


def test_short_chain_recovers_noise():
    X, y = tensor2(256, 3, noise=0.05)
    st = tensor_init(X, y, 0.2, OPTS, sigma2=0.05, beta=1.0)
    pr = Prior(a_sigma2=1.0, b_sigma2=1e-4, logrho_mu=math.log(0.2))
    s2 = []
    for _ in range(12):
        tensor_sweep(st, y, pr, BetaPrior(mu=1.0, sd=2.0), OPTS, seed=11)
        s2.append(st.sigma2)
    assert np.all(np.isfinite(s2))
    assert 0.5 * 0.05 ** 2 < np.median(s2[-6:]) < 3.0 * 0.05 ** 2
    fit = st.beta * products(st.F)
    assert np.sqrt(np.mean((fit - y) ** 2)) < 0.1
