"""Pins for the oracle's Algorithm 1 draw and Gibbs conditionals.

* Lemma 1: the draw is an affine map of the normals (a, b), so its exact
  covariance A_a A_a^T + A_b A_b^T is recovered column by column and compared
  with K~ M~^-1 formed densely; its mean with tau K~ M~^-1 y.
* The exact posterior of Eq. (gp_posterior) is recovered as eps -> 0.
* The sigma^2 / tau^2 conditional parameters and the Metropolis log ratio
  against dense closed forms.
* The KL divergence of the proof of Theorem 4.1: zero for identical laws, the
  1-D closed form, decreasing in eps and part (i) below 2 n^2 eps.
* A Monte-Carlo check of Philox-driven draws.
"""
import math

import numpy as np
import pytest

from oracle import dense, detmath, factor, hodlr, rng, sampler
from paper_2006_06537_gb300.inputs import uniform_sine


def _problem(n=48, B=12, eps=1e-12, nugget=1e-6, rho=0.15, kind=0):
    x, y = uniform_sine(n, 11)
    c = detmath.kernel_const(kind, rho)
    HC = hodlr.assemble(x, B, kind, c, nugget, eps, 64)
    return x, y, c, HC


def _linear_maps(HC, FC, FM, y, tau2, sigma2):
    n = HC.tree.n
    z = np.zeros(n)
    mean, _ = sampler.draw_f(HC, FC, FM, y, tau2, sigma2, z, z)
    Aa = np.empty((n, n))
    Ab = np.empty((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        Aa[:, i] = sampler.draw_f(HC, FC, FM, y, tau2, sigma2, e, z)[0] - mean
        Ab[:, i] = sampler.draw_f(HC, FC, FM, y, tau2, sigma2, z, e)[0] - mean
    return mean, Aa @ Aa.T + Ab @ Ab.T


def test_lemma1_exact_covariance_and_mean():
    x, y, c, HC = _problem()
    tau2, sigma2 = 1.3, 0.05
    FC = factor.factorize(HC)
    FM = factor.factorize(hodlr.shift_scale(HC, tau2 / sigma2))
    mean, cov = _linear_maps(HC, FC, FM, y, tau2, sigma2)
    Kt = tau2 * hodlr.dense(HC)
    Mt = hodlr.dense(hodlr.shift_scale(HC, tau2 / sigma2))
    Sig = Kt @ np.linalg.inv(Mt)
    np.testing.assert_allclose(cov, Sig, atol=1e-10 * np.abs(Sig).max())
    np.testing.assert_allclose(mean, Sig @ y / sigma2, atol=1e-10 * np.abs(mean).max())


def test_draw_law_approaches_exact_posterior():
    x, y, c, HC = _problem(eps=1e-14)
    tau2, sigma2 = 0.8, 0.02
    FC = factor.factorize(HC)
    FM = factor.factorize(hodlr.shift_scale(HC, tau2 / sigma2))
    mean, cov = _linear_maps(HC, FC, FM, y, tau2, sigma2)
    K = tau2 * hodlr.dense_kernel(x, 0, c, 1e-6)
    mu, Sig = dense.posterior(K, y, sigma2)
    mu2, Sig2 = dense.posterior_alt(K, y, sigma2)
    np.testing.assert_allclose(mu, mu2, atol=1e-9)
    np.testing.assert_allclose(Sig, Sig2, atol=1e-9)
    np.testing.assert_allclose(mean, mu, atol=1e-8)
    np.testing.assert_allclose(cov, Sig, atol=1e-8)


def test_kl_formula_and_theorem_bound():
    mu = np.array([0.3])
    S = np.array([[2.0]])
    mq = np.array([-0.1])
    Sq = np.array([[0.5]])
    kl, _ = dense.kl_gauss(mu, S, mq, Sq)
    ref = math.log(math.sqrt(0.5) / math.sqrt(2.0)) + (2.0 + 0.4 ** 2) / (2 * 0.5) - 0.5
    assert kl == pytest.approx(ref, rel=1e-14)
    assert dense.kl_gauss(mu, S, mu, S)[0] == pytest.approx(0.0, abs=1e-15)
    # P: exact posterior, Q: the HODLR approximation, Theorem 4.1
    n, tau2, sigma2 = 48, 1.0, 0.1
    kls = []
    for eps in (1e-4, 1e-7, 1e-10):
        x, y, c, HC = _problem(n=n, eps=eps, nugget=1e-4)
        K = tau2 * hodlr.dense_kernel(x, 0, c, 1e-4)
        mu_p, S_p = dense.posterior(K, y, sigma2)
        Kt = tau2 * hodlr.dense(HC)
        Mt = Kt / sigma2 + np.eye(n)
        S_q = Kt @ np.linalg.inv(Mt)
        S_q = 0.5 * (S_q + S_q.T)
        mu_q = S_q @ y / sigma2
        kl, parts = dense.kl_gauss(mu_p, S_p, mu_q, S_q)
        e_max = max(np.abs(Kt - K).max(), np.abs(Mt - (K / sigma2 + np.eye(n))).max())
        assert kl >= -1e-12
        assert abs(parts["logdet"]) <= 2 * n * n * e_max
        kls.append(kl)
    assert kls[0] > kls[1] > kls[2] or kls[2] < 1e-12


def test_gibbs_conditionals_match_dense():
    x, y, c, HC = _problem(n=64, B=16)
    f = np.sin(3 * x)
    a_s, b_s = dense.sigma2_conditional(y, f, 1.0, 1.0)
    assert a_s == 1.0 + 32 and b_s == pytest.approx(1.0 + 0.5 * np.sum((y - f) ** 2), rel=1e-15)
    FC = factor.factorize(HC)
    q = float(np.sum(factor.apply_W(FC, f, inverse=True) ** 2))
    C = hodlr.dense(HC)
    _, b_t = dense.tau2_conditional(C, f, 1.0, 1.0)
    assert 1.0 + 0.5 * q == pytest.approx(b_t, rel=1e-9)
    # Metropolis log ratio equals the dense log-density difference
    tau2 = 0.7
    c2 = detmath.kernel_const(0, 0.22)
    HC2 = hodlr.assemble(x, 16, 0, c2, 1e-6, 1e-12, 64)
    FC2 = factor.factorize(HC2)
    q2 = float(np.sum(factor.apply_W(FC2, f, inverse=True) ** 2))
    lr = -0.5 * (FC2.logdet - FC.logdet) - (q2 - q) / (2 * tau2)
    ref = dense.log_density_eta(hodlr.dense(HC2), f, tau2) - dense.log_density_eta(C, f, tau2)
    assert lr == pytest.approx(ref, rel=1e-8, abs=1e-8)


def test_philox_driven_draws_monte_carlo():
    x, y, c, HC = _problem(n=24, B=6)
    tau2, sigma2 = 1.0, 0.1
    FC = factor.factorize(HC)
    FM = factor.factorize(hodlr.shift_scale(HC, tau2 / sigma2))
    draws = np.array([sampler.draw_f(HC, FC, FM, y, tau2, sigma2,
                                     rng.normals(24, 3, rng.TAG_A, t, 0), rng.normals(24, 3, rng.TAG_B, t, 0))[0]
                      for t in range(3000)])
    Kt = tau2 * hodlr.dense(HC)
    Sig = Kt @ np.linalg.inv(Kt / sigma2 + np.eye(24))
    mu = Sig @ y / sigma2
    sd = np.sqrt(np.diag(Sig))
    assert np.all(np.abs(draws.mean(0) - mu) < 5 * sd / math.sqrt(3000))
    var_ratio = draws.var(0) / np.diag(Sig)
    assert np.all(np.abs(var_ratio - 1) < 5 * math.sqrt(2 / 3000))


def test_gibbs_chain_recovers_noise_level():
    x, y = uniform_sine(256, 0, noise=0.1)
    opts = sampler.Opts(B=32, eps=1e-10, cap=64, kind=0, nugget=1e-6)
    # a vague IG(1e-3, 1e-3) prior: with IG(1, 1) the prior scale (1) rivals rss/2 (~1.3)
    prior = sampler.Prior(a_sigma2=1e-3, b_sigma2=1e-3, logrho_mu=math.log(0.2))
    st = sampler.init_state(x, y, 0.2, opts)
    for _ in range(30):
        sampler.gibbs_step(st, x, y, prior, opts, seed=0, chain=0)
    s2 = np.array([t["sigma2"] for t in st.trace[10:]])
    assert 0.007 < np.median(s2) < 0.014
    assert any(t["accept"] for t in st.trace)


def test_additive_block_gibbs_recovers_components():
    # y = f_1(x_1) + f_2(x_2) + noise; the sweep must separate the two components
    g = np.random.default_rng(21)
    n = 400
    X = g.uniform(0, 1, (n, 2))
    f1, f2 = np.sin(2 * math.pi * X[:, 0]), 0.5 * np.cos(2 * math.pi * X[:, 1])
    y = f1 + f2 + 0.05 * g.standard_normal(n)
    opts = sampler.Opts(B=32, eps=1e-10, cap=32, kind=0, nugget=1e-6)
    prior = sampler.Prior(a_sigma2=1e-3, b_sigma2=1e-3, logrho_mu=math.log(0.2))
    st = sampler.additive_init(X, y, 0.2, opts)
    for _ in range(25):
        sampler.additive_sweep(st, y, prior, opts, seed=3)
    s2 = np.median([t["sigma2"] for t in st.trace[10:]])
    assert 0.0015 < s2 < 0.004
    # each component is identified up to a constant shift between the two
    c1 = st.F[:, 0] - st.F[:, 0].mean()
    c2 = st.F[:, 1] - st.F[:, 1].mean()
    assert np.corrcoef(c1, f1)[0, 1] > 0.95 and np.corrcoef(c2, f2)[0, 1] > 0.9
