"""Pins of oracle/rhogrid.py (Eq. posterior_gibs4, length-scale on a grid).

* the log-weights against the dense Gaussian log-density of f under every
  K_h = tau2 C~(s_h) (numpy slogdet and solve, with the n log tau2 and
  2 pi terms kept): the differences between grid points agree within
  8 kappa u of the log-densities' size, and so do the probabilities;
* a single grid point always has probability 1 and index 0; a uniform prior
  given explicitly changes nothing; a prior that puts all but one point at
  -inf selects that point;
* the draw is the inverse CDF: u just below and just above each cumulative
  boundary picks the two neighbouring indices.
"""
import numpy as np
import pytest

from oracle import detmath, hodlr
from oracle.factor import factorize
from oracle.rhogrid import grid_draw, grid_logw, grid_probs, grid_step, grid_terms
from paper_2006_06537_gb300.inputs import uniform_sine

U = np.finfo(np.float64).eps / 2
GRID = [0.05, 0.08, 0.12, 0.2, 0.3]


def _grid(n=128, B=16, nug=1e-6):
    x, _ = uniform_sine(n, 4)
    Hs = [hodlr.assemble(x, B, 0, detmath.kernel_const(0, r), nug, 1e-12, 32) for r in GRID]
    return x, Hs, [factorize(H) for H in Hs]


def test_probabilities_match_dense_densities():
    x, Hs, Fs = _grid()
    n = len(x)
    tau2 = 0.6
    f = np.random.default_rng(7).standard_normal(n) * 0.3
    p = grid_step(Fs, f, tau2, 0.5)[1]
    logdens, kap = [], 0.0
    for H in Hs:
        K = tau2 * hodlr.dense(H)
        sign, ld = np.linalg.slogdet(K)
        assert sign > 0
        logdens.append(-0.5 * ld - 0.5 * f @ np.linalg.solve(K, f) - 0.5 * n * np.log(2 * np.pi))
        kap = max(kap, np.linalg.cond(K))
    logdens = np.array(logdens)
    e = 8 * kap * U * np.max(np.abs(logdens))
    lw = grid_logw(*grid_terms(Fs, f), tau2)
    assert np.max(np.abs((lw - lw[0]) - (logdens - logdens[0]))) <= 2 * e
    ref = np.exp(logdens - logdens.max())
    ref /= ref.sum()
    # an absolute error e in the log-densities moves the probabilities by at most about 2 e
    assert np.max(np.abs(p - ref)) <= 2 * e + 1e-15
    assert p.sum() == pytest.approx(1.0, abs=1e-15)


def test_single_point_and_priors():
    x, Hs, Fs = _grid()
    f = np.random.default_rng(8).standard_normal(len(x)) * 0.3
    idx, p = grid_step(Fs[:1], f, 0.5, 0.999)
    assert idx == 0 and p[0] == 1.0
    ld, q = grid_terms(Fs, f)
    base = grid_probs(ld, q, 0.5)
    np.testing.assert_allclose(grid_probs(ld, q, 0.5, log_prior=np.full(len(GRID), -np.log(len(GRID)))), base,
                               rtol=1e-14)
    only = np.full(len(GRID), -np.inf)
    only[3] = 0.0
    p3 = grid_probs(ld, q, 0.5, log_prior=only)
    assert p3[3] == 1.0 and np.all(np.delete(p3, 3) == 0.0)


def test_draw_is_inverse_cdf():
    p = np.array([0.1, 0.25, 0.05, 0.6])
    cdf = np.cumsum(p)
    assert grid_draw(p, 0.0) == 0
    for h in range(len(p) - 1):
        assert grid_draw(p, np.nextafter(cdf[h], 0.0)) == h
        assert grid_draw(p, cdf[h]) == h + 1
    assert grid_draw(p, np.nextafter(1.0, 0.0)) == len(p) - 1
