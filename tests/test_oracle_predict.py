"""Pins of oracle/predict.py (Eq. gp_posterior_newx) by routes other than its own formula.

* one training input: the scalar closed form;
* the joint Gaussian of (f, f*): its Cholesky factor gives the conditional
  mean L21 L11^-1 f and variance L22^2 without any solve with C~ alone;
* a new input equal to a training input x_j (nugget d on the training block
  only, one dense leaf so that C~ = C + d I exactly): mu* = f_j - d (C~^-1 f)_j
  and sigma*^2 = tau2 d (1 - d (C~^-1)_jj), exact identities that fix where
  the nugget sits;
* a new input far from every training input: mu* = 0, sigma*^2 = tau2.

Two correct FP64 routes through C~ agree to about kappa(C~) u relative to the
magnitudes of the products involved, so the comparisons use 8 kappa u times
those magnitudes (kappa computed densely), as the GPU parity tests do.
"""
import numpy as np
import pytest

from oracle import detmath, hodlr
from oracle.predict import predict
from paper_2006_06537_gb300.inputs import uniform_sine

U = np.finfo(np.float64).eps / 2


def _setup(n=256, B=32, kind=0, rho=0.1, nug=1e-6, eps=1e-12, seed=3):
    x, _ = uniform_sine(n, seed)
    c = detmath.kernel_const(kind, rho)
    H = hodlr.assemble(x, B, kind, c, nug, eps, 32)
    f = np.random.default_rng(seed).standard_normal(n)
    return x, H, f, c


def test_single_input_closed_form():
    x = np.array([0.3])
    nug, tau2, kind, rho = 1e-3, 2.5, 0, 0.2
    c = detmath.kernel_const(kind, rho)
    H = hodlr.assemble(x, 8, kind, c, nug, 1e-12, 8)
    xs = np.array([0.1, 0.3, 0.45])
    f = np.array([1.7])
    mean, var = predict(H, x, xs, f, tau2, kind, c)
    k = np.exp(-(xs - 0.3) ** 2 / (2 * rho ** 2))
    np.testing.assert_allclose(mean, k * 1.7 / (1 + nug), rtol=1e-14)
    np.testing.assert_allclose(var, tau2 * (1 - k ** 2 / (1 + nug)), rtol=1e-12)


@pytest.mark.parametrize("kind", [0, 1])
def test_matches_joint_gaussian_cholesky(kind):
    x, H, f, c = _setup(kind=kind)
    tau2 = 0.7
    xs = np.array([0.0137, 0.5001, 0.9876])
    mean, var = predict(H, x, xs, f, tau2, kind, c)
    A = hodlr.dense(H)
    n = len(x)
    tol = 8 * np.linalg.cond(A) * U
    alpha = np.linalg.solve(A, f)
    for q, xq in enumerate(xs):
        J = np.empty((n + 1, n + 1))
        J[:n, :n] = A
        cq = detmath.kernel_entries(kind, c, np.full(n, xq), x)
        J[n, :n] = cq
        J[:n, n] = cq
        J[n, n] = 1.0
        L = np.linalg.cholesky(tau2 * J)
        z = np.linalg.solve(L[:n, :n], f)          # lower-triangular system
        m_ref = L[n, :n] @ z
        v_ref = L[n, n] ** 2
        assert abs(mean[q] - m_ref) <= tol * (np.abs(cq) @ np.abs(alpha))
        assert abs(var[q] - v_ref) <= tol * tau2 * (1.0 + np.abs(cq) @ np.abs(np.linalg.solve(A, cq)))


def test_new_input_at_a_training_input():
    nug = 1e-4
    x, H, f, c = _setup(n=64, B=64, nug=nug)  # one leaf: C~ = C + nug I exactly
    assert H.tree.L == 0
    tau2 = 1.3
    j = 37
    mean, var = predict(H, x, x[j:j + 1], f, tau2, 0, c)
    A = hodlr.dense(H)
    tol = 8 * np.linalg.cond(A) * U
    Ainv = np.linalg.inv(A)
    alpha = Ainv @ f
    assert abs(mean[0] - (f[j] - nug * alpha[j])) <= tol * (np.abs(A[j]) @ np.abs(alpha))
    v_ref = tau2 * nug * (1 - nug * Ainv[j, j])
    assert abs(var[0] - v_ref) <= tol * tau2 * (1.0 + np.abs(A[j]) @ np.abs(Ainv[:, j]))
    assert 0.0 < var[0] <= tau2 * nug


def test_new_input_far_away():
    x, H, f, c = _setup()
    tau2 = 0.9
    mean, var = predict(H, x, np.array([50.0]), f, tau2, 0, c)
    assert mean[0] == 0.0
    assert var[0] == tau2
