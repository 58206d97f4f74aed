"""Tensor product of 1-D GPs for d > 1 inputs (Sec. 4.2, Eq. tensor_prod),
oracle side; test infrastructure only.

    y_i = beta f_1(x_{1,i}) ... f_d(x_{d,i}) + e_i,   e_i ~ N(0, sigma2),
    f_h ~ GP(m_h, C(rho_h)),   C a unit-variance kernel (plus the nugget).

Block update of f_h (Sec. 4.2: the conditional of each f_h has heteroskedastic
noise): with g_i = beta prod_{k != h} f_k(x_{k,i}), the value y_i / g_i
observes f_h(x_{h,i}) with precision d_i = g_i^2 / sigma2, so f_h - m_h is drawn
by Algorithm 1.h (oracle/hetero.py) with K~ = C~(rho_h) (tau2 = 1), D = diag(d)
and data y / g - m_h, in the order of the sorted x_h.

Readings (the paper leaves these open):
  * m_h = 1 for every h: a constant prior mean that keeps the product away
    from zero; every f_h starts at 1;
  * beta ~ N(mu_beta, s_beta^2), drawn from its conjugate normal conditional
    given the products G_i = prod_h f_h(x_{h,i});
  * sigma2 ~ IG(a + n/2, b + ||y - beta G||^2 / 2) as in the 1-D sampler;
  * rho_h by the random-walk Metropolis step on log rho_h of the 1-D sampler
    with tau2 = 1 and q = (f_h - m_h)^T C~_h^-1 (f_h - m_h);
  * a zero g_i (no information on f_h at that input) is an error.

Sweep order: f_1 .. f_d, beta, sigma2, then the d Metropolis steps.  Random
numbers: block h draws its normals a, b and its Metropolis numbers from Philox
stream id h, sigma2 from stream id d, beta from stream id d + 1 (tag A), all
at counter word 2 = the sweep index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import rng
from .factor import NotSPD, apply_W
from .hetero import draw_f_hetero
from .sampler import Opts, Prior, assemble_factor, log_prior_eta


@dataclass
class BetaPrior:
    mu: float = 1.0
    sd: float = 1.0


@dataclass
class TensorState:
    F: np.ndarray          # n x d, original order
    beta: float
    sigma2: float
    blocks: list           # per block: dict(perm, x, eta, HC, FC, m)
    it: int = 0
    trace: list = field(default_factory=list)


def tensor_init(X, y, rho0, opts: Opts, sigma2=None, beta=1.0):
    n, d = X.shape
    blocks = []
    for h in range(d):
        perm = np.argsort(X[:, h], kind="stable")
        xs = X[perm, h]
        HC, FC = assemble_factor(xs, rho0, opts)
        blocks.append(dict(perm=perm, x=xs, eta=math.log(rho0), HC=HC, FC=FC, m=1.0))
    s2 = 0.5 * float(np.var(y)) if sigma2 is None else sigma2
    return TensorState(F=np.ones((n, d)), beta=beta, sigma2=s2, blocks=blocks)


def products(F, skip=None):
    """prod_h F[:, h] over h != skip, multiplied in h order."""
    g = np.ones(F.shape[0])
    for h in range(F.shape[1]):
        if h != skip:
            g = g * F[:, h]
    return g


def block_data(st: TensorState, y, h):
    """(data y/g - m_h, precisions g^2/sigma2) of block h, in the order of the sorted x_h."""
    b = st.blocks[h]
    g = st.beta * products(st.F, skip=h)
    if np.any(g == 0.0):
        raise ValueError("a zero product carries no information on f_h")
    yt = np.asarray(y, dtype=np.float64) / g - b["m"]
    d = g * g / st.sigma2
    return yt[b["perm"]], d[b["perm"]]


def beta_conditional(G, y, sigma2, prior: BetaPrior):
    """(mean, variance) of beta | y, G: prior N(mu, sd^2), data y = beta G + e."""
    G = np.asarray(G, dtype=np.float64)
    prec = 1.0 / prior.sd ** 2 + float(G @ G) / sigma2
    v = 1.0 / prec
    m = v * (prior.mu / prior.sd ** 2 + float(G @ np.asarray(y, dtype=np.float64)) / sigma2)
    return m, v


def tensor_sweep(st: TensorState, y, prior: Prior, bprior: BetaPrior, opts: Opts, seed: int):
    n, d = st.F.shape
    it = st.it
    y = np.asarray(y, dtype=np.float64)
    for h, b in enumerate(st.blocks):
        yt, dd = block_data(st, y, h)
        a0 = rng.normals(n, seed, rng.TAG_A, it, h)
        b0 = rng.normals(n, seed, rng.TAG_B, it, h)
        g, _ = draw_f_hetero(b["HC"], b["FC"], yt, 1.0, dd, a0, b0)
        b["g"] = g
        st.F[b["perm"], h] = b["m"] + g
    G = products(st.F)
    m, v = beta_conditional(G, y, st.sigma2, bprior)
    st.beta = m + math.sqrt(v) * rng.scalar_normal(0, seed, rng.TAG_A, it, d + 1)
    res = y - st.beta * G
    rss = float(np.sum(res * res))
    st.sigma2 = rng.inv_gamma_draw(prior.a_sigma2 + 0.5 * n, prior.b_sigma2 + 0.5 * rss, seed, rng.TAG_SIGMA2, it, d)
    row = dict(it=it, beta=st.beta, sigma2=st.sigma2, rss=rss, rho=[], accept=[])
    for h, b in enumerate(st.blocks):
        g = b["g"]
        q = float(np.sum(apply_W(b["FC"], g, inverse=True) ** 2))
        z = rng.scalar_normal(0, seed, rng.TAG_MH_PROP, it, h)
        eta_p = b["eta"] + prior.prop_sd * z
        u = rng.scalar_uniform(0, seed, rng.TAG_MH_UNIF, it, h)
        accept = False
        try:
            HCp, FCp = assemble_factor(b["x"], math.exp(eta_p), opts)
            qp = float(np.sum(apply_W(FCp, g, inverse=True) ** 2))
            la = (-0.5 * (FCp.logdet - b["FC"].logdet) - 0.5 * (qp - q)
                  + log_prior_eta(eta_p, prior) - log_prior_eta(b["eta"], prior))
            accept = math.log(u) < la
        except NotSPD:
            pass
        if accept:
            b["eta"], b["HC"], b["FC"] = eta_p, HCp, FCp
        row["rho"].append(math.exp(b["eta"]))
        row["accept"].append(accept)
    st.trace.append(row)
    st.it = it + 1
    return st
