"""Algorithm 1 and one Gibbs iteration (oracle side), Sec. 4.1 of the paper.

Parameterisation (the workloads' form; the paper's symbols in brackets):
    y = f + e,  e ~ N(0, sigma2 I)                [precision tau = 1/sigma2]
    f ~ N(0, K),  K = tau2 * C(rho)               [sigma_f^2 = tau2]
    C(rho) = unit-variance kernel + nugget * I,  C~ its HODLR approximation,
    K~ = tau2 C~,  M~ = K~/sigma2 + I = s C~ + I with s = tau2/sigma2.
With W_C W_C^T = C~, the factor of K~ is W = sqrt(tau2) W_C.

Algorithm 1 (draw of f | y, Theta):
    a, b ~ N(0, I)
    Z = sqrt(1/sigma2) K~ a + W b   = (tau2/sigma) C~ a + tau W_C b
    solve M~ w = Z
    solve M~ r = y / sigma2
    return f = w + K~ r             (K~ r = tau2 C~ r is the posterior mean)

Gibbs iteration, in the order of Eqs. (posterior_gibs1)-(posterior_gibs4),
with conjugate inverse-gamma priors IG(shape, scale) on the two variances
(equivalent to the paper's gamma priors on the precisions) and, for the
length-scale, the Metropolis step the paper names as the alternative to its
discrete grid (Sec. 4.1), on eta = log rho with a normal prior:
    f       ~ Algorithm 1
    sigma2  ~ IG(a_s + n/2, b_s + ||y - f||^2 / 2)
    tau2    ~ IG(a_t + n/2, b_t + q / 2),  q = f^T C~^-1 f = ||W_C^-1 f||^2
    eta'    = eta + prop_sd * z;  C~' = C~(exp eta') assembled and factored;
    log alpha = -(logdet C~' - logdet C~)/2 - (q' - q)/(2 tau2)
                + log prior(eta') - log prior(eta)
    accept eta' if log u < log alpha (a non-positive-definite C~' is rejected).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import rng
from .detmath import kernel_const
from .factor import NotSPD, apply_W, factorize, solve
from .hodlr import assemble, matvec, shift_scale


def draw_f(HC, FC, FM, y, tau2, sigma2, a, b):
    """Algorithm 1 with given normals a, b. Returns (f, posterior mean tau2 C~ r)."""
    sig = math.sqrt(sigma2)
    tau = math.sqrt(tau2)
    Z = (tau2 / sig) * matvec(HC, a) + tau * apply_W(FC, b)
    w = solve(FM, Z)
    r = solve(FM, np.asarray(y) / sigma2)
    mean = tau2 * matvec(HC, r)
    return w + mean, mean


@dataclass
class Prior:
    a_tau2: float = 1.0
    b_tau2: float = 1.0
    a_sigma2: float = 1.0
    b_sigma2: float = 1.0
    logrho_mu: float = math.log(0.1)
    logrho_sd: float = 1.0
    prop_sd: float = 0.2


@dataclass
class Opts:
    B: int = 64
    eps: float = 1e-12
    cap: int = 64
    kind: int = 0
    nugget: float = 1e-8


@dataclass
class State:
    f: np.ndarray
    sigma2: float
    tau2: float
    eta: float
    HC: object = None
    FC: object = None
    it: int = 0
    trace: list = field(default_factory=list)


def log_prior_eta(eta, prior: Prior):
    z = (eta - prior.logrho_mu) / prior.logrho_sd
    return -0.5 * z * z


def assemble_factor(x, rho, opts: Opts):
    HC = assemble(x, opts.B, opts.kind, kernel_const(opts.kind, rho), opts.nugget, opts.eps, opts.cap)
    FC = factorize(HC)
    return HC, FC


def init_state(x, y, rho0, opts: Opts, sigma2=None, tau2=None):
    vy = float(np.var(y))
    s2 = 0.5 * vy if sigma2 is None else sigma2
    t2 = vy if tau2 is None else tau2
    HC, FC = assemble_factor(x, rho0, opts)
    return State(f=np.zeros(len(x)), sigma2=s2, tau2=t2, eta=math.log(rho0), HC=HC, FC=FC)


def gibbs_step(st: State, x, y, prior: Prior, opts: Opts, seed: int, chain: int):
    n = len(x)
    it = st.it
    y = np.asarray(y, dtype=np.float64)
    # f | y, tau2, sigma2, rho  (Algorithm 1)
    s = st.tau2 / st.sigma2
    FM = factorize(shift_scale(st.HC, s))
    a = rng.normals(n, seed, rng.TAG_A, it, chain)
    b = rng.normals(n, seed, rng.TAG_B, it, chain)
    f, mean = draw_f(st.HC, st.FC, FM, y, st.tau2, st.sigma2, a, b)
    # sigma2 | y, f
    rss = float(np.sum((y - f) ** 2))
    sigma2 = rng.inv_gamma_draw(prior.a_sigma2 + 0.5 * n, prior.b_sigma2 + 0.5 * rss,
                                seed, rng.TAG_SIGMA2, it, chain)
    # tau2 | f, rho
    q = float(np.sum(apply_W(st.FC, f, inverse=True) ** 2))
    tau2 = rng.inv_gamma_draw(prior.a_tau2 + 0.5 * n, prior.b_tau2 + 0.5 * q,
                              seed, rng.TAG_TAU2, it, chain)
    # rho | f, tau2 (random-walk Metropolis on eta = log rho)
    z = rng.scalar_normal(0, seed, rng.TAG_MH_PROP, it, chain)
    eta_p = st.eta + prior.prop_sd * z
    u = rng.scalar_uniform(0, seed, rng.TAG_MH_UNIF, it, chain)
    accept = False
    log_alpha = -math.inf
    try:
        HCp, FCp = assemble_factor(x, math.exp(eta_p), opts)
        qp = float(np.sum(apply_W(FCp, f, inverse=True) ** 2))
        log_alpha = (-0.5 * (FCp.logdet - st.FC.logdet) - (qp - q) / (2.0 * tau2)
                     + log_prior_eta(eta_p, prior) - log_prior_eta(st.eta, prior))
        accept = math.log(u) < log_alpha
    except NotSPD:
        pass
    st.trace.append(dict(it=it, sigma2=sigma2, tau2=tau2, eta_prop=eta_p, log_alpha=log_alpha,
                         accept=accept, q=q, rss=rss, logdet=st.FC.logdet))
    st.f, st.sigma2, st.tau2 = f, sigma2, tau2
    st.mean = mean
    if accept:
        st.eta, st.HC, st.FC = eta_p, HCp, FCp
    st.it = it + 1
    return st


# ---------------------------------------------------------------------------
# Additive model built from 1-D GPs (Sec. 4.2 notes that an additive model may
# suffice; the workload's d-dimensional surface): y = sum_k f_k(x_k) + e,
# f_k ~ GP(0, tau2_k C(rho_k)) on the k-th input coordinate, shared sigma2.
# One block-Gibbs sweep:
#   for k = 0..d-1:  r = y - sum_{j != k} f_j (subtracted in j order), sorted by
#                    x_k; f_k | r by Algorithm 1 with (tau2_k, sigma2, rho_k)
#   sigma2 | y, f    (Philox stream id d)
#   for k:           tau2_k | f_k, then the Metropolis step on log rho_k
# Block k draws its normals, gamma variates and Metropolis numbers from Philox
# stream id k, all at counter word 2 = sweep index.
# ---------------------------------------------------------------------------
@dataclass
class AdditiveState:
    F: np.ndarray          # n x d, original order
    sigma2: float
    blocks: list           # per block: dict(perm, x, tau2, eta, HC, FC)
    it: int = 0
    trace: list = field(default_factory=list)


def additive_init(X, y, rho0, opts: Opts, sigma2=None, tau2=None):
    n, d = X.shape
    vy = float(np.var(y))
    blocks = []
    for k in range(d):
        perm = np.argsort(X[:, k], kind="stable")
        xs = X[perm, k]
        HC, FC = assemble_factor(xs, rho0, opts)
        blocks.append(dict(perm=perm, x=xs, tau2=(vy / d if tau2 is None else tau2), eta=math.log(rho0), HC=HC, FC=FC))
    return AdditiveState(F=np.zeros((n, d)), sigma2=(0.5 * vy if sigma2 is None else sigma2), blocks=blocks)


def additive_sweep(st: AdditiveState, y, prior: Prior, opts: Opts, seed: int):
    n, d = st.F.shape
    it = st.it
    y = np.asarray(y, dtype=np.float64)
    for k, b in enumerate(st.blocks):
        r = y.copy()
        for j in range(d):
            if j != k:
                r = r - st.F[:, j]
        rs = r[b["perm"]]
        FM = factorize(shift_scale(b["HC"], b["tau2"] / st.sigma2))
        a_ = rng.normals(n, seed, rng.TAG_A, it, k)
        b_ = rng.normals(n, seed, rng.TAG_B, it, k)
        fs, _ = draw_f(b["HC"], b["FC"], FM, rs, b["tau2"], st.sigma2, a_, b_)
        b["f"] = fs
        st.F[b["perm"], k] = fs
    res = y.copy()
    for j in range(d):
        res = res - st.F[:, j]
    rss = float(np.sum(res * res))
    st.sigma2 = rng.inv_gamma_draw(prior.a_sigma2 + 0.5 * n, prior.b_sigma2 + 0.5 * rss, seed, rng.TAG_SIGMA2, it, d)
    row = dict(it=it, sigma2=st.sigma2, rss=rss, tau2=[], rho=[], accept=[])
    for k, b in enumerate(st.blocks):
        fs = b["f"]
        q = float(np.sum(apply_W(b["FC"], fs, inverse=True) ** 2))
        b["tau2"] = rng.inv_gamma_draw(prior.a_tau2 + 0.5 * n, prior.b_tau2 + 0.5 * q, seed, rng.TAG_TAU2, it, k)
        z = rng.scalar_normal(0, seed, rng.TAG_MH_PROP, it, k)
        eta_p = b["eta"] + prior.prop_sd * z
        u = rng.scalar_uniform(0, seed, rng.TAG_MH_UNIF, it, k)
        accept = False
        try:
            HCp, FCp = assemble_factor(b["x"], math.exp(eta_p), opts)
            qp = float(np.sum(apply_W(FCp, fs, inverse=True) ** 2))
            la = (-0.5 * (FCp.logdet - b["FC"].logdet) - (qp - q) / (2.0 * b["tau2"])
                  + log_prior_eta(eta_p, prior) - log_prior_eta(b["eta"], prior))
            accept = math.log(u) < la
        except NotSPD:
            pass
        if accept:
            b["eta"], b["HC"], b["FC"] = eta_p, HCp, FCp
        row["tau2"].append(b["tau2"])
        row["rho"].append(math.exp(b["eta"]))
        row["accept"].append(accept)
    st.trace.append(row)
    st.it = it + 1
    return st
