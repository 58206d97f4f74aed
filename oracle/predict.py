"""Function posterior at new inputs (oracle side; test infrastructure only).

Sec. "Function posterior at new inputs", Eq. (gp_posterior_newx): conditioned
on the function values f at the training inputs (the Gibbs state), the value
f* at a new input x* is normal with

    mu*      = k_{*n} K^-1 f,
    sigma*^2 = k_{**} - k_{*n} K^-1 k_{n*}.

Here K = tau2 C~ is the compressed prior covariance of the training inputs
(C~ carries the nugget on its diagonal) and k = tau2 c for the unit-variance
kernel c, so

    mu*      = c_{*n} C~^-1 f,
    sigma*^2 = tau2 (1 - c_{*n} C~^-1 c_{n*}),

with k_{**} = tau2 c(x*, x*) = tau2.  Reading: the nugget regularizes the
training block only; the cross kernel c_{*n} and k_{**} have none.

Plain dense linear algebra on the n x n matrix the HODLR representation stands
for (small n only); no blocking or reordering beyond the formulas above.
"""
from __future__ import annotations

import numpy as np

from .detmath import kernel_entries
from .hodlr import HMat, dense


def predict(H: HMat, x, x_star, f, tau2: float, kind: int, c: float):
    """(mu*, sigma*^2) at every new input of x_star given f at the inputs x of H."""
    x = np.asarray(x, dtype=np.float64)
    xs = np.atleast_1d(np.asarray(x_star, dtype=np.float64))
    A = dense(H)                                         # C~
    Cs = kernel_entries(kind, c, xs[:, None], x[None, :])  # c_{*n}, one row per new input
    alpha = np.linalg.solve(A, np.asarray(f, dtype=np.float64))
    mean = Cs @ alpha
    Z = np.linalg.solve(A, Cs.T)                         # C~^-1 c_{n*}
    var = tau2 * (1.0 - np.einsum("ij,ji->i", Cs, Z))
    return mean, var
