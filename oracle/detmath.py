"""Deterministic exponential and covariance kernels (oracle side).

The ACA pivots must be bit-identical between this oracle and the GPU, so the
kernel entries feeding them must be bit-identical too.  Library ``exp``
functions differ in their last bit between platforms, so both sides evaluate
``det_exp``: a fixed sequence of IEEE-754 binary64 multiplications and
additions (no fused multiply-add), defined here from the textbook method:

* Cody & Waite (1980) argument reduction: x = k ln2 + r with k = rint(x / ln2),
  ln2 split as LN2_HI + LN2_LO where LN2_HI keeps only the leading 32 significand
  bits of ln2 so that k * LN2_HI is exact for |k| < 2**21;
* the Taylor series of e**r truncated after r**13/13! (|r| <= ln2/2, truncation
  error below 2e-18 relative), evaluated by Horner's rule highest power first;
* scaling by 2**k, built exactly as a power of two.

Inputs below -708 return exactly 0.0 (the true value is below 3.3e-308, and
this cut keeps every nonzero result a normal number).

Kernels (Sec. 2.1 and Sec. 4.1 of the paper; the parameterisation is the
length-scale form used by the workloads):

* squared exponential:  k(d) = exp(-d^2 / (2 rho^2)),
  evaluated as det_exp(-((d*d)*c)) with c = 0.5/(rho*rho);
* Matern-5/2:  k(d) = (1 + t + t^2/3) exp(-t), t = sqrt(5)|d|/rho,
  evaluated as ((1+t) + (t*t)/3) * det_exp(-t) with t = |d| * (sqrt(5)/rho).

Both are unit-variance correlations; the nugget is added to the diagonal by
the caller (Sec. 4.1.4, "Additional considerations").
"""
from __future__ import annotations

import math
import struct
from decimal import Decimal, getcontext

import numpy as np

KERNEL_SE = 0
KERNEL_MATERN52 = 1


def _ln2_split():
    """LN2_HI = ln 2 truncated to 32 significand bits; LN2_LO = ln2 - LN2_HI (rounded)."""
    getcontext().prec = 50
    ln2 = Decimal(2).ln()
    bits = struct.unpack("<Q", struct.pack("<d", float(ln2)))[0]
    hi_bits = bits & ~((1 << (52 - 31)) - 1)  # keep sign, exponent, 31 explicit + 1 implicit bits
    hi = struct.unpack("<d", struct.pack("<Q", hi_bits))[0]
    lo = float(ln2 - Decimal(hi))
    return hi, lo


LN2_HI, LN2_LO = _ln2_split()
INV_LN2 = float(1 / Decimal(2).ln())
# 1/j! correctly rounded; j! is exact in binary64 for j <= 18.
TAYLOR = [1.0 / math.factorial(j) for j in range(14)]
EXP_MIN_ARG = -708.0


def det_exp(x):
    """Elementwise e**x by the fixed operation sequence described in the module doc."""
    x = np.asarray(x, dtype=np.float64)
    k = np.rint(x * INV_LN2)
    r = (x - k * LN2_HI) - k * LN2_LO
    p = np.full_like(x, TAYLOR[13])
    for j in range(12, -1, -1):
        p = p * r + TAYLOR[j]
    kk = np.where(x < EXP_MIN_ARG, 0, k).astype(np.int64)
    scale = ((kk + 1023) << 52).view(np.float64)
    out = p * scale
    return np.where(x < EXP_MIN_ARG, 0.0, out)


def kernel_const(kind: int, rho: float) -> float:
    """Per-kernel constant c: 0.5/(rho*rho) (SE) or sqrt(5)/rho (Matern-5/2)."""
    if kind == KERNEL_SE:
        return 0.5 / (rho * rho)
    if kind == KERNEL_MATERN52:
        return math.sqrt(5.0) / rho
    raise ValueError("unknown kernel")


def kernel_entries(kind: int, c: float, xa, xb):
    """Unit-variance correlation between xa and xb (broadcast), no nugget."""
    d = np.subtract(xa, xb, dtype=np.float64)
    if kind == KERNEL_SE:
        return det_exp(-((d * d) * c))
    if kind == KERNEL_MATERN52:
        t = np.abs(d) * c
        poly = (1.0 + t) + (t * t) / 3.0
        return poly * det_exp(-t)
    raise ValueError("unknown kernel")
