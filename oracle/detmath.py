"""Deterministic exponential and covariance kernels (oracle side).

The ACA pivots must be bit-identical between this oracle and the GPU, so the
kernel entries feeding them must be bit-identical too.  Library ``exp``
functions differ in their last bit between platforms, so both sides evaluate
``det_exp``: a fixed sequence of IEEE-754 binary64 operations (products,
and fused multiply-adds with one rounding each, `oracle/fmath.py`), defined
here from the textbook method (Tang's table-driven exponential):

* argument reduction x = (32 m + j) ln2/32 + r with k = 32 m + j = rint(x 32/ln2),
  0 <= j < 32, ln2/32 split as HI + LO where HI keeps only the leading 32
  significand bits so that k * HI is exact for |k| < 2**21 (Cody & Waite);
  r = fma(-k, LO, fma(-k, HI, x));
* e**x = 2**m 2**(j/32) e**r with 2**(j/32) from a 32-entry table of correctly
  rounded values (computed here in 60-digit decimal arithmetic) and
  e**r = 1 + q, q = r(1 + r/2 + ... + r**5/6!) (|r| <= ln2/64, truncation
  below 4e-18 relative) by Horner's rule highest power first, each step one
  fused multiply-add p = fma(p, r, 1/j!), then q = p * r;
* the result fma(t, q, t) with t = 2**(j/32) 2**m built exactly (exponent field).

Inputs below -708 return exactly 0.0 (the true value is below 3.3e-308, and
this cut keeps every nonzero result a normal number).

Kernels (Sec. 2.1 and Sec. 4.1 of the paper; the parameterisation is the
length-scale form used by the workloads):

* squared exponential:  k(d) = exp(-d^2 / (2 rho^2)),
  evaluated as det_exp(-((d*d)*c)) with c = 0.5/(rho*rho);
* Matern-5/2:  k(d) = (1 + t + t^2/3) exp(-t), t = sqrt(5)|d|/rho,
  evaluated as fma(t*t, THIRD, 1+t) * det_exp(-t) with t = |d| * (sqrt(5)/rho)
  and THIRD = 1/3 rounded to binary64.

Both are unit-variance correlations; the nugget is added to the diagonal by
the caller (Sec. 4.1.4, "Additional considerations").
"""
from __future__ import annotations

import math
import struct
from decimal import Decimal, getcontext

import numpy as np

from .fmath import fma

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
EXP_TABLE_N = 32
# ln2/32 split (exact divisions by 32 of the ln2 split) and 32/ln2
LN2N_HI, LN2N_LO = LN2_HI / EXP_TABLE_N, LN2_LO / EXP_TABLE_N
INV_LN2N = INV_LN2 * EXP_TABLE_N


def _exp2_table():
    """2**(j/32), j = 0..31, correctly rounded to binary64 from 60-digit decimals."""
    getcontext().prec = 60
    return np.array([float(Decimal(2) ** (Decimal(j) / EXP_TABLE_N)) for j in range(EXP_TABLE_N)])


EXP2_TABLE = _exp2_table()
# 1/j! correctly rounded; j! is exact in binary64 for j <= 18.
TAYLOR = [1.0 / math.factorial(j) for j in range(7)]
EXP_MIN_ARG = -708.0
THIRD = 1.0 / 3.0  # binary64 nearest to 1/3 (IEEE division)


def det_exp(x):
    """Elementwise e**x by the fixed operation sequence described in the module doc."""
    x = np.asarray(x, dtype=np.float64)
    k = np.rint(x * INV_LN2N)
    r = fma(-k, LN2N_LO, fma(-k, LN2N_HI, x))
    p = np.full_like(x, TAYLOR[6])
    for j in range(5, 0, -1):
        p = fma(p, r, TAYLOR[j])
    q = p * r
    ki = np.where(x < EXP_MIN_ARG, 0, k).astype(np.int64)
    j = ki & (EXP_TABLE_N - 1)
    m = ki >> 5
    t = (EXP2_TABLE[j].view(np.int64) + (m << 52)).view(np.float64)
    out = fma(t, q, t)
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
        poly = fma(t * t, THIRD, 1.0 + t)
        return poly * det_exp(-t)
    raise ValueError("unknown kernel")
