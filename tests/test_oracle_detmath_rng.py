"""Pins for the oracle's deterministic exponential, kernels and random numbers.

Each check ties the oracle to something outside itself: exact rational
arithmetic for the fused multiply-add, libm's exp and the
closed-form kernels, the mathematical definitions of the Philox Weyl
increments, distribution laws of uniforms / normals / gamma variates
(scipy.stats), and bit-avalanche behaviour of a 10-round Philox.
"""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

from oracle import detmath, fmath, rng


def _fma_exact(a, b, c):
    """a * b + c in exact rational arithmetic, rounded once (float(Fraction) rounds to nearest-even)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def test_fma_is_one_rounding_of_the_exact_value():
    g = np.random.default_rng(5)
    a = g.standard_normal(3000) * 2.0 ** g.integers(-40, 40, 3000)
    b = g.standard_normal(3000) * 2.0 ** g.integers(-40, 40, 3000)
    # c near -a*b: the cases where a separately rounded product loses the most
    c = np.concatenate([-(a[:1000] * b[:1000]), g.standard_normal(2000)])
    got = fmath.fma(a, b, c)
    ref = np.array([_fma_exact(float(x), float(y), float(z)) for x, y, z in zip(a, b, c)])
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    # a case a product-then-sum gets wrong: (1 + 2^-30)(1 - 2^-30) - 1 = -2^-60 exactly
    t = fmath.fma(1 + 2.0 ** -30, 1 - 2.0 ** -30, -1.0)
    assert t == -(2.0 ** -60) and (1 + 2.0 ** -30) * (1 - 2.0 ** -30) - 1.0 == 0.0
    # ties round to even: 1 + 2^-53 (exactly between 1 and 1 + 2^-52)
    assert fmath.fma(2.0 ** -27, 2.0 ** -26, 1.0) == 1.0
    assert fmath.fma(3 * 2.0 ** -27, 2.0 ** -26, 1.0) == 1 + 2.0 ** -51
    # broadcasting and shapes
    assert fmath.fma(np.ones((2, 3)), 2.0, np.arange(3.0)).shape == (2, 3)


def test_det_exp_within_one_ulp_of_libm():
    g = np.random.default_rng(0)
    x = np.concatenate([-g.uniform(0, 708, 100000), -g.uniform(0, 1, 50000),
                        -g.uniform(0, 1e-8, 1000), [0.0, -1e-300, -708.0]])
    y = detmath.det_exp(x)
    ref = np.array([math.exp(v) for v in x])
    ulp = np.abs(y - ref) / np.spacing(ref)
    assert ulp.max() <= 1.0


def test_det_exp_special_values():
    assert detmath.det_exp(np.array([0.0]))[0] == 1.0
    assert detmath.det_exp(np.array([-708.5, -1e4]))[1] == 0.0
    # ln2 split: 32 significand bits in the high part, and hi + lo = ln 2 to half an ulp of lo (~1.3e-26)
    bits = np.float64(detmath.LN2_HI).view(np.uint64)
    assert int(bits) & ((1 << 21) - 1) == 0
    getcontext().prec = 50
    assert abs(Decimal(detmath.LN2_HI) + Decimal(detmath.LN2_LO) - Decimal(2).ln()) < Decimal("2e-26")
    # the ln2/32 split is the ln2 split scaled by an exact power of two, and 32/ln2 is correctly rounded
    assert detmath.LN2N_HI * 32 == detmath.LN2_HI and detmath.LN2N_LO * 32 == detmath.LN2_LO
    inv = Decimal(32) / Decimal(2).ln()
    assert abs(Decimal(detmath.INV_LN2N) - inv) <= Decimal(np.spacing(detmath.INV_LN2N)) / 2


def test_exp2_table_against_independent_values():
    t = detmath.EXP2_TABLE
    assert t[0] == 1.0
    assert t[16] == math.sqrt(2.0)          # IEEE square root is correctly rounded
    assert t[8] == math.sqrt(math.sqrt(2.0)) or abs(t[8] - 2 ** 0.25) <= np.spacing(t[8])
    for j in range(32):
        ref = 2.0 ** (j / 32)                # libm pow: within an ulp of the correctly rounded value
        assert abs(t[j] - ref) <= np.spacing(ref), j
        if j:
            assert abs(t[j] * t[32 - j] - 2.0) <= 4 * np.spacing(2.0), j
    assert np.all(np.diff(t) > 0)


def test_det_exp_near_reduction_boundaries():
    # arguments at and next to multiples of ln2/32, where r changes sign and j wraps
    k = np.arange(-32685, 1)
    x0 = k * (math.log(2.0) / 32)
    x = np.concatenate([x0, np.nextafter(x0, -np.inf), np.nextafter(x0, np.inf)])
    x = x[(x <= 0) & (x >= -708)]
    y = detmath.det_exp(x)
    ref = np.exp(x)
    assert (np.abs(y - ref) / np.spacing(ref)).max() <= 1.0


@pytest.mark.parametrize("kind", [detmath.KERNEL_SE, detmath.KERNEL_MATERN52])
def test_kernels_match_closed_form(kind):
    g = np.random.default_rng(1)
    rho = 0.07
    c = detmath.kernel_const(kind, rho)
    xa, xb = g.uniform(0, 1, 2000), g.uniform(0, 1, 2000)
    got = detmath.kernel_entries(kind, c, xa, xb)
    d = np.abs(xa - xb)
    if kind == detmath.KERNEL_SE:
        ref = np.exp(-d * d / (2 * rho * rho))
    else:
        t = math.sqrt(5.0) * d / rho
        ref = (1 + t + t * t / 3) * np.exp(-t)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-300)
    # symmetric in the argument order, bit for bit
    assert np.array_equal(got, detmath.kernel_entries(kind, c, xb, xa))


def test_philox_weyl_increments_from_definition():
    getcontext().prec = 60
    phi = (1 + Decimal(5).sqrt()) / 2
    assert rng.W0 == int((phi - 1) * (1 << 32))
    assert rng.W1 == int((Decimal(3).sqrt() - 1) * (1 << 32))


def test_philox_avalanche():
    # flipping one counter bit should flip about half of the 128 output bits
    g = np.random.default_rng(2)
    ctr = g.integers(0, 2 ** 32, (4000, 4), dtype=np.uint64)
    base = rng.philox4x32_10(ctr, (123, 456))
    flips = []
    for word in range(4):
        for bit in (0, 13, 31):
            c2 = ctr.copy()
            c2[:, word] ^= np.uint64(1 << bit)
            out = rng.philox4x32_10(c2, (123, 456))
            x = (base ^ out).astype(np.uint64)
            nb = sum(np.unpackbits(x[:, w].astype(">u4").view(np.uint8)).reshape(len(x), 32).sum(1) for w in range(4))
            flips.append(nb.mean())
    assert all(abs(f - 64.0) < 1.0 for f in flips)


def test_uniform_and_normal_laws():
    z = rng.normals(400000, seed=9, tag=rng.TAG_A, it=3, chain=1)
    assert abs(z.mean()) < 5 / math.sqrt(len(z))
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / len(z))
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # different streams are independent
    z2 = rng.normals(400000, seed=9, tag=rng.TAG_B, it=3, chain=1)
    assert abs(np.corrcoef(z, z2)[0, 1]) < 5 / math.sqrt(len(z))
    w = rng.philox4x32_10(np.stack([np.arange(200000), np.zeros(200000), np.zeros(200000), np.zeros(200000)], 1), (1, 0))
    u = rng.uniforms_from_words(w[:, 0], w[:, 1])
    assert u.min() > 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-3


@pytest.mark.parametrize("alpha", [1.0, 2.5, 1025.0])
def test_gamma_sampler_law(alpha):
    draws = np.array([rng.gamma_draw(alpha, seed=5, tag=rng.TAG_TAU2, it=t, chain=0)[0] for t in range(4000)])
    assert stats.kstest(draws, stats.gamma(alpha).cdf).pvalue > 1e-3
    assert abs(draws.mean() - alpha) < 5 * math.sqrt(alpha / len(draws))
