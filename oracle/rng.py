"""Counter-based random numbers for the Gibbs sampler (oracle side).

Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11): a 128-bit counter and a 64-bit key pass through ten
rounds.  One round takes the counter words (c0, c1, c2, c3) and key (k0, k1):

    (hi0, lo0) = 64-bit product M0 * c0 split in halves
    (hi1, lo1) = 64-bit product M1 * c2 split in halves
    out        = (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)

and between rounds the key advances by the Weyl increments
W0 = floor(2**32 (phi - 1)) and W1 = floor(2**32 (sqrt(3) - 1)).
The multipliers M0 = 0xD2511F53 and M1 = 0xCD9E8D57 are the ones the paper
chose for the 4x32 variant.

Pinned against cuRAND's curand_Philox4x32_10 (known answers in
tests/test_oracle_philox_kat.py).

Counter layout used by the sampler (one call yields four 32-bit words):
    word 0: element-pair or attempt index, word 1: stream tag,
    word 2: Gibbs iteration (low 32 bits), word 3: chain id (low 32 bits);
    key = seed (low word, high word).
Stream tags: 0 = a, 1 = b (Algorithm 1 normals), 2 = sigma^2 gamma draw,
3 = tau^2 gamma draw, 4 = Metropolis proposal, 5 = Metropolis uniform.

Uniforms: u = (k + 0.5) * 2**-52 with k = (w_a << 20) | (w_b >> 12), a 52-bit
integer, so u lies strictly inside (0, 1) and is exact in binary64.
Normals: Box-Muller on the two uniforms of one call, giving two normals.
Gamma(alpha, 1), alpha >= 1: Marsaglia & Tsang (2000), "A simple method for
generating gamma variables", attempt t uses counters 2t (normal) and 2t+1
(uniform).
"""
from __future__ import annotations

import math

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

TAG_A, TAG_B, TAG_SIGMA2, TAG_TAU2, TAG_MH_PROP, TAG_MH_UNIF = 0, 1, 2, 3, 4, 5
GAMMA_MAX_ATTEMPTS = 64


def philox4x32_10(ctr, key):
    """ctr: (N, 4) uint32-valued array; key: (k0, k1). Returns (N, 4) uint64 words < 2**32."""
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4).copy()
    k0, k1 = np.uint64(key[0] & MASK32), np.uint64(key[1] & MASK32)
    m32 = np.uint64(MASK32)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(W0)) & m32
            k1 = (k1 + np.uint64(W1)) & m32
        p0 = np.uint64(M0) * c[:, 0]
        p1 = np.uint64(M1) * c[:, 2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & m32
        hi1, lo1 = p1 >> np.uint64(32), p1 & m32
        c = np.stack([hi1 ^ c[:, 1] ^ k0, lo1, hi0 ^ c[:, 3] ^ k1, lo0], axis=1)
    return c


def key_of(seed: int):
    return (seed & MASK32, (seed >> 32) & MASK32)


def uniforms_from_words(wa, wb):
    k = (np.asarray(wa, dtype=np.uint64) << np.uint64(20)) | (np.asarray(wb, dtype=np.uint64) >> np.uint64(12))
    return (k.astype(np.float64) + 0.5) * 2.0 ** -52


def _box_muller(u0, u1):
    rad = np.sqrt(-2.0 * np.log(u0))
    ang = 2.0 * math.pi * u1
    return rad * np.cos(ang), rad * np.sin(ang)


def normals(n: int, seed: int, tag: int, it: int, chain: int):
    """n standard normals of stream (tag, iteration, chain): call q gives elements 2q, 2q+1."""
    nq = (n + 1) // 2
    ctr = np.zeros((nq, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nq, dtype=np.uint64)
    ctr[:, 1] = tag
    ctr[:, 2] = it & MASK32
    ctr[:, 3] = chain & MASK32
    w = philox4x32_10(ctr, key_of(seed))
    z0, z1 = _box_muller(uniforms_from_words(w[:, 0], w[:, 1]), uniforms_from_words(w[:, 2], w[:, 3]))
    out = np.empty(2 * nq)
    out[0::2] = z0
    out[1::2] = z1
    return out[:n]


def _call(idx, seed, tag, it, chain):
    w = philox4x32_10([[idx, tag, it & MASK32, chain & MASK32]], key_of(seed))[0]
    return w


def scalar_normal(idx, seed, tag, it, chain):
    w = _call(idx, seed, tag, it, chain)
    z0, _ = _box_muller(uniforms_from_words(w[0], w[1]), uniforms_from_words(w[2], w[3]))
    return float(z0)


def scalar_uniform(idx, seed, tag, it, chain):
    w = _call(idx, seed, tag, it, chain)
    return float(uniforms_from_words(w[0], w[1]))


def gamma_draw(alpha: float, seed: int, tag: int, it: int, chain: int):
    """Gamma(alpha, 1) by Marsaglia-Tsang; returns (value, attempts used)."""
    if not alpha >= 1.0:
        raise ValueError("alpha must be >= 1")
    d = alpha - 1.0 / 3.0
    c = 1.0 / math.sqrt(9.0 * d)
    for t in range(GAMMA_MAX_ATTEMPTS):
        z = scalar_normal(2 * t, seed, tag, it, chain)
        u = scalar_uniform(2 * t + 1, seed, tag, it, chain)
        v = 1.0 + c * z
        if v <= 0.0:
            continue
        v = v * v * v
        if math.log(u) < 0.5 * z * z + d - d * v + d * math.log(v):
            return d * v, t + 1
    return d, GAMMA_MAX_ATTEMPTS


def inv_gamma_draw(shape: float, scale: float, seed: int, tag: int, it: int, chain: int):
    """IG(shape, scale) = scale / Gamma(shape, 1)."""
    g, _ = gamma_draw(shape, seed, tag, it, chain)
    return scale / g
