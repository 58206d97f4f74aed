"""Known-answer pin of the oracle's Philox4x32-10 against an independent
implementation: the cuRAND header function curand_Philox4x32_10 (counter,
key), which implements Salmon et al.'s generator (SC'11) and which
tests/curand_philox_kat.cu compiles as host code and calls.  A swapped output
word, a wrong hi/lo pairing, a dropped round or a wrong key schedule in
oracle/rng.philox4x32_10 changes the output words and fails here.

Counters and keys: all zeros, all ones, the first 192 bits of the hexadecimal
expansion of pi (computed here, not typed), and 2000 random ones.  Needs nvcc
(host compilation only, no GPU).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import rng

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def curand_philox(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("kat") / "philox_kat")
    res = subprocess.run([nvcc, "-std=c++17", "-o", exe, os.path.join(HERE, "curand_philox_kat.cu")],
                         capture_output=True, text=True)
    if res.returncode != 0:
        pytest.skip(f"cannot compile the cuRAND known-answer helper: {res.stderr[-400:]}")

    def run(rows):
        text = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
        return np.array([[int(t) for t in line.split()] for line in out.strip().splitlines()], dtype=np.uint64)

    return run


def _arctan_inv(x, one):
    """one * atan(1/x) for an integer x > 1 by its alternating series (integers only)."""
    total = term = one // x
    x2, k, sign = x * x, 1, -1
    while term:
        term //= x2
        total += sign * (term // (2 * k + 1))
        sign, k = -sign, k + 1
    return total


def _pi_hex_words(count):
    """The first `count` 32-bit words of the fractional hexadecimal expansion of
    pi, from Machin's formula pi = 16 atan(1/5) - 4 atan(1/239) in integers."""
    guard = 64
    one = 1 << (32 * count + guard)
    pi = 16 * _arctan_inv(5, one) - 4 * _arctan_inv(239, one)
    frac = (pi - 3 * one) >> guard
    return [(frac >> (32 * (count - 1 - i))) & 0xFFFFFFFF for i in range(count)]


def _oracle(rows):
    rows = np.asarray(rows, dtype=np.uint64)
    out = np.empty((len(rows), 4), dtype=np.uint64)
    for i, r in enumerate(rows):
        out[i] = rng.philox4x32_10([r[:4]], (int(r[4]), int(r[5])))[0]
    return out


def test_pi_words_are_the_known_expansion():
    # 3.243F6A88 85A308D3 ... : the leading word of pi's hexadecimal fraction
    assert _pi_hex_words(1)[0] == 0x243F6A88


def test_philox_known_answers_special_counters(curand_philox):
    m = 0xFFFFFFFF
    pi = _pi_hex_words(6)
    rows = [[0, 0, 0, 0, 0, 0], [m, m, m, m, m, m], pi]
    assert np.array_equal(_oracle(rows), curand_philox(rows))


def test_philox_known_answers_random_counters_and_keys(curand_philox):
    g = np.random.default_rng(123)
    rows = g.integers(0, 2 ** 32, size=(2000, 6), dtype=np.uint64)
    rows[:50, 4:] = 0            # zero key, varied counters
    rows[50:100, :4] = 0         # zero counter, varied keys
    rows[100:150, 1:4] = 0       # only word 0 varies (the sampler's element index)
    assert np.array_equal(_oracle(rows), curand_philox(rows))


def test_sampler_counter_layout_matches_the_known_answer(curand_philox):
    # the stream words the sampler feeds Philox: (pair index, tag, iteration, chain), key = seed (lo, hi)
    seed = 0x123456789ABCDEF0
    k0, k1 = rng.key_of(seed)
    rows = [[q, tag, 7, 3, k0, k1] for q in range(8) for tag in range(6)]
    ref = curand_philox(rows)
    for row, want in zip(rows, ref):
        got = rng._call(row[0], seed, row[1], 7, 3)
        assert [int(v) for v in got] == [int(v) for v in want]
