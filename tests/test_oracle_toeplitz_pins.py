"""Pins of the oracle's Toeplitz hashing (the comparison scheme of Sec. 1 /
Table 1): z = T x over GF(2), T[i][j] = s[i - j + n - 1], s of n + r - 1 bits.
Checked against the matrix built explicitly (exhaustively on tiny sizes), a
carry-less product restated with Python integers, unit vectors, GF(2)
linearity, and the exact universal-hashing count: for x != 0 exactly
2^(n - 1) of the 2^(n + r - 1) seeds give T x = 0."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2105_13678_gb300 import synthetic


def _bits(words, nbits):
    v = oracle.words_to_int(words)
    return [(v >> t) & 1 for t in range(nbits)]


def _words(bits):
    v = 0
    for t, b in enumerate(bits):
        v |= (b & 1) << t
    return oracle.int_to_words(v, max(1, oracle.words(len(bits))))


def _matrix(s_bits, n, r):
    return np.array([[s_bits[i - j + n - 1] for j in range(n)] for i in range(r)], dtype=np.int64)


def test_exhaustive_tiny_against_explicit_matrix():
    for n, r in ((1, 1), (3, 2), (4, 3), (5, 1), (2, 4)):
        for sv in range(1 << (n + r - 1)):
            s_bits = [(sv >> t) & 1 for t in range(n + r - 1)]
            T = _matrix(s_bits, n, r)
            for xv in range(1 << n):
                x_bits = [(xv >> t) & 1 for t in range(n)]
                want = (T @ np.array(x_bits)) % 2
                got = _bits(oracle.toeplitz(_words(x_bits), n, _words(s_bits), r), r)
                assert list(want) == got, (n, r, sv, xv)


def test_universal_count_is_exact():
    """Toeplitz hashing is a universal family: for every x != 0 exactly
    2^(n-1) seeds map x to 0 (probability 2^-r)."""
    for n, r in ((4, 2), (3, 3), (5, 2)):
        seeds = [_words([(sv >> t) & 1 for t in range(n + r - 1)]) for sv in range(1 << (n + r - 1))]
        for xv in range(1, 1 << n):
            x = _words([(xv >> t) & 1 for t in range(n)])
            zero = sum(1 for s in seeds if oracle.words_to_int(oracle.toeplitz(x, n, s, r)) == 0)
            assert zero == 1 << (n - 1), (n, r, xv, zero)


@pytest.mark.parametrize("n,r,seed_id", [(1000, 100, 1), (4097, 513, 2), (777, 1, 3), (64, 64, 4)])
def test_carryless_restatement(n, r, seed_id):
    """z_i = bit (i + n - 1) of the carry-less product of s and x (Python ints)."""
    key, seed = synthetic.block_inputs(seed_id, n, n + r - 1)
    S, Xv = oracle.words_to_int(seed), oracle.words_to_int(key)
    c = 0
    for j in range(n):
        if (Xv >> j) & 1:
            c ^= S << j
    want = (c >> (n - 1)) & ((1 << r) - 1)
    assert oracle.words_to_int(oracle.toeplitz(key, n, seed, r)) == want


def test_unit_vectors_read_columns_and_diagonals():
    n, r = 300, 70
    key, seed = synthetic.block_inputs(7, n, n + r - 1)
    s_bits = _bits(seed, n + r - 1)
    x_bits = _bits(key, n)
    for j in (0, 1, 150, n - 1):  # x = e_j: column j of T
        z = _bits(oracle.toeplitz(_words([int(t == j) for t in range(n)]), n, seed, r), r)
        assert z == [s_bits[i - j + n - 1] for i in range(r)]
    for m in (0, 5, n - 1, n + r - 2):  # s = e_m: one diagonal, z_i = x_(i + n - 1 - m)
        z = _bits(oracle.toeplitz(key, n, _words([int(t == m) for t in range(n + r - 1)]), r), r)
        want = [x_bits[i + n - 1 - m] if 0 <= i + n - 1 - m < n else 0 for i in range(r)]
        assert z == want


def test_gf2_linearity():
    n, r = 513, 97
    k1, s1 = synthetic.block_inputs(11, n, n + r - 1)
    k2, s2 = synthetic.block_inputs(12, n, n + r - 1)
    z = lambda k, s: oracle.words_to_int(oracle.toeplitz(k, n, s, r))  # noqa: E731
    assert z(k1 ^ k2, s1) == z(k1, s1) ^ z(k2, s1)
    assert z(k1, s1 ^ s2) == z(k1, s1) ^ z(k1, s2)


def test_selected_bits_equal_the_full_product():
    n, r = 3001, 777
    key, seed = synthetic.block_inputs(21, n, n + r - 1)
    full = _bits(oracle.toeplitz(key, n, seed, r), r)
    idx = [0, 1, 63, 64, 500, r - 1]
    assert list(oracle.toeplitz_bits(key, n, seed, r, idx)) == [full[i] for i in idx]
