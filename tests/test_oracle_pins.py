"""Pins for the CPU oracle (``oracle/``) against facts that do not come from
the oracle's own code: library routines (CPython big-integer ``*`` and ``%``),
closed forms (the exact MMH collision count of Eq. 2), invariants (MMH
linearity, MH shift-equivariance in c), brute force of Algorithm 1 from Eq. 2
and Eq. 4 on tiny inputs (every key at gamma <= 7), textbook primality tests of
the Mersenne table, and the parameter points printed in the paper (Table 3).

A plausible slip anywhere in the oracle (a dropped carry, a wrong bit offset,
a transposed seed slice, a missing final reduction) fails at least one check.
"""
import os
import random

import numpy as np
import pytest

import oracle
from paper_2105_13678_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ints_to_bits(values, width):
    """Concatenate integers of ``width`` bits LSB-first into u64 words."""
    acc = 0
    for i, v in enumerate(values):
        acc |= int(v) << (i * width)
    nbits = max(1, len(values) * width)
    return oracle.int_to_words(acc, oracle.words(nbits) + 1)


def _lucas_lehmer(p):
    if p == 2:
        return True
    m = (1 << p) - 1
    s = 4
    for _ in range(p - 2):
        s = (s * s - 2) % m
    return s == 0


def _is_prime(q):
    if q < 2:
        return False
    i = 2
    while i * i <= q:
        if q % i == 0:
            return False
        i += 1
    return True


# ------------------------------------------------------------ Mersenne table
def test_mersenne_table_matches_lucas_lehmer():
    """Every prime exponent up to 2281 is in the table iff 2^p - 1 is prime
    (Lucas-Lehmer, a textbook test independent of the table)."""
    table = oracle.mersenne_exponents()
    assert table == sorted(table) and len(table) == len(set(table)) == 52
    small = [p for p in range(2, 2282) if _is_prime(p) and _lucas_lehmer(p)]
    assert small == [e for e in table if e <= 2281]
    assert table[-1] == 136279841


# ------------------------------------------------------------- plan, Table 3
def _golden_table3():
    rows = []
    with open(os.path.join(GOLDEN, "table3_params.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, ratio, k, gamma, n = line.split()
            rows.append((name, float(ratio), int(k), int(gamma), int(n)))
    return rows


@pytest.mark.parametrize("row", _golden_table3(), ids=lambda r: r[0])
def test_plan_reproduces_table3(row):
    name, ratio, k_paper, gamma_paper, n = row
    r = int(np.floor(ratio * n))
    gamma, k = oracle.plan(n, r, margin=128)
    assert (gamma, k) == (gamma_paper, k_paper)
    assert k <= 1.0 / ratio          # Sec. 4: k <= 1 / compression ratio
    assert k * gamma == n            # the paper's points have no padding


def test_plan_config_sizes():
    # r = ceil(0.1 * 2^20) = 104858 -> smallest exponent >= r + 128 is 110503
    assert oracle.plan(1 << 20, 104858) == (110503, 10)
    assert oracle.plan(260_000_000, 26_000_000) == (30402457, 9)
    assert oracle.plan(260_000_000, 13_000_000) == (13466917, 20)
    assert oracle.plan(260_000_000, 78_000_000) == (82589933, 4)
    assert oracle.plan(1_000_000_000, 100_000_000) == (136279841, 8)
    with pytest.raises(ValueError):
        oracle.plan(10, 136279841)          # no exponent large enough
    with pytest.raises(ValueError):
        oracle.plan(100, 5, gamma=5)        # gamma must exceed r
    with pytest.raises(ValueError):
        oracle.plan(100, 3, gamma=11)       # 2^11 - 1 is not a Mersenne prime


# ------------------------------------------------ big-integer multiplication
@pytest.mark.parametrize("method", [0, 1])
def test_mul_matches_python(method):
    rng = random.Random(11)
    cases = [(0, 5), (1, 1), ((1 << 64) - 1, (1 << 64) - 1), ((1 << 4096) - 1, (1 << 4095) + 1)]
    for _ in range(60):
        a = rng.getrandbits(rng.randint(1, 9000))
        b = rng.getrandbits(rng.randint(1, 9000))
        cases.append((a, b))
    for a, b in cases:
        assert oracle.mul(a, b, method) == a * b


def test_karatsuba_deep_recursion_matches_python():
    rng = random.Random(12)
    try:
        oracle.set_karatsuba_threshold(4)
        for bits in (257, 1000, 64 * 37 + 5, 20000, 123457):
            a, b = rng.getrandbits(bits), rng.getrandbits(bits)
            assert oracle.mul(a, b, 1) == a * b
            a = (1 << bits) - 1
            assert oracle.mul(a, a, 1) == a * a
    finally:
        oracle.set_karatsuba_threshold(32)


def test_karatsuba_large_matches_python():
    rng = random.Random(13)
    a, b = rng.getrandbits(1 << 20), rng.getrandbits((1 << 20) - 77)
    assert oracle.mul(a, b, 1) == a * b


# ------------------------------------------------------ Mersenne reduction
@pytest.mark.parametrize("gamma", [2, 3, 5, 7, 13, 61, 127, 521, 4423, 110503])
def test_mod_mersenne_matches_python(gamma):
    rng = random.Random(gamma)
    p = (1 << gamma) - 1
    cases = [0, 1, p, p + 1, 2 * p, p - 1, p * p, (1 << (2 * gamma + 5)) - 1]
    cases += [rng.getrandbits(rng.randint(1, 2 * gamma + 6)) for _ in range(20)]
    for s in cases:
        assert oracle.mod_mersenne(s, gamma) == s % p


# ------------------------------------------------------------------- MMH
def _mmh_y(xs, as_, gamma):
    k = len(xs)
    key = _ints_to_bits(xs, gamma)
    seed = _ints_to_bits(list(as_) + [0, 0], gamma)
    rc, y = oracle.mmh(key, k * gamma, seed, gamma, k)
    return rc, oracle.words_to_int(y)


@pytest.mark.parametrize("gamma,k", [(5, 1), (7, 4), (61, 3), (127, 5), (521, 2)])
def test_mmh_unit_vector(gamma, k):
    """a = e_j selects segment j: g_a(x) = x_j (x_j < p)."""
    rng = random.Random(gamma * 100 + k)
    p = (1 << gamma) - 1
    xs = [rng.randrange(p) for _ in range(k)]
    for j in range(k):
        a = [0] * k
        a[j] = 1
        rc, y = _mmh_y(xs, a, gamma)
        assert rc == oracle.ORA_OK and y == xs[j]


@pytest.mark.parametrize("gamma,k", [(13, 3), (61, 7), (89, 2), (1279, 4)])
def test_mmh_linearity(gamma, k):
    """Eq. 2 is linear over Z_p in both the key and the seed."""
    rng = random.Random(gamma + k)
    p = (1 << gamma) - 1
    for _ in range(5):
        x = [rng.randrange(p) for _ in range(k)]
        x2 = [rng.randrange(p) for _ in range(k)]
        a = [rng.randrange(p) for _ in range(k)]
        a2 = [rng.randrange(p) for _ in range(k)]
        xs = [(u + v) % p for u, v in zip(x, x2)]
        as_ = [(u + v) % p for u, v in zip(a, a2)]
        y1, y2, y3 = _mmh_y(x, a, gamma)[1], _mmh_y(x2, a, gamma)[1], _mmh_y(xs, a, gamma)[1]
        assert (y1 + y2) % p == y3
        z1, z3 = _mmh_y(x, a2, gamma)[1], _mmh_y(x, as_, gamma)[1]
        assert (y1 + z1) % p == z3
        # scaling: g_{c a}(x) = c g_a(x)
        c = rng.randrange(p)
        assert _mmh_y(x, [(c * v) % p for v in a], gamma)[1] == (c * y1) % p


@pytest.mark.parametrize("gamma,k,pairs", [(3, 1, None), (3, 2, 40), (3, 3, 12), (5, 1, None), (5, 2, 10)])
def test_mmh_exact_collision_count(gamma, k, pairs):
    """Closed form for Eq. 2 (Halevi-Krawczyk; Appendix A definition): for
    x != x' in Z_p^k, exactly p^(k-1) of the p^k seeds a collide."""
    import itertools
    p = (1 << gamma) - 1
    keys = list(itertools.product(range(p), repeat=k))
    if pairs is None:
        pair_list = [(u, v) for i, u in enumerate(keys) for v in keys[i + 1:]]
    else:
        rng = random.Random(gamma * 7 + k)
        pair_list = []
        while len(pair_list) < pairs:
            u, v = rng.choice(keys), rng.choice(keys)
            if u != v:
                pair_list.append((u, v))
    seeds = list(itertools.product(range(p), repeat=k))
    for u, v in pair_list:
        hits = sum(1 for a in seeds if _mmh_y(u, a, gamma)[1] == _mmh_y(v, a, gamma)[1])
        assert hits == p ** (k - 1)


def test_mmh_all_ones_seed_slice_is_zero():
    """a_i in Z_p: the slice 2^gamma - 1 equals p, i.e. 0."""
    gamma, k = 13, 3
    p = (1 << gamma) - 1
    xs = [5, 77, 4000]
    assert _mmh_y(xs, [p, 9, 10], gamma)[1] == _mmh_y(xs, [0, 9, 10], gamma)[1] == (9 * 77 + 10 * 4000) % p


def test_reload_on_all_ones_segment():
    """Algorithm 1 reload rule: a key segment equal to 2^gamma - 1 forces a reload."""
    gamma, k, r = 61, 3, 20
    p = (1 << gamma) - 1
    key = _ints_to_bits([3, p, 9], gamma)
    seed = _ints_to_bits([1, 2, 3, 5, 7], gamma)
    rc, out, _ = oracle.pa_hash(key, k * gamma, seed, r, gamma, k)
    assert rc == oracle.ORA_RELOAD and not out.any()
    # the zero-padded last segment never triggers it: n < k * gamma
    key = _ints_to_bits([3, 4, p], gamma)
    rc, _, _ = oracle.pa_hash(key, k * gamma - 1, seed, r, gamma, k)
    assert rc == oracle.ORA_OK


# -------------------------------------------------------------------- MH
def _mh_z(y, b, c, gamma, r):
    seed = _ints_to_bits([b, c], gamma)   # k = 0: b, c are the first two slices
    out = oracle.mh(oracle.int_to_words(y, oracle.words(gamma)), seed, gamma, 0, r)
    return oracle.words_to_int(out)


@pytest.mark.parametrize("gamma", [7, 61, 127, 4423])
def test_mh_identity_seed_takes_top_bits(gamma):
    """b = 1, c = 0: Eq. 4 reduces to z = floor(y / 2^(gamma - beta))."""
    rng = random.Random(gamma)
    for r in {1, gamma // 2, gamma - 1}:
        y = rng.getrandbits(gamma) % ((1 << gamma) - 1)
        assert _mh_z(y, 1, 0, gamma, r) == y >> (gamma - r)


@pytest.mark.parametrize("gamma", [7, 61, 521, 4423])
def test_mh_shift_equivariance_in_c(gamma):
    """Adding m * 2^(gamma-beta) to c adds m to z modulo 2^beta, for any b, y."""
    rng = random.Random(gamma + 1)
    for r in (1, 3, gamma - 2):
        y = rng.getrandbits(gamma) % ((1 << gamma) - 1)
        b = rng.getrandbits(gamma) | 1
        c = rng.getrandbits(gamma)
        z0 = _mh_z(y, b, c, gamma, r)
        for m in (1, 2, 5):
            c2 = (c + m * (1 << (gamma - r))) % (1 << gamma)
            assert _mh_z(y, b, c2, gamma, r) == (z0 + m) % (1 << r)


def test_mh_forces_b_odd():
    """gcd(b, 2) = 1: an even b in the seed acts as b + 1."""
    gamma, r = 61, 30
    rng = random.Random(5)
    y, c = rng.getrandbits(60), rng.getrandbits(61)
    b = rng.getrandbits(61) & ~1
    assert _mh_z(y, b, c, gamma, r) == _mh_z(y, b | 1, c, gamma, r)


@pytest.mark.parametrize("gamma", [3, 5])
def test_mh_collision_bound(gamma):
    """Measured collision probability of Eq. 4 over all (b odd, c), every pair
    y != y', versus the multiply-add-shift bound 2^(1-beta) (Dietzfelbinger
    et al., 1997).  The paper's tighter 2^-beta is recorded, not assumed."""
    size = 1 << gamma
    seeds = [(b, c) for b in range(1, size, 2) for c in range(size)]
    ys = range(0, size - 1)
    for r in range(1, gamma):
        table = np.array([[_mh_z(y, b, c, gamma, r) for b, c in seeds] for y in ys])
        worst = 0.0
        for i in range(len(ys)):
            hits = (table[i + 1:] == table[i]).mean(axis=1) if i + 1 < len(ys) else np.zeros(1)
            worst = max(worst, float(hits.max()))
        assert worst <= 2.0 ** (1 - r) + 1e-12


# ------------------------------------------------------- whole Algorithm 1
def test_pa_hash_is_mh_of_mmh_and_ignores_bits_past_n():
    n, r = 5000, 300
    gamma, k = oracle.plan(n, r)
    key, seed = synthetic.block_inputs(3, n, (k + 2) * gamma)
    rc, out, y = oracle.pa_hash(key, n, seed, r, gamma, k)
    assert rc == oracle.ORA_OK
    rc2, y2 = oracle.mmh(key, n, seed, gamma, k)
    assert rc2 == oracle.ORA_OK and np.array_equal(y, y2)
    assert np.array_equal(out, oracle.mh(y, seed, gamma, k, r))
    dirty = key.copy()
    dirty[-1] |= np.uint64(0xFFFF) << np.uint64(48)       # bits at and past n are not key bits
    assert n % 64 <= 48
    assert np.array_equal(oracle.pa_hash(dirty, n, seed, r, gamma, k)[1], out)
    assert out.size == (r + 63) // 64
    assert int(out[-1]) >> (r % 64) == 0       # bits past r are zero


def _algorithm1_direct(key_int, n, seed_int, r, gamma, k):
    """Algorithm 1 evaluated from Eq. 2 and Eq. 4 on Python integers, slice by
    slice (brute force for tiny sizes)."""
    mask, p = (1 << gamma) - 1, (1 << gamma) - 1
    key_int &= (1 << n) - 1
    xs = [(key_int >> (i * gamma)) & mask for i in range(k)]
    if any(x == p for x in xs):
        return oracle.ORA_RELOAD, 0
    sl = [(seed_int >> (i * gamma)) & mask for i in range(k + 2)]
    y = sum((a % p) * x for a, x in zip(sl[:k], xs)) % p
    t = ((sl[k] | 1) * y + sl[k + 1]) % (1 << gamma)
    return oracle.ORA_OK, t >> (gamma - r)


@pytest.mark.parametrize("gamma,k", [(2, 1), (2, 2), (3, 1), (3, 2), (5, 1), (5, 2), (7, 1), (7, 2)])
def test_algorithm1_exhaustive_over_keys_tiny(gamma, k):
    """Brute force: every key of n = k gamma and n = k gamma - 1 bits, every
    beta < gamma, three seeds; the oracle's status and output bits equal the
    direct evaluation (reload included)."""
    rng = random.Random(gamma * 31 + k)
    for n in {k * gamma, k * gamma - 1} - {0}:
        for _ in range(3):
            seed_int = rng.getrandbits((k + 2) * gamma)
            seed = oracle.int_to_words(seed_int, oracle.words((k + 2) * gamma) + 1)
            for r in range(1, gamma):
                for key_int in range(1 << n):
                    key = oracle.int_to_words(key_int, oracle.words(n) + 1)
                    rc, out, _ = oracle.pa_hash(key, n, seed, r, gamma, k)
                    want_rc, want = _algorithm1_direct(key_int, n, seed_int, r, gamma, k)
                    assert rc == want_rc
                    assert oracle.words_to_int(out) == want


@pytest.mark.parametrize("gamma,k", [(13, 16), (17, 5), (19, 9), (31, 16), (61, 12), (89, 3), (607, 7)])
def test_algorithm1_random_keys_small(gamma, k):
    """The same direct evaluation on random keys, seeds and output lengths at
    the small Mersenne exponents, ragged n included."""
    rng = random.Random(gamma + 1000 * k)
    for _ in range(20):
        n = rng.randrange((k - 1) * gamma + 1, k * gamma + 1)
        r = rng.randrange(1, gamma)
        key_int = rng.getrandbits(n)
        seed_int = rng.getrandbits((k + 2) * gamma)
        key = oracle.int_to_words(key_int, oracle.words(n) + 1)
        seed = oracle.int_to_words(seed_int, oracle.words((k + 2) * gamma) + 1)
        rc, out, _ = oracle.pa_hash(key, n, seed, r, gamma, k)
        want_rc, want = _algorithm1_direct(key_int, n, seed_int, r, gamma, k)
        assert rc == want_rc and oracle.words_to_int(out) == want


def test_pa_hash_output_is_not_trivial():
    """Uniform inputs give an output with about r/2 ones and a 0.5 bit balance."""
    n, r = 1 << 16, 6554
    gamma, k = oracle.plan(n, r)
    key, seed = synthetic.block_inputs(1, n, (k + 2) * gamma)
    _, out, _ = oracle.pa_hash(key, n, seed, r, gamma, k)
    ones = sum(bin(int(w)).count("1") for w in out)
    assert abs(ones - r / 2) < 5 * (r ** 0.5) / 2


def test_composite_collision_bound_lemma2():
    """Lemma 2: the composition MMH -> MH is (delta_g + delta_h)-universal.
    Exhaustive over keys and seeds at gamma = 3, k = 2 (delta_g = 1/7 exactly,
    delta_h measured as in test_mh_collision_bound)."""
    import itertools
    gamma, k = 3, 2
    p = (1 << gamma) - 1
    size = 1 << gamma
    keys = list(itertools.product(range(p), repeat=k))
    mh_seeds = [(b, c) for b in range(1, size, 2) for c in range(size)]
    a_seeds = list(itertools.product(range(p), repeat=k))
    for r in (1, 2):
        # delta_h measured over all y != y' in Z_p
        zt = np.array([[_mh_z(y, b, c, gamma, r) for b, c in mh_seeds] for y in range(p)])
        delta_h = max(float((zt[i] == zt[j]).mean()) for i in range(p) for j in range(i + 1, p))
        # y table for every key and every a
        yt = np.array([[_mmh_y(x, a, gamma)[1] for a in a_seeds] for x in keys])
        worst = 0.0
        rng = random.Random(r)
        for _ in range(60):
            i, j = rng.sample(range(len(keys)), 2)
            # Pr over (a, b, c) of equal outputs = mean over a of Pr_(b,c)[z(y_i) = z(y_j)]
            pr = np.mean([(zt[yi] == zt[yj]).mean() for yi, yj in zip(yt[i], yt[j])])
            worst = max(worst, float(pr))
        assert worst <= 1.0 / p + delta_h + 1e-12
