"""The parallel oracle drivers used by the paper-scale GPU parity tests
(tests/helpers.py) give exactly the single-threaded oracle's result: the
Eq. 2 sum split by segment and recombined mod p, then Eq. 4."""
import numpy as np

import oracle
from paper_2105_13678_gb300 import synthetic

from helpers import oracle_hash_many, oracle_hash_parallel


def _cases():
    out = []
    for i, (n, r) in enumerate([(5000, 600), (20_000, 3000), (1 << 16, 7000), (44497 * 3, 21000), (9000, 4300)]):
        g, k = oracle.plan(n, r)
        key, seed = synthetic.block_inputs(900 + i, n, (k + 2) * g)
        out.append((key, n, seed, r, g, k))
    # a block whose second slice is all ones: reload
    n, r = 3 * 607, 300
    g, k = oracle.plan(n, r)
    key, seed = synthetic.block_inputs(950, n, (k + 2) * g)
    v = oracle.words_to_int(key) | (((1 << g) - 1) << g)
    key = oracle.int_to_words(v, key.size)
    out.append((key, n, seed, r, g, k))
    return out


def test_oracle_hash_many_equals_single_threaded_oracle():
    cases = _cases()
    got = oracle_hash_many(cases, workers=4)
    for (key, n, seed, r, g, k), (rc, out) in zip(cases, got):
        rc0, out0, _ = oracle.pa_hash(key, n, seed, r, g, k)
        assert rc == rc0 and np.array_equal(out, out0)
    assert got[-1][0] == oracle.ORA_RELOAD


def test_oracle_hash_parallel_equals_single_threaded_oracle():
    for key, n, seed, r, g, k in _cases():
        rc0, out0, _ = oracle.pa_hash(key, n, seed, r, g, k)
        rc, out, _ = oracle_hash_parallel(key, n, seed, r, g, k, workers=3)
        assert rc == rc0 and np.array_equal(out, out0)
