"""Toeplitz-hashing comparison scheme on the GPU (pa_toeplitz_plan): bit-exact
against the oracle's z = T x over GF(2) -- in full where the oracle's O(n r)
loop is quick, on sampled output bits at larger sizes -- across output blocks,
key segments, ragged n and r, and the transform sizes of both column kernels;
plus properties that hold at any size (unit key vectors read a column of T,
GF(2) linearity)."""
import numpy as np
import pytest

import oracle
from paper_2105_13678_gb300 import synthetic

from helpers import dev, host

pytestmark = pytest.mark.gpu


def _run(plan, key, seed):
    import torch
    from paper_2105_13678_gb300 import _lib
    out = torch.full((plan.info.out_words,), -1, dtype=torch.int64, device="cuda")
    st = torch.full((1,), -9, dtype=torch.int32, device="cuda")
    dk, ds = dev(key), dev(seed)  # held until the hash has run
    _lib.pa_hash(plan, dk.data_ptr(), ds.data_ptr(), out.data_ptr(), st.data_ptr(),
                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return host(out)


@pytest.mark.parametrize("n,r,block_log,seed_id", [
    (1000, 100, 6, 1), (5000, 700, 7, 2), (20011, 3001, 10, 3), (4096, 4096, 8, 4),
    (65536, 1000, 0, 5), (100_000, 2_000, 9, 6), (777, 1, 6, 7)])
def test_toeplitz_matches_oracle(n, r, block_log, seed_id):
    from paper_2105_13678_gb300 import _lib
    plan = _lib.Plan(n, r, toeplitz=True, block_log=block_log)
    key, seed = synthetic.block_inputs(seed_id, n, n + r - 1)
    got = _run(plan, key, seed)
    plan.close()
    assert np.array_equal(got, oracle.toeplitz(key, n, seed, r))


@pytest.mark.parametrize("n,r,block_log", [(3 * (1 << 18) + 123, (1 << 18) - 77, 18), (1 << 21, 300_000, 19)])
def test_toeplitz_large_transforms_sampled(n, r, block_log):
    """Transforms of 2^20 and 2^21 (the production column kernel): sampled
    output bits against the oracle, unit key vectors against T's columns, and
    linearity over GF(2)."""
    import torch
    from paper_2105_13678_gb300 import _lib
    plan = _lib.Plan(n, r, toeplitz=True, block_log=block_log)
    key, seed = synthetic.block_inputs(31, n, n + r - 1)
    z = _run(plan, key, seed)
    zb = np.unpackbits(z.view(np.uint8), bitorder="little")[:r]
    rng = np.random.default_rng(3)
    idx = np.unique(np.concatenate([[0, 1, r - 1, min(r - 1, (1 << block_log) - 1), min(r - 1, 1 << block_log)],
                                    rng.integers(0, r, 40)]))
    assert np.array_equal(zb[idx], oracle.toeplitz_bits(key, n, seed, r, idx))
    sb = np.unpackbits(seed.view(np.uint8), bitorder="little")
    for j in (0, 1, n // 2, n - 1):
        e = np.zeros_like(key)
        e[j // 64] = np.uint64(1) << np.uint64(j % 64)
        col = np.unpackbits(_run(plan, e, seed).view(np.uint8), bitorder="little")[:r]
        assert np.array_equal(col, sb[np.arange(r) - j + n - 1]), j
    key2, _ = synthetic.block_inputs(32, n, 64)
    z2 = _run(plan, key2, seed)
    z12 = _run(plan, key ^ key2, seed)
    assert np.array_equal(z12, z ^ z2)
    plan.close()
