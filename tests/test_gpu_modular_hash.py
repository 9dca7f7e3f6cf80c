"""The comparison scheme: modular-arithmetic-hash PA over the whole key
(Eq. 4 with alpha = n), bit-exact against the oracle's Eq. 4 with the key as
the hash input."""
import numpy as np
import pytest

import oracle
from paper_2105_13678_gb300 import synthetic

from helpers import dev, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,r", [(64, 5), (1000, 100), (1 << 16, 6554), (1_000_003, 100_000), (20_000_000, 2_000_000)])
def test_modular_hash_matches_oracle(n, r):
    import torch
    from paper_2105_13678_gb300 import _lib
    plan = _lib.Plan(n, r, modular_hash=True)
    assert plan.gamma == n and plan.k == 0 and plan.info.seed_words == (2 * n + 63) // 64
    key, seed = synthetic.block_inputs(n % 1000 + 17, n, 2 * n)
    dk, ds = dev(key), dev(seed)
    out = torch.zeros(plan.info.out_words, dtype=torch.int64, device="cuda")
    st = torch.full((1,), -9, dtype=torch.int32, device="cuda")
    _lib.pa_hash(plan, dk.data_ptr(), ds.data_ptr(), out.data_ptr(), st.data_ptr())
    torch.cuda.synchronize()
    ref = oracle.mh(key, seed, n, 0, r)   # Eq. 4 with y = x, b = seed[0, n), c = seed[n, 2n)
    assert int(st.item()) == 0 and np.array_equal(host(out), ref)
    with pytest.raises(_lib.PAError):
        _lib.pa_seed_prepare(plan, ds.data_ptr())
    plan.close()
