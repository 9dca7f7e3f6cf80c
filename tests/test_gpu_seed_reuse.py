"""Seed reuse (pa_seed_prepare + pa_hash_prepared): the same output bits as
pa_hash for every key hashed with a prepared seed, and as the oracle."""
import numpy as np
import pytest

import oracle
from paper_2105_13678_gb300 import synthetic

from helpers import dev, gpu_hash, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,r,gamma", [(1 << 20, 104858, 0), (3_000_000, 300_000, 0), (40 * 61 + 3, 20, 61),
                                       (10_000_000, 1_000_000, 0), (5 * 9689, 100, 9689)])
def test_prepared_matches_plain_for_several_keys(n, r, gamma):
    import torch
    from paper_2105_13678_gb300 import _lib
    plan = _lib.Plan(n, r, gamma=gamma, backend=_lib.BACKEND_GOLDILOCKS)
    g, k = plan.gamma, plan.k
    _, seed = synthetic.block_inputs(100 + n % 97, n, (k + 2) * g)
    ds = dev(seed)
    sp = torch.cuda.current_stream().cuda_stream
    _lib.pa_seed_prepare(plan, ds.data_ptr(), sp)
    for key_id in range(3):
        key, _ = synthetic.block_inputs(7000 + key_id, n, 64)
        dk = dev(key)
        out = torch.zeros(plan.info.out_words, dtype=torch.int64, device="cuda")
        st = torch.full((1,), -9, dtype=torch.int32, device="cuda")
        _lib.pa_hash_prepared(plan, dk.data_ptr(), out.data_ptr(), st.data_ptr(), sp)
        torch.cuda.synchronize()
        s2, plain, _, _ = gpu_hash(plan, key, seed)
        assert int(st.item()) == s2
        assert np.array_equal(host(out), plain)
        if key_id == 0:
            rc, ref, _ = oracle.pa_hash(key, n, seed, r, g, k)
            assert rc == s2 and np.array_equal(plain, ref)
    plan.close()


def test_prepared_requires_prepare():
    import torch
    from paper_2105_13678_gb300 import _lib
    plan = _lib.Plan(1 << 16, 1000, backend=_lib.BACKEND_GOLDILOCKS)
    buf = torch.zeros(plan.info.key_words + 8, dtype=torch.int64, device="cuda")
    with pytest.raises(_lib.PAError):
        _lib.pa_hash_prepared(plan, buf.data_ptr(), buf.data_ptr())
    plan.close()


def test_three_prime_plans_refuse_seed_reuse():
    """Seed reuse exists for the Goldilocks transforms only."""
    import torch
    from paper_2105_13678_gb300 import _lib
    plan = _lib.Plan(1 << 20, 104858, backend=_lib.BACKEND_P3)
    seed = torch.zeros((plan.k + 2) * plan.gamma // 64 + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(_lib.PAError) as e:
        _lib.pa_seed_prepare(plan, seed.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -7
    plan.close()
