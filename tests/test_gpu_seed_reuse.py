"""Seed reuse (pa_seed_prepare + pa_hash_prepared): the same output bits as
pa_hash for every key hashed with a prepared seed, and as the oracle, on both
transform backends."""
import numpy as np
import pytest

import oracle
from paper_2105_13678_gb300 import synthetic

from helpers import dev, gpu_hash, host

pytestmark = pytest.mark.gpu

GOLDILOCKS, P3 = 1, 2


def _plan_or_skip(n, r, gamma, backend):
    from paper_2105_13678_gb300 import _lib
    try:
        return _lib.Plan(n, r, gamma=gamma, backend=backend)
    except _lib.PAError as e:
        assert backend == P3 and e.code == -7  # three-prime sizes not feasible
        pytest.skip("three-prime transform not feasible at these sizes")


def _prepared(plan, dk):
    import torch
    from paper_2105_13678_gb300 import _lib
    out = torch.zeros(plan.info.out_words, dtype=torch.int64, device="cuda")
    st = torch.full((1,), -9, dtype=torch.int32, device="cuda")
    _lib.pa_hash_prepared(plan, dk.data_ptr(), out.data_ptr(), st.data_ptr(),
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return int(st.item()), host(out)


def _prepare(plan, seed):
    import torch
    from paper_2105_13678_gb300 import _lib
    ds = dev(seed)
    _lib.pa_seed_prepare(plan, ds.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()


@pytest.mark.parametrize("backend", [GOLDILOCKS, P3])
@pytest.mark.parametrize("n,r,gamma", [(1 << 20, 104858, 0), (3_000_000, 300_000, 0), (40 * 61 + 3, 20, 61),
                                       (10_000_000, 1_000_000, 0), (5 * 9689, 100, 9689)])
def test_prepared_matches_plain_for_several_keys(n, r, gamma, backend):
    plan = _plan_or_skip(n, r, gamma, backend)
    g, k = plan.gamma, plan.k
    _, seed = synthetic.block_inputs(100 + n % 97, n, (k + 2) * g)
    _prepare(plan, seed)
    for key_id in range(3):
        key, _ = synthetic.block_inputs(7000 + key_id, n, 64)
        st, out = _prepared(plan, dev(key))
        s2, plain, _, _ = gpu_hash(plan, key, seed)
        assert st == s2
        assert np.array_equal(out, plain)
        if key_id == 0:
            rc, ref, _ = oracle.pa_hash(key, n, seed, r, g, k)
            assert rc == s2 and np.array_equal(plain, ref)
    plan.close()


@pytest.mark.parametrize("backend,n,logc", [(GOLDILOCKS, 260_000_000, None), (P3, 260_000_000, 11),
                                             (P3, 500_000_000, 12), (P3, 600_000_000, 13), (P3, 1_000_000_000, 14)])
def test_prepared_at_paper_scale(backend, n, logc):
    """r = 0.1 n (n = 2.6e8: gamma = 30402457, k = 9), and on the three-prime
    plan row lengths 2^11 .. 2^14 (the 2^14 rows hold 16 accumulators per
    thread): prepared output equals the plain path's, whose parity with the
    oracle the paper-scale parity tests hold; a second seed replaces the
    first."""
    r = n // 10
    plan = _plan_or_skip(n, r, 0, backend)
    if logc is not None:
        assert plan.geometry(0)[1] == logc
    g, k = plan.gamma, plan.k
    key, seed = synthetic.block_inputs(2, n, (k + 2) * g)
    _, seed2 = synthetic.block_inputs(12, n, (k + 2) * g)
    dk = dev(key)
    for sd in (seed, seed2):
        _prepare(plan, sd)
        st, out = _prepared(plan, dk)
        s2, plain, _, _ = gpu_hash(plan, key, sd)
        assert st == s2 == 0
        assert np.array_equal(out, plain)
    plan.close()


@pytest.mark.parametrize("backend", [GOLDILOCKS, P3])
def test_prepared_reload_and_zero_mmh_value(backend):
    """An all-ones key slice gives the reload status and a zero output; a seed
    with a = 0 gives y = 0, so the output is the top bits of c."""
    n, r, gamma = 4 * 44497, 1000, 44497
    plan = _plan_or_skip(n, r, gamma, backend)
    k = plan.k
    key, seed = synthetic.block_inputs(31, n, (k + 2) * gamma)
    kv = oracle.words_to_int(key) | (((1 << gamma) - 1) << gamma)  # slice x_2 all ones
    ones_key = oracle.int_to_words(kv, key.size)
    _prepare(plan, seed)
    st, out = _prepared(plan, dev(ones_key))
    assert st == oracle.ORA_RELOAD and not out.any()
    sv = oracle.words_to_int(seed) & ~((1 << (k * gamma)) - 1)  # a_1..a_k = 0
    zseed = oracle.int_to_words(sv, seed.size)
    _prepare(plan, zseed)
    st, out = _prepared(plan, dev(key))
    rc, ref, y = oracle.pa_hash(key, n, zseed, r, gamma, k)
    assert rc == st == 0 and not y.any()
    assert np.array_equal(out, ref)
    plan.close()


def test_prepared_requires_prepare():
    import torch
    from paper_2105_13678_gb300 import _lib
    for backend in (GOLDILOCKS, P3):
        plan = _lib.Plan(1 << 20, 104858, backend=backend)
        buf = torch.zeros(plan.info.key_words + 8, dtype=torch.int64, device="cuda")
        with pytest.raises(_lib.PAError):
            _lib.pa_hash_prepared(plan, buf.data_ptr(), buf.data_ptr())
        plan.close()
