"""pa_hash_noalloc: the hash for callers that cannot allocate device memory
(their device memory belongs to another allocator or pool, or an allocation and
the device synchronisation it may cause is not allowed where they run).

The entry point keeps every intermediate buffer in a static device array owned
by the library, so it must give exactly the bits of the regular plan-based
path, call after call, while the device's free memory stays unchanged.  This
file is collected last so that a failure here does not hide the other tests."""
import numpy as np
import pytest

import oracle
from paper_2105_13678_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _noalloc(n, r, key_t, seed_t, out_t, st_t, stream):
    from paper_2105_13678_gb300 import _lib
    p = _lib.params()
    return _lib.lib().pa_hash_noalloc(n, r, p, key_t.data_ptr(), seed_t.data_ptr(), out_t.data_ptr(),
                                      st_t.data_ptr(), stream)


def test_noalloc_matches_pa_hash_two_calls_in_a_row():
    import torch
    from paper_2105_13678_gb300 import _lib
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(1 << 20, 104858, 1), (3_000_017, 250_000, 2)]
    for n, r, seed_id in cases:
        plan = _lib.Plan(n, r)
        key, seed = synthetic.block_inputs(seed_id, n, (plan.k + 2) * plan.gamma)
        dk = torch.from_numpy(key.view(np.int64)).cuda()
        ds = torch.from_numpy(seed.view(np.int64)).cuda()
        ref = torch.zeros(plan.info.out_words, dtype=torch.int64, device="cuda")
        st_ref = torch.full((1,), -9, dtype=torch.int32, device="cuda")
        _lib.pa_hash(plan, dk.data_ptr(), ds.data_ptr(), ref.data_ptr(), st_ref.data_ptr(), stream)
        torch.cuda.synchronize()
        free_before = None
        for call in range(2):
            out = torch.full((plan.info.out_words,), -1, dtype=torch.int64, device="cuda")
            st = torch.full((1,), -9, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            if call == 1:
                free_before = torch.cuda.mem_get_info()[0]
            assert _noalloc(n, r, dk, ds, out, st, stream) == _lib.PA_OK
            torch.cuda.synchronize()
            if call == 1:
                assert torch.cuda.mem_get_info()[0] == free_before
            assert int(st.item()) == int(st_ref.item()) == 0
            assert torch.equal(out, ref), f"call {call}: pa_hash_noalloc differs from pa_hash (n={n}, r={r})"
        plan.close()


def test_noalloc_rejects_blocks_beyond_the_static_scratch():
    import torch
    from paper_2105_13678_gb300 import _lib
    n, r = 260_000_000, 26_000_000
    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = _noalloc(n, r, dummy, dummy, dummy, st, torch.cuda.current_stream().cuda_stream)
    assert rc == _lib.PA_ERR_UNSUPPORTED


def test_noalloc_matches_oracle_and_reports_reload():
    """The same entry point against the oracle directly, at a ragged size, and
    on a key whose second slice is all ones (Algorithm 1's reload rule: status
    1 and a zero-filled output), on two calls in a row each."""
    import torch
    from paper_2105_13678_gb300 import _lib
    stream = torch.cuda.current_stream().cuda_stream
    n, r = 1_234_567, 99_999
    g, k = oracle.plan(n, r)
    key, seed = synthetic.block_inputs(31, n, (k + 2) * g)
    reload_key = oracle.int_to_words(oracle.words_to_int(key) | (((1 << g) - 1) << g), key.size)
    for kw, want_rc in ((key, oracle.ORA_OK), (reload_key, oracle.ORA_RELOAD)):
        rc, ref, _ = oracle.pa_hash(kw, n, seed, r, g, k)
        assert rc == want_rc
        dk = torch.from_numpy(kw.view(np.int64)).cuda()
        ds = torch.from_numpy(seed.view(np.int64)).cuda()
        for call in range(2):
            out = torch.full((oracle.words(r),), -1, dtype=torch.int64, device="cuda")
            st = torch.full((1,), -9, dtype=torch.int32, device="cuda")
            assert _noalloc(n, r, dk, ds, out, st, stream) == _lib.PA_OK
            torch.cuda.synchronize()
            assert int(st.item()) == rc, f"call {call}: status {int(st.item())}, oracle {rc}"
            assert np.array_equal(out.cpu().numpy().view(np.uint64), ref), f"call {call}: output differs from the oracle"
