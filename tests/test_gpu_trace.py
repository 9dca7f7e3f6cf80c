"""Per-kernel tracing (pa_trace_enable / pa_trace_select / pa_trace_collect)."""
import numpy as np
import pytest

from paper_2105_13678_gb300 import synthetic

from helpers import dev

pytestmark = pytest.mark.gpu


def _run(plan, key, seed, times=2):
    import torch
    from paper_2105_13678_gb300 import _lib
    dk, ds = dev(key), dev(seed)
    out = torch.zeros(plan.info.out_words, dtype=torch.int64, device="cuda")
    for _ in range(times):
        _lib.pa_hash(plan, dk.data_ptr(), ds.data_ptr(), out.data_ptr(), 0, 0)
    torch.cuda.synchronize()


@pytest.mark.parametrize("backend", [1, 2])
def test_trace_all_and_selected(backend):
    from paper_2105_13678_gb300 import _lib
    n, r = 2_000_003, 200_000
    plan = _lib.Plan(n, r, backend=backend)
    key, seed = synthetic.block_inputs(17, n, (plan.k + 2) * plan.gamma)
    _lib.trace_enable(True)
    _run(plan, key, seed)
    full = _lib.trace_collect()
    _lib.trace_enable(False)
    assert full and all(v[0] == 2 and v[1] > 0 for v in full.values())
    assert any(name.startswith("mmh.") for name in full) and any(name.startswith("mh.") for name in full)
    name = max(full.items(), key=lambda kv: kv[1][1])[0]
    _lib.trace_select(name)
    _lib.trace_enable(True)
    _run(plan, key, seed, times=3)
    sel = _lib.trace_collect()
    _lib.trace_enable(False)
    _lib.trace_select(None)
    assert list(sel) == [name] and sel[name][0] == 3
    plan.close()


def test_eq4_seed_transforms_beside_eq2():
    """Three-prime blocks with Eq. 4 transforms of 2^20 or 2^21 transform b on
    the plan's side stream (traced as mh_b.*, once per block) and y alone in
    Eq. 4, whose row pass multiplies by b's stored spectrum; the output is the
    one of the same block hashed through seed reuse, where b's spectrum comes
    from pa_seed_prepare."""
    import torch
    from paper_2105_13678_gb300 import _lib
    n, r = 100_000_000, 10_000_000
    plan = _lib.Plan(n, r, backend=2)
    assert plan.info.mh_len in (1 << 20, 1 << 21)
    key, seed = synthetic.block_inputs(18, n, (plan.k + 2) * plan.gamma)
    _lib.trace_enable(True)
    _run(plan, key, seed)
    tr = _lib.trace_collect()
    _lib.trace_enable(False)
    assert tr["mh_b.p3_fwd_col"][0] == 2 and tr["mh_b.p3_row_store"][0] == 2, tr
    assert tr["mh.p3_fwd_col"][0] == 2 and tr["mh.p3_row_mac"][0] == 2, tr
    dk, ds = dev(key), dev(seed)
    sp = torch.cuda.current_stream().cuda_stream
    o1 = torch.zeros(plan.info.out_words, dtype=torch.int64, device="cuda")
    o2 = torch.zeros_like(o1)
    _lib.pa_hash(plan, dk.data_ptr(), ds.data_ptr(), o1.data_ptr(), 0, sp)
    _lib.pa_seed_prepare(plan, ds.data_ptr(), sp)
    _lib.pa_hash_prepared(plan, dk.data_ptr(), o2.data_ptr(), 0, sp)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)
    plan.close()
