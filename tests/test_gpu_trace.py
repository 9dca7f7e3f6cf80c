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
