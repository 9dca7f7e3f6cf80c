"""Error paths, exercised from the host without faulting the GPU: server
shutdown with queued jobs, bounded waits that expire, a full queue, and device
or pinned allocations made to fail by the library's host-side injection hook
(pa_debug_fail_allocs).  After each failure the next call must succeed and give
the right bits, and nothing may leak."""

import numpy as np
import pytest

import oracle
from paper_2105_13678_gb300 import synthetic

from helpers import dev, gpu_hash, host

pytestmark = pytest.mark.gpu


def _inputs(n, r, seed_id):
    g, k = oracle.plan(n, r)
    key, seed = synthetic.block_inputs(seed_id, n, (k + 2) * g)
    return g, k, key, seed


def _fail(skip, count):
    from paper_2105_13678_gb300 import _lib
    _lib.lib().pa_debug_fail_allocs(skip, count)


# ------------------------------------------------------------------ server
def test_serve_shutdown_cancels_queued_jobs():
    """One slot: the first job is being planned while the rest queue up;
    shutdown cancels the queued ones (status PA_ERR_CANCELLED), lets the
    admitted one finish with the right bits, and refuses later submits."""
    import torch
    from paper_2105_13678_gb300 import _lib
    n, r = 100_000_000, 10_000_000
    g, k, key, seed = _inputs(n, r, 401)
    dk, ds = dev(key), dev(seed)
    outs = [torch.full(((r + 63) // 64,), -1, dtype=torch.int64, device="cuda") for _ in range(12)]
    srv = _lib.Server(16 << 30, slots=1)
    tickets = [srv.submit(n, r, dk.data_ptr(), ds.data_ptr(), o.data_ptr()) for o in outs]
    srv.shutdown()
    sts = [srv.poll(t) for t in tickets]
    st = srv.stats()
    with pytest.raises(_lib.PAError) as ei:
        srv.submit(n, r, dk.data_ptr(), ds.data_ptr(), outs[0].data_ptr())
    assert ei.value.code == _lib.PA_ERR_CANCELLED
    srv.close()
    assert all(s in (_lib.PA_OK, _lib.PA_ERR_CANCELLED) for s in sts), sts
    assert sts.count(_lib.PA_ERR_CANCELLED) >= 1 and sts[0] == _lib.PA_OK
    assert st["completed"] + st["cancelled"] == len(tickets) and st["cancelled"] == sts.count(_lib.PA_ERR_CANCELLED)
    p = _lib.Plan(n, r)
    s0, ref, _, _ = gpu_hash(p, key, seed)
    p.close()
    for s, o in zip(sts, outs):
        if s == _lib.PA_OK:
            assert np.array_equal(host(o), ref)


def test_serve_wait_expires_then_completes():
    """pa_serve_wait with a timeout shorter than the job returns PA_ERR_TIMEOUT;
    waiting again returns the job's status."""
    import torch
    from paper_2105_13678_gb300 import _lib
    n, r = 260_000_000, 26_000_000
    g, k, key, seed = _inputs(n, r, 402)
    dk, ds = dev(key), dev(seed)
    o = torch.zeros((r + 63) // 64, dtype=torch.int64, device="cuda")
    srv = _lib.Server(16 << 30, slots=1)
    t = srv.submit(n, r, dk.data_ptr(), ds.data_ptr(), o.data_ptr())
    with pytest.raises(_lib.PAError) as ei:
        srv.wait(t, 1e-6)
    assert ei.value.code == _lib.PA_ERR_TIMEOUT
    assert srv.wait(t, 120.0) == _lib.PA_OK
    srv.close()


def test_serve_full_queue_is_busy():
    """max_queue = 2: submits beyond the queue's room return PA_ERR_BUSY; every
    accepted job still completes."""
    import torch
    from paper_2105_13678_gb300 import _lib
    n, r = 10_000_000, 1_000_000
    g, k, key, seed = _inputs(n, r, 403)
    dk, ds = dev(key), dev(seed)
    srv = _lib.Server(16 << 30, slots=1, max_queue=2)
    outs, tickets, busy = [], [], 0
    for _ in range(8):
        o = torch.zeros((r + 63) // 64, dtype=torch.int64, device="cuda")
        try:
            tickets.append(srv.submit(n, r, dk.data_ptr(), ds.data_ptr(), o.data_ptr()))
            outs.append(o)
        except _lib.PAError as e:
            assert e.code == _lib.PA_ERR_BUSY
            busy += 1
    assert busy >= 1 and len(tickets) >= 2
    assert all(srv.wait(t, 120.0) == _lib.PA_OK for t in tickets)
    srv.close()
    rc, ref, _ = oracle.pa_hash(key, n, seed, r, g, k)
    assert all(np.array_equal(host(o), ref) for o in outs)


# ------------------------------------------------------- allocation failures
@pytest.mark.parametrize("backend", [1, 2])
def test_plan_creation_fails_cleanly_at_every_allocation(backend):
    """The i-th device allocation of plan creation fails, for every i: the call
    returns PA_ERR_NOMEM, frees what it had, and the next plan works."""
    import torch
    from paper_2105_13678_gb300 import _lib
    n, r = 30_000_000, 3_000_000
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for i in range(200):
        _fail(i, 1)
        try:
            p = _lib.Plan(n, r, backend=backend)
        except _lib.PAError as e:
            assert e.code == _lib.PA_ERR_NOMEM, e
            failures += 1
            continue
        finally:
            _fail(0, 0)
        p.close()
        break
    else:
        pytest.fail("plan creation still failing after 200 allocations")
    assert failures >= 8
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (16 << 20), "plan creation leaked device memory"
    g, k, key, seed = _inputs(1 << 20, 104858, 404)
    p = _lib.Plan(1 << 20, 104858, backend=backend)
    s, out, _, _ = gpu_hash(p, key, seed)
    p.close()
    rc, ref, _ = oracle.pa_hash(key, 1 << 20, seed, 104858, g, k)
    assert s == rc == 0 and np.array_equal(out, ref)


@pytest.mark.parametrize("backend", [1, 2])
@pytest.mark.parametrize("skip", [0, 1, 2])
def test_seed_prepare_retries_after_failed_allocation(backend, skip):
    """One of the seed-reuse buffers cannot be allocated: pa_seed_prepare
    returns PA_ERR_NOMEM and the plan has no prepared seed; the next call
    allocates the rest and pa_hash_prepared gives pa_hash's bits."""
    import torch
    from paper_2105_13678_gb300 import _lib
    n, r = 3_000_017, 250_000
    p = _lib.Plan(n, r, backend=backend)
    g, k, key, seed = _inputs(n, r, 405)
    dk, ds = dev(key), dev(seed)
    sp = torch.cuda.current_stream().cuda_stream
    _fail(skip, 1)
    try:
        rc = _lib.lib().pa_seed_prepare(p.handle, ds.data_ptr(), sp)
    finally:
        _fail(0, 0)
    assert rc == _lib.PA_ERR_NOMEM
    o = torch.zeros(p.info.out_words, dtype=torch.int64, device="cuda")
    assert _lib.lib().pa_hash_prepared(p.handle, dk.data_ptr(), o.data_ptr(), None, sp) == _lib.PA_ERR_INVALID
    _lib.pa_seed_prepare(p, ds.data_ptr(), sp)
    st = torch.full((1,), -9, dtype=torch.int32, device="cuda")
    _lib.pa_hash_prepared(p, dk.data_ptr(), o.data_ptr(), st.data_ptr(), sp)
    torch.cuda.synchronize()
    s0, ref, _, _ = gpu_hash(p, key, seed)
    assert int(st.item()) == s0 == 0 and np.array_equal(host(o), ref)
    p.close()


@pytest.mark.parametrize("backend", [1, 2])
def test_host_staging_retries_after_failed_allocation(backend):
    """The host-buffer entry point's staging slot (device buffer, then pinned
    status word) cannot be set up: PA_ERR_NOMEM; the next call completes the
    slot and hashes correctly."""
    import torch
    from paper_2105_13678_gb300 import _lib
    n, r = 2_000_003, 200_000
    p = _lib.Plan(n, r, backend=backend)
    g, k, key, seed = _inputs(n, r, 406)
    hk = torch.from_numpy(key.view(np.int64)).pin_memory()
    hs = torch.from_numpy(seed.view(np.int64)).pin_memory()
    ho = torch.zeros(p.info.out_words, dtype=torch.int64).pin_memory()
    hst = torch.full((1,), -9, dtype=torch.int32).pin_memory()
    sp = torch.cuda.current_stream().cuda_stream
    L = _lib.lib()
    for skip in (0, 1):  # the slot's device buffer, then its pinned status word
        _fail(skip, 1)
        try:
            rc = L.pa_hash_host_async(p.handle, hk.data_ptr(), hs.data_ptr(), ho.data_ptr(), hst.data_ptr(), sp)
        finally:
            _fail(0, 0)
        assert rc == _lib.PA_ERR_NOMEM
        # the failed call took a slot turn; the other slot is set up normally by this call
        assert L.pa_hash_host_async(p.handle, hk.data_ptr(), hs.data_ptr(), ho.data_ptr(), hst.data_ptr(), sp) == 0
        torch.cuda.synchronize()
        rc0, ref, _ = oracle.pa_hash(key, n, seed, r, g, k)
        assert int(hst.item()) == rc0 == 0 and np.array_equal(ho.numpy().view(np.uint64), ref)
    # and the slot that failed completes its set-up on its next turn
    for _ in range(2):
        ho.zero_()
        assert L.pa_hash_host_async(p.handle, hk.data_ptr(), hs.data_ptr(), ho.data_ptr(), hst.data_ptr(), sp) == 0
        torch.cuda.synchronize()
        assert np.array_equal(ho.numpy().view(np.uint64), ref)
    p.close()
