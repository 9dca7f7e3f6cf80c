"""Batched (one CUDA-graph launch over many blocks) and served (continuous
batching) modes: every result is bit-identical to the same block hashed alone
and to the oracle."""
import math
import time

import numpy as np
import pytest

import oracle
from paper_2105_13678_gb300 import synthetic

from helpers import dev, gpu_hash, host, oracle_hash_many, oracle_hash_parallel

pytestmark = pytest.mark.gpu


def _blocks(shapes):
    import torch
    from paper_2105_13678_gb300 import _lib
    out = []
    for n, r, s in shapes:
        p = _lib.Plan(n, r)
        key, seed = synthetic.block_inputs(s, n, (p.k + 2) * p.gamma)
        out.append(dict(plan=p, n=n, r=r, key=key, seed=seed, dk=dev(key), ds=dev(seed),
                        do=torch.zeros(p.info.out_words, dtype=torch.int64, device="cuda")))
    return out


def _run_batch(blocks, reps=1):
    import torch
    from paper_2105_13678_gb300 import _lib
    st = torch.full((len(blocks),), -9, dtype=torch.int32, device="cuda")
    for _ in range(reps):
        _lib.pa_hash_batch([b["plan"] for b in blocks], [b["dk"].data_ptr() for b in blocks],
                           [b["ds"].data_ptr() for b in blocks], [b["do"].data_ptr() for b in blocks],
                           st.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st.cpu().numpy()


def test_batch_small_blocks_match_oracle():
    rng = np.random.default_rng(3)
    shapes = []
    for i in range(12):
        n = int(2 ** rng.uniform(12, 21))
        r = max(1, int(n * rng.uniform(0.05, 0.5)))
        shapes.append((n, r, 1000 + i))
    blocks = _blocks(shapes)
    st = _run_batch(blocks, reps=2)
    for b, s in zip(blocks, st):
        rc, out, _ = oracle.pa_hash(b["key"], b["n"], b["seed"], b["r"], b["plan"].gamma, b["plan"].k)
        assert s == rc
        assert np.array_equal(host(b["do"]), out)


def test_batch_replays_current_buffer_contents():
    import torch
    shapes = [(1 << 16, 5000, 1), (1 << 18, 20000, 2), (1 << 17, 3000, 3)]
    blocks = _blocks(shapes)
    _run_batch(blocks)
    first = [host(b["do"]).copy() for b in blocks]
    b0 = blocks[0]
    key2, _ = synthetic.block_inputs(99, b0["n"], 64)
    b0["dk"].copy_(torch.from_numpy(key2.view(np.int64)))
    _run_batch(blocks)
    rc, out, _ = oracle.pa_hash(key2, b0["n"], b0["seed"], b0["r"], b0["plan"].gamma, b0["plan"].k)
    assert np.array_equal(host(b0["do"]), out) and not np.array_equal(out, first[0])
    for b, f in zip(blocks[1:], first[1:]):
        assert np.array_equal(host(b["do"]), f)


def test_batch_config4_64_blocks():
    """64 blocks, n log-uniform in [2^20, 2^27], r/n in [0.05, 0.5] (seed 7):
    every block of the graph batch equals the oracle, and each block hashed
    alone gives the same bits."""
    shapes = synthetic.batch_shapes(7)
    blocks = _blocks(shapes)
    st = _run_batch(blocks, reps=2)
    assert (st == 0).all()
    batch_out = [host(b["do"]).copy() for b in blocks]
    ref = oracle_hash_many([(b["key"], b["n"], b["seed"], b["r"], b["plan"].gamma, b["plan"].k) for b in blocks])
    for i, (b, bo, (rc, out)) in enumerate(zip(blocks, batch_out, ref)):
        assert rc == 0 and np.array_equal(bo, out), f"block {i}: n={b['n']} r={b['r']} differs from the oracle"
    for b, bo in zip(blocks, batch_out):
        s, out, _, _ = gpu_hash(b["plan"], b["key"], b["seed"])
        assert s == 0 and np.array_equal(out, bo)
    for b in blocks:
        b["plan"].close()


def test_serve_alone_equals_in_mix():
    """Jobs submitted together (overlapping on the device) give the same bits
    as each job hashed alone."""
    import torch
    from paper_2105_13678_gb300 import _lib
    rng = np.random.default_rng(8)
    jobs = []
    for i in range(40):
        n = int(rng.choice([1 << 16, 10_000_000, 3_000_000, 1 << 20]))
        r = int(math.ceil(0.1 * n))
        g, k = oracle.plan(n, r)
        key, seed = synthetic.block_inputs(5000 + i, n, (k + 2) * g)
        jobs.append(dict(n=n, r=r, key=key, seed=seed, dk=dev(key), ds=dev(seed),
                         do=torch.zeros((r + 63) // 64, dtype=torch.int64, device="cuda")))
    srv = _lib.Server(8 << 30, slots=6)
    tickets = [srv.submit(j["n"], j["r"], j["dk"].data_ptr(), j["ds"].data_ptr(), j["do"].data_ptr()) for j in jobs]
    sts = [srv.wait(t, 120.0) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert all(s == 0 for s in sts)
    assert stats["completed"] == len(jobs) and stats["peak_budget_bytes"] <= 8 << 30
    for j in jobs:
        p = _lib.Plan(j["n"], j["r"])
        s, alone, _, _ = gpu_hash(p, j["key"], j["seed"])
        p.close()
        assert s == 0 and np.array_equal(alone, host(j["do"]))
    for j in jobs[:8]:
        g, k = oracle.plan(j["n"], j["r"])
        rc, out, _ = oracle_hash_parallel(j["key"], j["n"], j["seed"], j["r"], g, k)
        assert np.array_equal(out, host(j["do"]))


def test_serve_paper_scale_jobs_in_mix_match_oracle():
    """Served mix of the paper's sizes in flight together: 2.6e8-, 1e8- and
    1e7-bit jobs (r = 0.1 n) submitted at once onto 6 slots under a 16 GB
    budget; every result, taken from the mix, equals the oracle."""
    import torch
    from paper_2105_13678_gb300 import _lib
    sizes = [260_000_000, 10_000_000, 100_000_000, 10_000_000, 260_000_000, 100_000_000,
             10_000_000, 100_000_000, 10_000_000, 10_000_000]
    jobs = []
    for i, n in enumerate(sizes):
        r = int(math.ceil(0.1 * n))
        g, k = oracle.plan(n, r)
        key, seed = synthetic.block_inputs((8 << 32) + 7000 + i, n, (k + 2) * g)
        jobs.append(dict(n=n, r=r, g=g, k=k, key=key, seed=seed, dk=dev(key), ds=dev(seed),
                         do=torch.full(((r + 63) // 64,), -1, dtype=torch.int64, device="cuda")))
    srv = _lib.Server(16 << 30, slots=6)
    tickets = [srv.submit(j["n"], j["r"], j["dk"].data_ptr(), j["ds"].data_ptr(), j["do"].data_ptr()) for j in jobs]
    sts = [srv.wait(t, 300.0) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert all(s == 0 for s in sts)
    assert stats["completed"] == len(jobs) and stats["peak_budget_bytes"] <= 16 << 30
    ref = oracle_hash_many([(j["key"], j["n"], j["seed"], j["r"], j["g"], j["k"]) for j in jobs])
    for i, (j, (rc, out)) in enumerate(zip(jobs, ref)):
        assert rc == 0 and np.array_equal(out, host(j["do"])), f"job {i} (n={j['n']}) differs from the oracle"


def test_serve_budget_admission():
    """A budget that holds one plan at a time still completes every job; a job
    larger than the whole budget is refused at submit."""
    import torch
    from paper_2105_13678_gb300 import _lib
    n, r = 10_000_000, 1_000_000
    need = _lib.plan_estimate_bytes(n, r)
    g, k = oracle.plan(n, r)
    key, seed = synthetic.block_inputs(77, n, (k + 2) * g)
    dk, ds = dev(key), dev(seed)
    outs = [torch.zeros((r + 63) // 64, dtype=torch.int64, device="cuda") for _ in range(6)]
    srv = _lib.Server(int(need * 1.5), slots=4)
    ts = [srv.submit(n, r, dk.data_ptr(), ds.data_ptr(), o.data_ptr()) for o in outs]
    assert all(srv.wait(t, 120.0) == 0 for t in ts)
    st = srv.stats()
    assert st["peak_budget_bytes"] <= need * 1.5 and st["completed"] == 6
    with pytest.raises(_lib.PAError) as ei:
        srv.submit(100_000_000, 10_000_000, dk.data_ptr(), ds.data_ptr(), outs[0].data_ptr())
    assert ei.value.code == _lib.PA_ERR_BUDGET
    srv.close()
    ref = host(outs[0])
    assert all(np.array_equal(host(o), ref) for o in outs)


def test_serve_poll_and_stats_latency():
    import torch
    from paper_2105_13678_gb300 import _lib
    n, r = 1 << 20, 104858
    g, k = oracle.plan(n, r)
    key, seed = synthetic.block_inputs(1, n, (k + 2) * g)
    dk, ds = dev(key), dev(seed)
    o = torch.zeros((r + 63) // 64, dtype=torch.int64, device="cuda")
    srv = _lib.Server(1 << 30, slots=2)
    t = srv.submit(n, r, dk.data_ptr(), ds.data_ptr(), o.data_ptr())
    deadline = time.time() + 60
    while srv.poll(t) is None and time.time() < deadline:
        time.sleep(0.001)
    assert srv.poll(t) == 0
    st = srv.stats()
    srv.close()
    assert st["completed"] == 1 and st["p50_latency_ms"] > 0
    rc, out, _ = oracle.pa_hash(key, n, seed, r, g, k)
    assert np.array_equal(host(o), out)


@pytest.mark.parametrize("n,r", [(1 << 20, 104858), (30_000_000, 9_000_000), (5_000_000, 250_000)])
def test_autotuned_plan_gives_the_same_bits(n, r):
    """pa_params.tune picks the four-step split and column tile by timing;
    the output bits must not depend on the choice."""
    from paper_2105_13678_gb300 import _lib
    p0 = _lib.Plan(n, r, backend=_lib.BACKEND_GOLDILOCKS)
    p1 = _lib.Plan(n, r, tune=True, backend=_lib.BACKEND_GOLDILOCKS)
    key, seed = synthetic.block_inputs(55, n, (p0.k + 2) * p0.gamma)
    s0, o0, y0, _ = gpu_hash(p0, key, seed)
    s1, o1, y1, _ = gpu_hash(p1, key, seed)
    assert s0 == s1 == 0 and np.array_equal(o0, o1) and np.array_equal(y0, y1)
    if n <= (1 << 20):
        rc, ref, _ = oracle.pa_hash(key, n, seed, r, p0.gamma, p0.k)
        assert np.array_equal(o1, ref)
    p0.close()
    p1.close()
