"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerance: zero differing bits (the hash is an exact integer function)."""
import numpy as np
import pytest

import oracle
from paper_2105_13678_gb300 import synthetic

from helpers import gpu_hash, oracle_hash_parallel

pytestmark = pytest.mark.gpu


GOLDILOCKS, P3 = 1, 2


def _plan(n, r, gamma=0, margin=128, backend=GOLDILOCKS):
    from paper_2105_13678_gb300 import _lib
    return _lib.Plan(n, r, gamma=gamma, margin=margin, backend=backend)


def _p3_plan(n, r, gamma=0, margin=128):
    """The three-prime plan, or None where its sizes are not feasible."""
    from paper_2105_13678_gb300 import _lib
    try:
        return _plan(n, r, gamma, margin, P3)
    except _lib.PAError as e:
        assert e.code == -7  # PA_ERR_UNSUPPORTED
        return None


def _check(n, r, seed_id, gamma=0, margin=128, parallel=False, key=None, hseed=None):
    """Both backends (Goldilocks, three-prime) against one oracle result."""
    plans = [_plan(n, r, gamma, margin, GOLDILOCKS), _p3_plan(n, r, gamma, margin)]
    g, k = plans[0].gamma, plans[0].k
    assert (g, k) == oracle.plan(n, r, margin=margin, gamma=gamma)
    if key is None:
        key, hseed = synthetic.block_inputs(seed_id, n, (k + 2) * g)
    if parallel:
        rc, out, y = oracle_hash_parallel(key, n, hseed, r, g, k)
    else:
        rc, out, y = oracle.pa_hash(key, n, hseed, r, g, k)
    for plan in plans:
        if plan is None:
            continue
        tag = f"backend={plan.backend} n={n} r={r} gamma={g} k={k}"
        st, gout, gy, st2 = gpu_hash(plan, key, hseed)
        assert st == rc and st2 == rc, tag
        assert np.array_equal(gout, out), f"output mismatch {tag}"
        if rc == oracle.ORA_OK:
            assert np.array_equal(gy, y[: gy.size]), f"MMH value mismatch {tag}"
        plan.close()
    return plans[0]


def test_config1_plain_block_2p20():
    """n = 2^20 uniform bits (splitmix64 seed 1), r = ceil(0.1 n) = 104858."""
    p = _check(1 << 20, 104858, 1)
    assert (p.gamma, p.k) == (110503, 10)


@pytest.mark.parametrize("gamma", [2, 3, 5, 7, 13, 17, 19, 31, 61, 89, 107, 127, 521, 607, 1279, 2203, 4423])
def test_small_gammas(gamma):
    rng = np.random.default_rng(gamma)
    for n in (gamma, 3 * gamma, 7 * gamma + 1, 40 * gamma - 3):
        for r in sorted({1, max(1, gamma // 2), gamma - 1}):
            if r >= gamma:
                continue
            _check(n, r, int(rng.integers(1 << 30)), gamma=gamma)


@pytest.mark.parametrize("n,r", [(64, 1), (65, 7), (1000, 100), (4096, 1000), (12345, 3000), (100000, 10000),
                                 (300000, 29000), (2**20 + 17, 50000), (3 * 110503, 100000), (5 * 756839, 300000)])
def test_ragged_sizes(n, r):
    _check(n, r, n ^ r)


@pytest.mark.parametrize("n,r,gamma", [(10 * 9689, 500, 9689), (5 * 44497, 20000, 44497), (86243, 2000, 86243),
                                       (1000, 10, 1279)])
def test_no_padding_and_k1(n, r, gamma):
    _check(n, r, 77, gamma=gamma)


@pytest.mark.parametrize("backend", [GOLDILOCKS, P3])
def test_reload_on_all_ones_slice(backend):
    n, r, gamma = 4 * 4423, 100, 4423
    plan = _plan(n, r, gamma, backend=backend)
    k = plan.k
    key, hseed = synthetic.block_inputs(5, n, (k + 2) * gamma)
    kv = oracle.words_to_int(key) | (((1 << gamma) - 1) << (2 * gamma))  # slice x_3 all ones
    key = oracle.int_to_words(kv, key.size)
    rc, out, _ = oracle.pa_hash(key, n, hseed, r, gamma, k)
    assert rc == oracle.ORA_RELOAD
    st, gout, _, _ = gpu_hash(plan, key, hseed)
    assert st == oracle.ORA_RELOAD and not gout.any()


@pytest.mark.parametrize("backend", [GOLDILOCKS, P3])
def test_reload_on_all_ones_slice_1024_row_columns(backend):
    """The reload rule where the three-prime column pass runs on 1024-row tiles
    (transform of 2^20 points, one CTA walking several tiles): a random key
    hashes normally, and an all-ones slice in the middle or as the last slice
    gives the reload status and a zero output."""
    gamma = 13466917
    n, r = 4 * gamma, 1000
    plan = _plan(n, r, gamma, backend=backend)
    if backend == P3:
        assert plan.geometry(0)[0] == 10
    key, hseed = synthetic.block_inputs(6, n, (plan.k + 2) * gamma)
    st, _, _, _ = gpu_hash(plan, key, hseed)
    assert st == oracle.ORA_OK
    kv = oracle.words_to_int(key)
    for sl in (1, plan.k - 1):
        kv2 = kv | (((1 << gamma) - 1) << (sl * gamma))
        st, out, _, _ = gpu_hash(plan, oracle.int_to_words(kv2, key.size), hseed)
        assert st == oracle.ORA_RELOAD and not out.any()


@pytest.mark.parametrize("gamma", [44497, 1257787])
def test_zero_mmh_value_and_all_ones_representation(gamma):
    """Seeds that make y = 0: a = 0, and a pair with a_2 = -a_1, x_2 = x_1 (the
    carry ring may land on the all-ones representation of 0); at gamma = 44497
    the three-prime plan resolves carries in one CTA, at 1257787 in the fused
    multi-CTA pass."""
    n, r = 2 * gamma, 1000
    plan = _plan(n, r, gamma)  # k and the seed layout (both backends are checked below)
    k = plan.k
    key, hseed = synthetic.block_inputs(9, n, (k + 2) * gamma)
    p = (1 << gamma) - 1
    sv = oracle.words_to_int(hseed)
    mask = (1 << (2 * gamma)) - 1
    for a1, a2, x_same in ((0, 0, False), (12345, p - 12345, True), (1, p - 1, True), (p, 0, False)):
        s2 = (sv & ~mask) | a1 | (a2 << gamma)
        seed2 = oracle.int_to_words(s2, hseed.size)
        key2 = key
        if x_same:
            kv = oracle.words_to_int(key)
            x1 = kv & ((1 << gamma) - 1)
            key2 = oracle.int_to_words(x1 | (x1 << gamma), key.size)
        _check(n, r, 0, gamma=gamma, key=key2, hseed=seed2)


@pytest.mark.parametrize("backend", [GOLDILOCKS, P3])
def test_bits_past_n_ignored(backend):
    n, r = 100003, 5000
    plan = _plan(n, r, backend=backend)
    k, g = plan.k, plan.gamma
    key, hseed = synthetic.block_inputs(21, n, (k + 2) * g)
    dirty = key.copy()
    dirty[-1] |= ~np.uint64((1 << (n % 64)) - 1)
    st, a, _, _ = gpu_hash(plan, key, hseed)
    st2, b, _, _ = gpu_hash(plan, dirty, hseed)
    assert st == st2 == 0 and np.array_equal(a, b)


@pytest.mark.parametrize("backend", [GOLDILOCKS, P3])
@pytest.mark.parametrize("n,r,gamma", [(1 << 20, 104858, 0), (7 * 4423 + 5, 300, 4423), (3_000_001, 290_000, 0),
                                       (4 * 4423, 100, 4423)])
def test_host_entry_point_matches_device(n, r, gamma, backend):
    """pa_hash_host (pipelined host-to-device copies) equals pa_hash; the last
    case plants an all-ones slice, so both must report a reload."""
    from paper_2105_13678_gb300 import _lib
    plan = _plan(n, r, gamma, backend=backend)
    key, hseed = synthetic.block_inputs(1, n, (plan.k + 2) * plan.gamma)
    if n == 4 * 4423:
        kv = oracle.words_to_int(key) | (((1 << 4423) - 1) << 4423)
        key = oracle.int_to_words(kv, key.size)
    for _ in range(2):
        st, out = _lib.pa_hash_host(plan, key, hseed)
        st2, out2, _, _ = gpu_hash(plan, key, hseed)
        assert st == st2 and np.array_equal(out, out2)
    rc, ref, _ = oracle.pa_hash(key, n, hseed, r, plan.gamma, plan.k)
    assert st == rc and np.array_equal(out, ref)


@pytest.mark.parametrize("backend", [GOLDILOCKS, P3])
def test_repeat_calls_identical(backend):
    n, r = 3_000_000, 300_000
    plan = _plan(n, r, backend=backend)
    key, hseed = synthetic.block_inputs(4, n, (plan.k + 2) * plan.gamma)
    outs = [gpu_hash(plan, key, hseed)[1] for _ in range(3)]
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


@pytest.mark.parametrize("n,r,seed_id", [(10_000_000, 1_000_000, 3), (100_000_000, 10_000_000, 4),
                                         (260_000_000, 26_000_000, 5), (1_000_000_000, 100_000_000, 6)])
def test_sweep_sizes(n, r, seed_id):
    """Block-size sweep n = 1e7, 1e8, 2.6e8, 1e9 (r = 0.1 n, seeds 3..6); the
    1e9 block (gamma = 136279841, the largest tabulated exponent) needs the
    oracle for several minutes."""
    _check(n, r, seed_id, parallel=True)


@pytest.mark.parametrize("ratio", [0.1, 0.05, 0.3])
def test_paper_scale_2p6e8(ratio):
    """Paper-scale block n = 2.6e8 (seed 2) at r/n = 0.1, 0.05, 0.3."""
    n = 260_000_000
    r = int(np.ceil(ratio * n))
    _check(n, r, 2, parallel=True)


def test_paper_points_cv_dv():
    """The paper's unpadded points: CV n = 10 * 25964951, DV n = 3 * 74207281."""
    for n, ratio in ((10 * 25964951, 0.0972), (3 * 74207281, 0.2957)):
        r = int(np.floor(ratio * n))
        p = _check(n, r, 11, parallel=True)
        assert p.k * p.gamma == n


def test_paper_point_cv_max_8e8():
    """The largest CV block of Sec. 4 (k = 10, about 8e8 bits): n = 10 * 82589933,
    r = floor(0.0972 n), no padding; both backends against the oracle."""
    n = 10 * 82589933
    r = int(np.floor(0.0972 * n))
    p = _check(n, r, 12, parallel=True)
    assert (p.gamma, p.k) == (82589933, 10) and p.k * p.gamma == n


@pytest.mark.parametrize("backend", [GOLDILOCKS, P3])
def test_host_async_stream_of_blocks(backend):
    """pa_hash_host_async: several blocks in flight on one stream (staging slots
    alternate, copies overlap the previous block); every output equals pa_hash."""
    import torch
    from paper_2105_13678_gb300 import _lib
    n, r = 2_000_003, 200_000
    plan = _plan(n, r, backend=backend)
    keys, seeds, outs = [], [], []
    for i in range(5):
        key, seed = synthetic.block_inputs(300 + i, n, (plan.k + 2) * plan.gamma)
        keys.append(torch.from_numpy(key.view(np.int64)).pin_memory())
        seeds.append(torch.from_numpy(seed.view(np.int64)).pin_memory())
        outs.append(torch.zeros(plan.info.out_words, dtype=torch.int64).pin_memory())
    stat = torch.full((5,), -9, dtype=torch.int32).pin_memory()
    sp = torch.cuda.current_stream().cuda_stream
    for i in range(5):
        _lib.check(_lib.lib().pa_hash_host_async(plan.handle, keys[i].data_ptr(), seeds[i].data_ptr(),
                                                 outs[i].data_ptr(), stat.data_ptr() + 4 * i, sp), "async")
    torch.cuda.synchronize()
    assert (stat.numpy() == 0).all()
    for i in range(5):
        st, ref, _, _ = gpu_hash(plan, keys[i].numpy().view(np.uint64), seeds[i].numpy().view(np.uint64))
        assert st == 0 and np.array_equal(outs[i].numpy().view(np.uint64), ref)
    plan.close()


def test_backend_lengths_and_auto_choice():
    """Transform lengths of both backends at the 2.6e8-bit and 1e9-bit blocks;
    PA_BACKEND_AUTO takes the three-prime plan where its Eq. 2 transform is no
    longer (2.6e8, 2^20) and the Goldilocks plan where it would be (1e9, tiny)."""
    from paper_2105_13678_gb300 import _lib
    a = _lib.Plan(260_000_000, 26_000_000, backend=P3)
    assert a.info.mmh_len == 1 << 21 and a.info.mh_len == 1 << 21
    g = _lib.Plan(260_000_000, 26_000_000, backend=GOLDILOCKS)
    assert g.info.mmh_len == 1 << 21 and g.info.mh_len == 1 << 22
    auto = _lib.Plan(260_000_000, 26_000_000)
    assert auto.backend == P3
    b = _lib.Plan(1_000_000_000, 100_000_000, backend=P3)
    assert b.info.mmh_len == 1 << 24
    b2 = _lib.Plan(1_000_000_000, 100_000_000)
    assert b2.backend == GOLDILOCKS and b2.info.mmh_len == 1 << 23
    small = _lib.Plan(1 << 20, 104858)
    assert small.backend == P3 and small.info.mmh_len == 1 << 13
    tiny = _lib.Plan(600, 10, gamma=61)  # the three-prime transforms start at 2^8
    assert tiny.backend == GOLDILOCKS
    mid = _lib.Plan(10_000_000, 1_000_000)  # T = 2^17 against N = 2^16
    assert mid.backend == P3 and mid.info.mmh_len == 1 << 17
    for p in (a, g, auto, b, b2, small, tiny, mid):
        p.close()


@pytest.mark.parametrize("gamma,k", [(521, 1), (521, 3), (607, 2), (4423, 5), (9689, 4), (44497, 3)])
def test_p3_fold_offsets_wrap(gamma, k):
    """Three-prime plans where the digit grid M b overshoots gamma by more than a
    digit (the Mersenne fold places whole digits past gamma back at offset
    (t b) mod gamma), every k up to the segment count."""
    n = k * gamma - 3
    _check(n, max(1, gamma // 3), gamma * 31 + k, gamma=gamma)


def test_tuned_auto_plan_measures_the_backend(tmp_path):
    """pa_params.tune with backend AUTO builds both backends and keeps the one
    that hashed faster; the decision is cached per (gamma, k), written by
    pa_tune_cache_save, and the plan gives the oracle's bits."""
    from paper_2105_13678_gb300 import _lib
    for n, r, seed_id in ((10_000_000, 1_000_000, 41), (1 << 20, 104858, 42)):
        p = _lib.Plan(n, r, tune=True)
        assert p.backend in (GOLDILOCKS, P3)
        key, hseed = synthetic.block_inputs(seed_id, n, (p.k + 2) * p.gamma)
        st, out, _, _ = gpu_hash(p, key, hseed)
        rc, ref, _ = oracle_hash_parallel(key, n, hseed, r, p.gamma, p.k)
        assert st == rc == 0 and np.array_equal(out, ref)
        again = _lib.Plan(n, r, tune=True)  # cached decision
        assert again.backend == p.backend
        path = tmp_path / "tune.txt"
        assert _lib.lib().pa_tune_cache_save(str(path).encode()) >= 1
        assert f"backend {p.gamma} {p.k} {p.backend}" in path.read_text().split("\n")
        p.close()
        again.close()
