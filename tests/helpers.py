"""Shared helpers for the GPU parity tests: device buffers (torch for memory
only) and a multi-threaded driver of the CPU oracle for paper-scale blocks."""
from __future__ import annotations

import concurrent.futures
import os

import numpy as np

import oracle


def dev(a: np.ndarray):
    """Copy u64 words to a CUDA tensor (int64 view of the same bytes)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def gpu_hash(plan, key: np.ndarray, seed: np.ndarray, stream: int = 0):
    """pa_hash on device copies of key and seed; returns (status, out, y)."""
    import torch
    from paper_2105_13678_gb300 import _lib
    dk, ds = dev(key), dev(seed)
    out = torch.zeros(plan.info.out_words, dtype=torch.int64, device="cuda")
    y = torch.zeros((plan.gamma + 63) // 64, dtype=torch.int64, device="cuda")
    st = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    st2 = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    _lib.pa_hash(plan, dk.data_ptr(), ds.data_ptr(), out.data_ptr(), st.data_ptr(), stream)
    _lib.pa_debug_mmh(plan, dk.data_ptr(), ds.data_ptr(), y.data_ptr(), st2.data_ptr(), stream)
    torch.cuda.synchronize()
    return int(st.item()), host(out), host(y), int(st2.item())


def _slice_words(w: np.ndarray, nbits_total: int, lo: int, hi: int) -> np.ndarray:
    """Bits [lo, hi) of a word array as a new word array (bits past nbits_total are 0)."""
    v = int.from_bytes(np.ascontiguousarray(w, dtype=np.uint64).tobytes(), "little")
    v &= (1 << nbits_total) - 1
    v = (v >> lo) & ((1 << (hi - lo)) - 1)
    nw = max(1, (hi - lo + 63) // 64)
    return np.frombuffer(v.to_bytes(8 * nw, "little"), dtype=np.uint64).copy()


def oracle_hash_parallel(key, n, seed, r, gamma, k, workers: int | None = None):
    """Algorithm 1 by the oracle, its k segment products spread over threads.

    Each thread runs the oracle's MMH on a contiguous group of segments (a
    sub-key and the matching a_i slices); the partial values are summed mod
    p = 2^gamma - 1 with Python integers (Eq. 2 is a sum over segments), then
    the oracle's MH runs on the total.  Returns (status, out words, y words)."""
    workers = workers or min(k, os.cpu_count() or 1)
    groups = [list(range(i, min(k, i + (k + workers - 1) // workers)))
              for i in range(0, k, (k + workers - 1) // workers)]
    p = (1 << gamma) - 1

    def part(g):
        i0, i1 = g[0], g[-1] + 1
        kk = i1 - i0
        nn = min(n, i1 * gamma) - i0 * gamma
        sub_key = _slice_words(key, n, i0 * gamma, i0 * gamma + nn)
        sub_seed = np.zeros(oracle.words((kk + 2) * gamma) + 1, dtype=np.uint64)
        a = _slice_words(seed, (k + 2) * gamma, i0 * gamma, i1 * gamma)
        sub_seed[:a.size] = a[:sub_seed.size]
        rc, y = oracle.mmh(sub_key, nn, sub_seed, gamma, kk)
        return rc, oracle.words_to_int(y)

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(groups)) as ex:
        parts = list(ex.map(part, groups))
    out_words = oracle.words(r)
    if any(rc == oracle.ORA_RELOAD for rc, _ in parts):
        return oracle.ORA_RELOAD, np.zeros(out_words, dtype=np.uint64), None
    y = sum(v for _, v in parts) % p
    yw = oracle.int_to_words(y, oracle.words(gamma))
    out = oracle.mh(yw, seed, gamma, k, r)
    return oracle.ORA_OK, out, yw


def oracle_hash_many(blocks, workers: int | None = None):
    """Algorithm 1 by the oracle for many blocks at once.

    ``blocks`` is a list of (key, n, seed, r, gamma, k).  Every block's k
    segment products (Eq. 2, one per segment) go to one thread pool, then
    every block's Eq. 4 product; the oracle's C code releases the GIL, so the
    host's cores all work.  Returns [(status, out words)] in input order."""
    workers = workers or (os.cpu_count() or 1)
    p_of = [(1 << b[4]) - 1 for b in blocks]

    def seg(job):
        bi, i = job
        key, n, seed, r, gamma, k = blocks[bi]
        nn = min(n, (i + 1) * gamma) - i * gamma
        sub_key = _slice_words(key, n, i * gamma, i * gamma + nn)
        sub_seed = np.zeros(oracle.words(3 * gamma) + 1, dtype=np.uint64)
        a = _slice_words(seed, (k + 2) * gamma, i * gamma, (i + 1) * gamma)
        sub_seed[:a.size] = a[:sub_seed.size]
        rc, y = oracle.mmh(sub_key, nn, sub_seed, gamma, 1)
        return bi, rc, oracle.words_to_int(y)

    jobs = [(bi, i) for bi, b in enumerate(blocks) for i in range(b[5])]
    # largest products first so that the pool finishes together
    jobs.sort(key=lambda j: -blocks[j[0]][4])
    acc = [0] * len(blocks)
    reload = [False] * len(blocks)
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        for bi, rc, v in ex.map(seg, jobs):
            reload[bi] = reload[bi] or rc == oracle.ORA_RELOAD
            acc[bi] += v

        def fin(bi):
            key, n, seed, r, gamma, k = blocks[bi]
            if reload[bi]:
                return oracle.ORA_RELOAD, np.zeros(oracle.words(r), dtype=np.uint64)
            yw = oracle.int_to_words(acc[bi] % p_of[bi], oracle.words(gamma))
            return oracle.ORA_OK, oracle.mh(yw, seed, gamma, k, r)

        order = sorted(range(len(blocks)), key=lambda b: -blocks[b][4])
        res = dict(zip(order, ex.map(fin, order)))
    return [res[i] for i in range(len(blocks))]
