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
