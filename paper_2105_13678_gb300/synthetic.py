"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the hash: it only draws uniform random bits.
The generator is splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state advances by the golden
gamma 0x9E3779B97F4A7C15 and each output is the state passed through the
published 64-bit finaliser.  Output i (0-based) of stream ``seed`` is
``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``, which vectorises.

Draw order for one privacy-amplification block: the key words
(ceil(n/64)) first, then the hash seed words (ceil(seed_bits/64)); bits at or
past n (resp. seed_bits) in the last word are cleared.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of the splitmix64 stream with this seed."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def words(bits: int) -> int:
    return (int(bits) + 63) // 64


def clear_tail(w: np.ndarray, bits: int) -> np.ndarray:
    """Zero the bits at or beyond ``bits`` in the last used word (in place)."""
    nw = words(bits)
    if nw and bits % 64:
        w[nw - 1] &= np.uint64((1 << (bits % 64)) - 1)
    w[nw:] = 0
    return w


def block_inputs(seed: int, n_bits: int, seed_bits: int, start: int = 0):
    """Key (ceil(n/64) words) then hash seed (ceil(seed_bits/64) words)."""
    nk, ns = words(n_bits), words(seed_bits)
    stream = splitmix64(seed, nk + ns, start)
    key = clear_tail(stream[:nk].copy(), n_bits)
    hseed = clear_tail(stream[nk:].copy(), seed_bits)
    return key, hseed


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the stream."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def batch_shapes(seed: int = 7, blocks: int = 64, log2_lo: int = 20, log2_hi: int = 27,
                 ratio_lo: float = 0.05, ratio_hi: float = 0.5):
    """Heterogeneous batch: n log-uniform in [2^lo, 2^hi] bits, r/n uniform in
    [ratio_lo, ratio_hi], r = ceil(ratio * n).  Returns [(n, r, block_seed)].
    Block b draws its key and hash seed from stream ``(seed << 32) + b``."""
    u = uniform01(seed, 2 * blocks)
    out = []
    for b in range(blocks):
        n = int(math.floor(2.0 ** (log2_lo + (log2_hi - log2_lo) * u[2 * b])))
        ratio = ratio_lo + (ratio_hi - ratio_lo) * u[2 * b + 1]
        r = max(1, int(math.ceil(ratio * n)))
        out.append((n, r, (seed << 32) + b))
    return out


def served_arrivals(seed: int = 8, jobs: int = 2000, rate_per_s: float = 200.0,
                    sizes=((1e7, 0.70), (1e8, 0.25), (2.6e8, 0.05)), ratio: float = 0.1):
    """Poisson arrivals (exponential gaps of mean 1/rate) with n drawn from the
    size mix; r = ceil(ratio * n).  Returns [(t_arrival_s, n, r)]."""
    u = uniform01(seed, 2 * jobs)
    t = 0.0
    out = []
    cum = np.cumsum([p for _, p in sizes])
    for j in range(jobs):
        t += -math.log(1.0 - u[2 * j]) / rate_per_s
        cls = int(np.searchsorted(cum, u[2 * j + 1], side="right"))
        cls = min(cls, len(sizes) - 1)
        n = int(sizes[cls][0])
        out.append((t, n, max(1, int(math.ceil(ratio * n)))))
    return out
