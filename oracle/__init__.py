"""Reference oracle for the MMH-MH privacy-amplification hash (arXiv 2105.13678).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this package, and this package imports nothing from the product.

The arithmetic lives in ``pa_oracle.c`` (plain single-threaded C, exact
integers): Algorithm 1 of Sec. 3.1, the MMH definition (Eq. 2), the MH
definition (Eq. 4), the Mersenne reduction of Sec. 3.1 and the parameter rule
of Sec. 4 / Table 3.  This module only marshals numpy arrays to it.

Parity status of each function is recorded in the test suite
(``tests/test_oracle_pins.py``); every function below is pinned by at least
one check that does not reuse the oracle's own code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pa_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORA_OK = 0
ORA_RELOAD = 1

_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile pa_oracle.c into liboracle.so next to it (plain gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.ora_plan.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)]
            lib.ora_pa_hash.argtypes = [_u64p, ctypes.c_uint64, _u64p, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint64, _u64p, _u64p]
            lib.ora_mul.argtypes = [_u64p, ctypes.c_size_t, _u64p, ctypes.c_size_t, _u64p, ctypes.c_int]
            lib.ora_mod_mersenne.argtypes = [_u64p, ctypes.c_size_t, ctypes.c_uint32]
            lib.ora_mmh.argtypes = [_u64p, ctypes.c_uint64, _u64p, ctypes.c_uint32, ctypes.c_uint64, _u64p]
            lib.ora_mh.argtypes = [_u64p, _u64p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, _u64p]
            lib.ora_mersenne_at.restype = ctypes.c_uint32
            lib.ora_set_karatsuba_threshold.argtypes = [ctypes.c_size_t]
            lib.ora_toeplitz.argtypes = [_u64p, ctypes.c_uint64, _u64p, ctypes.c_uint64, _u64p]
            lib.ora_toeplitz_bits.argtypes = [_u64p, ctypes.c_uint64, _u64p, ctypes.c_uint64, _u64p, ctypes.c_uint64,
                                              ctypes.POINTER(ctypes.c_uint8)]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u64p)


def words(bits: int) -> int:
    return (int(bits) + 63) // 64


def mersenne_exponents() -> list[int]:
    lib = _load()
    return [int(lib.ora_mersenne_at(i)) for i in range(lib.ora_mersenne_count())]


def plan(n: int, r: int, margin: int = 128, gamma: int = 0) -> tuple[int, int]:
    """Step 0 (Sec. 4): returns (gamma, k)."""
    lib = _load()
    g = ctypes.c_uint32()
    k = ctypes.c_uint64()
    rc = lib.ora_plan(n, r, margin, gamma, ctypes.byref(g), ctypes.byref(k))
    if rc != ORA_OK:
        raise ValueError(f"oracle plan rejected n={n} r={r} margin={margin} gamma={gamma}")
    return int(g.value), int(k.value)


def pa_hash(key: np.ndarray, n: int, seed: np.ndarray, r: int, gamma: int, k: int):
    """Algorithm 1.  Returns (status, out words, y words)."""
    lib = _load()
    key = np.ascontiguousarray(key, dtype=np.uint64)
    seed = np.ascontiguousarray(seed, dtype=np.uint64)
    assert key.size >= words(n) and seed.size >= words((k + 2) * gamma)
    out = np.zeros(words(r), dtype=np.uint64)
    y = np.zeros(words(gamma), dtype=np.uint64)
    rc = lib.ora_pa_hash(_ptr(key), n, _ptr(seed), r, gamma, k, _ptr(out), _ptr(y))
    if rc < 0:
        raise RuntimeError(f"oracle error {rc}")
    return rc, out, y


def mmh(key: np.ndarray, n: int, seed: np.ndarray, gamma: int, k: int):
    """Eq. 2: returns (status, y words)."""
    lib = _load()
    key = np.ascontiguousarray(key, dtype=np.uint64)
    seed = np.ascontiguousarray(seed, dtype=np.uint64)
    y = np.zeros(words(gamma), dtype=np.uint64)
    rc = lib.ora_mmh(_ptr(key), n, _ptr(seed), gamma, k, _ptr(y))
    if rc < 0:
        raise RuntimeError(f"oracle error {rc}")
    return rc, y


def mh(y: np.ndarray, seed: np.ndarray, gamma: int, k: int, r: int) -> np.ndarray:
    """Eq. 4 on an MMH value y, with b, c taken from the seed's last two slices."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.uint64)
    seed = np.ascontiguousarray(seed, dtype=np.uint64)
    out = np.zeros(words(r), dtype=np.uint64)
    rc = lib.ora_mh(_ptr(y), _ptr(seed), gamma, k, r, _ptr(out))
    if rc < 0:
        raise RuntimeError(f"oracle error {rc}")
    return out


def int_to_words(x: int, nwords: int) -> np.ndarray:
    return np.frombuffer(int(x).to_bytes(8 * nwords, "little"), dtype=np.uint64).copy()


def words_to_int(w: np.ndarray) -> int:
    return int.from_bytes(np.ascontiguousarray(w, dtype=np.uint64).tobytes(), "little")


def mul(a: int, b: int, method: int = 1) -> int:
    """The oracle's big-integer product (method 0 schoolbook, 1 Karatsuba)."""
    lib = _load()
    na, nb = max(1, words(a.bit_length())), max(1, words(b.bit_length()))
    aw, bw = int_to_words(a, na), int_to_words(b, nb)
    rw = np.zeros(na + nb, dtype=np.uint64)
    if lib.ora_mul(_ptr(aw), na, _ptr(bw), nb, _ptr(rw), method) != ORA_OK:
        raise MemoryError
    return words_to_int(rw)


def mod_mersenne(s: int, gamma: int) -> int:
    """The oracle's reduction mod 2^gamma - 1 (Sec. 3.1 fold)."""
    lib = _load()
    ns = max(words(s.bit_length()), words(gamma)) + 1
    sw = int_to_words(s, ns)
    lib.ora_mod_mersenne(_ptr(sw), ns, gamma)
    return words_to_int(sw)


def set_karatsuba_threshold(limbs: int) -> None:
    _load().ora_set_karatsuba_threshold(limbs)


def toeplitz(key: np.ndarray, n: int, seed: np.ndarray, r: int) -> np.ndarray:
    """Toeplitz-hashing PA (the comparison scheme of Sec. 1 / Table 1): z = T x
    over GF(2), T[i][j] = s[i - j + n - 1], s of n + r - 1 bits.  Returns the
    r output bits as words."""
    lib = _load()
    key = np.ascontiguousarray(key, dtype=np.uint64)
    seed = np.ascontiguousarray(seed, dtype=np.uint64)
    assert key.size >= words(n) and seed.size >= words(n + r - 1)
    out = np.zeros(words(r), dtype=np.uint64)
    rc = lib.ora_toeplitz(_ptr(key), n, _ptr(seed), r, _ptr(out))
    if rc < 0:
        raise RuntimeError(f"oracle error {rc}")
    return out


def toeplitz_bits(key: np.ndarray, n: int, seed: np.ndarray, r: int, idx) -> np.ndarray:
    """Output bits z_i of the Toeplitz product for the indices idx (each O(n))."""
    lib = _load()
    key = np.ascontiguousarray(key, dtype=np.uint64)
    seed = np.ascontiguousarray(seed, dtype=np.uint64)
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    out = np.zeros(ix.size, dtype=np.uint8)
    rc = lib.ora_toeplitz_bits(_ptr(key), n, _ptr(seed), r, _ptr(ix), ix.size,
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    if rc < 0:
        raise RuntimeError(f"oracle error {rc}")
    return out
