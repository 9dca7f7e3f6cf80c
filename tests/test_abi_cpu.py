"""Host-side checks of the C-ABI library (no device work): it loads, exports
every symbol the headers declare, and its host-side plan logic and field
constants are right."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2105_13678_gb300 import _lib, synthetic

from helpers import oracle_hash_parallel

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
Q = 2**64 - 2**32 + 1


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(pa_\w+)\s*\(", txt, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    declared = _declared()
    assert {"pa_plan", "pa_hash", "pa_hash_batch", "pa_serve_create", "pa_hash_host"} <= declared
    for name in declared:
        assert hasattr(L, name), name
    assert set(_lib.SIGNATURES) >= declared


def test_field_constants():
    for l in range(0, 27):
        w, t = _lib.field_constants(l)
        assert pow(t, 1 << l, Q) == 2
        assert pow(w, 1 << l, Q) == 1
        if l:
            assert pow(w, 1 << (l - 1), Q) == Q - 1
        if l >= 3:
            # the radix-8 rounds hard-code omega_8 = -2^24 (and 2^96 = -1)
            assert pow(w, 1 << (l - 3), Q) == Q - (1 << 24)
    assert pow(2, 96, Q) == Q - 1
    with pytest.raises(_lib.PAError):
        _lib.field_constants(27)


@pytest.mark.parametrize("G,K", [(110503, 10), (30402457, 9), (60804914, 1), (136279841, 8), (272559682, 1),
                                 (5, 1), (127, 3), (61, 1000)])
def test_transform_len_is_smallest_exact(G, K):
    """The chosen length keeps 2 K N (2^b - 1)^2 + 2^b below q and is minimal."""
    l = _lib.transform_len(G, K)
    N = 1 << l
    b = -(-G // N)
    assert b <= 31 and 2 * K * N * (2**b - 1) ** 2 + 2**b - 1 < Q
    if l:
        N2 = N // 2
        b2 = -(-G // N2)
        assert b2 > 31 or 2 * K * N2 * (2**b2 - 1) ** 2 + 2**b2 - 1 >= Q


def test_plan_estimate_and_status_strings():
    assert _lib.plan_estimate_bytes(260_000_000, 26_000_000) > 260_000_000 // 8
    assert _lib.lib().pa_status_string(1).decode().startswith("reload")
    with pytest.raises(_lib.PAError):
        _lib.plan_estimate_bytes(10, 136279841)


def test_parallel_oracle_driver_matches_serial():
    n, r = 1_000_003, 90_000
    g, k = oracle.plan(n, r)
    key, seed = synthetic.block_inputs(31, n, (k + 2) * g)
    rc, out, y = oracle.pa_hash(key, n, seed, r, g, k)
    rc2, out2, y2 = oracle_hash_parallel(key, n, seed, r, g, k, workers=3)
    assert rc == rc2 == 0 and np.array_equal(out, out2) and np.array_equal(y, y2)


def test_backend_parameter_and_estimates():
    """pa_params.backend: both backends size their workspace on the host; an
    unknown backend is rejected; the three-prime plan of the 2.6e8-bit block
    holds its spectra as 32-bit residues of three primes (3 x 4 bytes per
    element against 8 for Goldilocks, same Eq. 2 length, half the Eq. 4 length)."""
    g = _lib.plan_estimate_bytes(260_000_000, 26_000_000, backend=_lib.BACKEND_GOLDILOCKS)
    p3 = _lib.plan_estimate_bytes(260_000_000, 26_000_000, backend=_lib.BACKEND_P3)
    auto = _lib.plan_estimate_bytes(260_000_000, 26_000_000)
    assert auto == p3 and p3 > 0  # PA_BACKEND_AUTO takes the three-prime plan at this size
    assert 3 * 2 * 9 * (1 << 21) * 4 < p3 < 3 * g
    with pytest.raises(_lib.PAError) as e:
        _lib.plan_estimate_bytes(1000, 10, backend=3)
    assert e.value.code == -1
    assert _lib.plan_estimate_bytes(61 * 3, 10, gamma=61, backend=_lib.BACKEND_P3) > 0
    # n = 1e9 (gamma = 136279841): the three-prime Eq. 2 transform would be twice the Goldilocks one
    g9 = _lib.plan_estimate_bytes(1_000_000_000, 100_000_000, backend=_lib.BACKEND_GOLDILOCKS)
    assert _lib.plan_estimate_bytes(1_000_000_000, 100_000_000) == g9
    assert _lib.plan_estimate_bytes(1_000_000_000, 100_000_000, backend=_lib.BACKEND_P3) > g9


def test_oracle_and_library_share_no_code():
    """The oracle includes only C standard headers and the package never names
    the oracle: the two sides share no code, header or table, and only the
    seeded input generator (which holds none of the hash arithmetic) serves
    both."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "oracle", "pa_oracle.c")) as f:
        incs = re.findall(r'#include\s*[<"]([^>"]+)[>"]', f.read())
    assert incs and all(h in ("stdint.h", "stdlib.h", "string.h", "stdio.h", "stddef.h") for h in incs), incs
    pkg = os.path.join(root, "paper_2105_13678_gb300")
    for dirpath, _, files in os.walk(pkg):
        for name in files:
            if name.endswith((".py", ".cu", ".cuh", ".h", ".cpp")) and name != "synthetic.py":
                with open(os.path.join(dirpath, name)) as f:
                    text = f.read()
                assert not re.search(r"\bimport\s+oracle\b|\bfrom\s+oracle\b|pa_oracle|liboracle", text), name


@pytest.mark.parametrize("n,r,gamma", [(0, 10, 0), (100, 0, 0), (1000, 10, 100), (1000, 200, 61), (1000, 10, 1),
                                       (10**12, 10**11, 0)])
def test_plan_rejects_invalid_arguments(n, r, gamma):
    """n = 0, r = 0, a gamma outside the Mersenne exponent list, r >= gamma, and
    r + margin above the largest listed exponent are PA_ERR_INVALID for both
    backends (the plan rule runs on the host)."""
    for backend in (_lib.BACKEND_AUTO, _lib.BACKEND_GOLDILOCKS, _lib.BACKEND_P3):
        with pytest.raises(_lib.PAError) as e:
            _lib.plan_estimate_bytes(n, r, gamma=gamma, backend=backend)
        assert e.value.code == _lib.PA_ERR_INVALID
