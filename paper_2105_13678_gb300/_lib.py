"""ctypes binding of ``libpa_gb300.so`` (declared in ``include/pa_gb300.h``).

Argument marshalling only: every step of the hash runs in the library's CUDA
kernels.  Device buffers are passed as raw pointers (``tensor.data_ptr()``),
streams as ``torch.cuda.Stream.cuda_stream`` integers.  If the library has not
been built, loading raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpa_gb300.so")

PA_OK = 0
PA_RELOAD = 1
PA_ERR_INVALID = -1
PA_ERR_NOMEM = -2
PA_ERR_CUDA = -3
PA_ERR_TIMEOUT = -4
PA_ERR_BUDGET = -5
PA_ERR_CANCELLED = -6
PA_ERR_UNSUPPORTED = -7
PA_ERR_BUSY = -8

_u64 = ctypes.c_uint64
_vp = ctypes.c_void_p


class pa_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_uint32), ("gamma_margin", ctypes.c_uint32), ("tune", ctypes.c_uint32),
                ("backend", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 4)]


class pa_plan_info(ctypes.Structure):
    _fields_ = [("n_bits", _u64), ("r_bits", _u64), ("gamma", ctypes.c_uint32), ("backend", ctypes.c_uint32),
                ("k", _u64), ("key_words", _u64), ("seed_words", _u64), ("out_words", _u64),
                ("mmh_len", _u64), ("mh_len", _u64), ("workspace_bytes", _u64)]


class pa_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", _u64), ("slots", ctypes.c_uint32), ("max_queue", ctypes.c_uint32),
                ("params", pa_params)]


class pa_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", _u64), ("completed", _u64), ("failed", _u64), ("cancelled", _u64),
                ("queued", _u64), ("running", _u64), ("bits_completed", _u64),
                ("p50_latency_ms", ctypes.c_double), ("p99_latency_ms", ctypes.c_double),
                ("max_latency_ms", ctypes.c_double), ("busy_seconds", ctypes.c_double),
                ("peak_budget_bytes", _u64)]


class pa_trace_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", _u64), ("total_ms", ctypes.c_double)]


# name -> (restype, argtypes), in header order
SIGNATURES = {
    "pa_plan": (ctypes.c_int, [_u64, _u64, ctypes.POINTER(pa_params), ctypes.POINTER(_vp)]),
    "pa_plan_info_get": (ctypes.c_int, [_vp, ctypes.POINTER(pa_plan_info)]),
    "pa_mh_plan": (ctypes.c_int, [_u64, _u64, ctypes.POINTER(_vp)]),
    "pa_toeplitz_plan": (ctypes.c_int, [_u64, _u64, ctypes.c_uint32, ctypes.POINTER(_vp)]),
    "pa_plan_destroy": (ctypes.c_int, [_vp]),
    "pa_hash": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "pa_hash_host": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pa_hash_host_async": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "pa_debug_mmh": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "pa_seed_prepare": (ctypes.c_int, [_vp, _vp, _vp]),
    "pa_hash_prepared": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pa_hash_noalloc": (ctypes.c_int, [_u64, _u64, ctypes.POINTER(pa_params), _vp, _vp, _vp, _vp, _vp]),
    "pa_hash_batch": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                     ctypes.POINTER(_vp), _vp, ctypes.c_int, _vp]),
    "pa_batch_cache_clear": (ctypes.c_int, []),
    "pa_serve_create": (ctypes.c_int, [ctypes.POINTER(pa_serve_config), ctypes.POINTER(_vp)]),
    "pa_serve_submit": (ctypes.c_int, [_vp, _u64, _u64, _vp, _vp, _vp, ctypes.POINTER(_u64)]),
    "pa_serve_poll": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(ctypes.c_int)]),
    "pa_serve_wait": (ctypes.c_int, [_vp, _u64, _u64, ctypes.POINTER(ctypes.c_int)]),
    "pa_serve_stats_get": (ctypes.c_int, [_vp, ctypes.POINTER(pa_serve_stats)]),
    "pa_serve_stats_reset": (ctypes.c_int, [_vp]),
    "pa_serve_shutdown": (ctypes.c_int, [_vp]),
    "pa_serve_destroy": (ctypes.c_int, [_vp]),
    "pa_trace_enable": (ctypes.c_int, [ctypes.c_int]),
    "pa_trace_collect": (ctypes.c_int, [ctypes.POINTER(pa_trace_entry), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "pa_trace_select": (ctypes.c_int, [ctypes.c_char_p]),
    "pa_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
    "pa_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "pa_tc_limbconv_tile": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "pa_tc_int8_rate": (ctypes.c_int, [_u64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
    "pa_debug_fail_allocs": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32]),
    "pa_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pa_version": (ctypes.c_char_p, []),
    "pa_plan_estimate_bytes": (ctypes.c_int, [_u64, _u64, ctypes.POINTER(pa_params), ctypes.POINTER(_u64)]),
    "pa_field_constants": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "pa_transform_len": (ctypes.c_int, [_u64, _u64, ctypes.POINTER(ctypes.c_uint32)]),
    "pa_selftest_field": (ctypes.c_int, [_vp, _vp, _vp, _u64, _vp]),
    "pa_plan_geometry": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_uint32)]),
}

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded library; raises if it was not built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2105_13678_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class PAError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {lib().pa_status_string(code).decode()} ({code})")


def check(code: int, what: str) -> int:
    if code < 0:
        raise PAError(code, what)
    return code


BACKEND_AUTO, BACKEND_GOLDILOCKS, BACKEND_P3 = 0, 1, 2


def params(gamma: int = 0, margin: int = 128, tune: bool = False, backend: int = BACKEND_AUTO) -> pa_params:
    p = pa_params()
    p.gamma = gamma
    p.gamma_margin = margin
    p.tune = 1 if tune else 0
    p.backend = backend
    return p


class Plan:
    """Owns a ``pa_plan_t``: step 0 of Algorithm 1 plus the device workspace.
    ``modular_hash=True`` builds the comparison scheme (Eq. 4 over the whole key),
    ``toeplitz=True`` the Toeplitz-hashing comparison scheme."""

    def __init__(self, n_bits: int, r_bits: int, gamma: int = 0, margin: int = 128, tune: bool = False,
                 modular_hash: bool = False, backend: int = BACKEND_AUTO, toeplitz: bool = False,
                 block_log: int = 0):
        h = _vp()
        if toeplitz:
            check(lib().pa_toeplitz_plan(n_bits, r_bits, block_log, ctypes.byref(h)), "pa_toeplitz_plan")
        elif modular_hash:
            check(lib().pa_mh_plan(n_bits, r_bits, ctypes.byref(h)), "pa_mh_plan")
        else:
            p = params(gamma, margin, tune, backend)
            check(lib().pa_plan(n_bits, r_bits, ctypes.byref(p), ctypes.byref(h)), "pa_plan")
        self.handle = h
        info = pa_plan_info()
        check(lib().pa_plan_info_get(h, ctypes.byref(info)), "pa_plan_info_get")
        self.info = info
        self.n, self.r, self.gamma, self.k = info.n_bits, info.r_bits, info.gamma, info.k
        self.backend = info.backend

    def geometry(self, stage: int):
        """(log2 R, log2 C, column tile width) of the stage's transform."""
        a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        check(lib().pa_plan_geometry(self.handle, stage, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
              "pa_plan_geometry")
        return int(a.value), int(b.value), int(c.value)

    def close(self):
        if self.handle:
            lib().pa_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def pa_hash(plan: Plan, key_ptr: int, seed_ptr: int, out_ptr: int, status_ptr: int = 0, stream: int = 0) -> int:
    return check(lib().pa_hash(plan.handle, key_ptr, seed_ptr, out_ptr, status_ptr or None, stream or None),
                 "pa_hash")


def pa_seed_prepare(plan: Plan, seed_ptr: int, stream: int = 0) -> int:
    return check(lib().pa_seed_prepare(plan.handle, seed_ptr, stream or None), "pa_seed_prepare")


def pa_hash_prepared(plan: Plan, key_ptr: int, out_ptr: int, status_ptr: int = 0, stream: int = 0) -> int:
    return check(lib().pa_hash_prepared(plan.handle, key_ptr, out_ptr, status_ptr or None, stream or None),
                 "pa_hash_prepared")


def pa_debug_mmh(plan: Plan, key_ptr: int, seed_ptr: int, y_ptr: int, status_ptr: int = 0, stream: int = 0) -> int:
    return check(lib().pa_debug_mmh(plan.handle, key_ptr, seed_ptr, y_ptr, status_ptr or None, stream or None),
                 "pa_debug_mmh")


def pa_hash_host(plan: Plan, key: np.ndarray, seed: np.ndarray, stream: int = 0):
    """Host buffers in and out (copies inside).  Returns (status, out words)."""
    key = np.ascontiguousarray(key, dtype=np.uint64)
    seed = np.ascontiguousarray(seed, dtype=np.uint64)
    if key.size < plan.info.key_words or seed.size < plan.info.seed_words:
        raise ValueError("key or seed shorter than the plan requires")
    out = np.zeros(plan.info.out_words, dtype=np.uint64)
    rc = check(lib().pa_hash_host(plan.handle, key.ctypes.data, seed.ctypes.data, out.ctypes.data,
                                  stream or None), "pa_hash_host")
    return rc, out


def pa_hash_batch(plans, key_ptrs, seed_ptrs, out_ptrs, statuses_ptr: int = 0, stream: int = 0) -> int:
    n = len(plans)
    arr = lambda xs: (_vp * n)(*xs)  # noqa: E731
    return check(lib().pa_hash_batch(arr([p.handle.value for p in plans]), arr(key_ptrs), arr(seed_ptrs),
                                     arr(out_ptrs), statuses_ptr or None, n, stream or None), "pa_hash_batch")


def trace_enable(on: bool) -> None:
    check(lib().pa_trace_enable(1 if on else 0), "pa_trace_enable")


def trace_select(name: str | None) -> None:
    """Record only the launches called `name` (None: all)."""
    check(lib().pa_trace_select(name.encode() if name else None), "pa_trace_select")


def trace_collect() -> dict:
    """{name: (launches, total_ms)} for the launches recorded since trace_enable(True)."""
    ent = (pa_trace_entry * 128)()
    cnt = ctypes.c_int()
    check(lib().pa_trace_collect(ent, 128, ctypes.byref(cnt)), "pa_trace_collect")
    return {ent[i].name.decode(): (int(ent[i].launches), float(ent[i].total_ms)) for i in range(min(cnt.value, 128))}


def field_constants(log_n: int):
    w, t = _u64(), _u64()
    check(lib().pa_field_constants(log_n, ctypes.byref(w), ctypes.byref(t)), "pa_field_constants")
    return int(w.value), int(t.value)


def transform_len(G: int, K: int) -> int:
    l = ctypes.c_uint32()
    check(lib().pa_transform_len(G, K, ctypes.byref(l)), "pa_transform_len")
    return int(l.value)


def plan_estimate_bytes(n: int, r: int, gamma: int = 0, margin: int = 128, backend: int = BACKEND_AUTO) -> int:
    b = _u64()
    p = params(gamma, margin, backend=backend)
    check(lib().pa_plan_estimate_bytes(n, r, ctypes.byref(p), ctypes.byref(b)), "pa_plan_estimate_bytes")
    return int(b.value)


class Server:
    """``pa_serve_*``: continuous-batching request loop on the current device."""

    def __init__(self, hbm_budget_bytes: int, slots: int = 8, max_queue: int = 0, gamma: int = 0,
                 margin: int = 128, tune: bool = False, backend: int = BACKEND_AUTO):
        cfg = pa_serve_config()
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.slots = slots
        cfg.max_queue = max_queue
        cfg.params = params(gamma, margin, tune, backend)
        h = _vp()
        check(lib().pa_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "pa_serve_create")
        self.handle = h

    def submit(self, n: int, r: int, key_ptr: int, seed_ptr: int, out_ptr: int) -> int:
        t = _u64()
        check(lib().pa_serve_submit(self.handle, n, r, key_ptr, seed_ptr, out_ptr, ctypes.byref(t)),
              "pa_serve_submit")
        return int(t.value)

    def poll(self, ticket: int):
        st = ctypes.c_int()
        rc = lib().pa_serve_poll(self.handle, ticket, ctypes.byref(st))
        if rc == PA_ERR_BUSY:
            return None
        check(rc, "pa_serve_poll")
        return int(st.value)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> int:
        st = ctypes.c_int()
        check(lib().pa_serve_wait(self.handle, ticket, int(timeout_s * 1e9), ctypes.byref(st)), "pa_serve_wait")
        return int(st.value)

    def stats(self) -> dict:
        s = pa_serve_stats()
        check(lib().pa_serve_stats_get(self.handle, ctypes.byref(s)), "pa_serve_stats_get")
        return {name: getattr(s, name) for name, _ in pa_serve_stats._fields_}

    def stats_reset(self):
        check(lib().pa_serve_stats_reset(self.handle), "pa_serve_stats_reset")

    def shutdown(self):
        """Cancel the queued jobs and wait for the running ones; poll, wait and
        stats keep working until close()."""
        check(lib().pa_serve_shutdown(self.handle), "pa_serve_shutdown")

    def close(self):
        if self.handle:
            lib().pa_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_int8_rate(iters: int = 20000, ctas_per_sm: int = 4):
    """(achieved int8 TOPS of mma.sync m16n8k32, ms) on the current device."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    check(lib().pa_tc_int8_rate(iters, ctas_per_sm, ctypes.byref(t), ctypes.byref(ms)), "pa_tc_int8_rate")
    return float(t.value), float(ms.value)
