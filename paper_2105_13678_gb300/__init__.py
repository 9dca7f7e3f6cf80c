"""GB300-native MMH-MH privacy amplification (arXiv 2105.13678).

The hash runs in ``libpa_gb300.so`` (hand-written CUDA for sm_103a behind the
C ABI of ``include/pa_gb300.h``); ``_lib`` is its ctypes binding.  Importing
this package does not load the library; the first call does, and fails loudly
if it has not been built.
"""
from . import synthetic  # noqa: F401  (input generator, no hash arithmetic)


def __getattr__(name):
    if name in ("Plan", "Server", "pa_hash", "pa_hash_host", "pa_hash_batch", "pa_debug_mmh", "lib",
                "field_constants", "transform_len", "plan_estimate_bytes", "PAError"):
        from . import _lib
        return getattr(_lib, name)
    raise AttributeError(name)
