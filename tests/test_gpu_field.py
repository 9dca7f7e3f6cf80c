"""Device F_q arithmetic (q = 2^64 - 2^32 + 1) against Python integers, on
edge values (0, 1, q - 1, q, values in [q, 2^64), limb boundaries) and on
random 64-bit inputs.  The transforms keep values in [0, 2^64) lazily, so the
device ops must be right for every 64-bit input, not only canonical ones."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

Q = 2**64 - 2**32 + 1


def test_field_ops_edge_and_random():
    import torch
    from paper_2105_13678_gb300 import _lib
    edges = [0, 1, 2, 2**32 - 1, 2**32, 2**32 + 1, 2**63, Q - 2, Q - 1, Q, Q + 1, 2**64 - 2**32,
             2**64 - 2, 2**64 - 1, 0xFFFFFFFF00000000, 0x00000000FFFFFFFF, 0x8000000080000000]
    pairs = [(a, b) for a in edges for b in edges]
    rng = np.random.default_rng(1)
    rnd = rng.integers(0, 2**64, size=(20000, 2), dtype=np.uint64)
    a = np.array([p[0] for p in pairs], dtype=np.uint64)
    b = np.array([p[1] for p in pairs], dtype=np.uint64)
    a = np.concatenate([a, rnd[:, 0]])
    b = np.concatenate([b, rnd[:, 1]])
    da = torch.from_numpy(a.view(np.int64)).cuda()
    db = torch.from_numpy(b.view(np.int64)).cuda()
    out = torch.zeros(4 * a.size, dtype=torch.int64, device="cuda")
    _lib.check(_lib.lib().pa_selftest_field(da.data_ptr(), db.data_ptr(), out.data_ptr(), a.size, None), "selftest")
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64).reshape(-1, 4)
    for i in range(a.size):
        x, y = int(a[i]), int(b[i])
        assert int(got[i, 0]) == (x + y) % Q, (hex(x), hex(y), "add")
        assert int(got[i, 1]) == (x - y) % Q, (hex(x), hex(y), "sub")
        assert int(got[i, 2]) == (x * y) % Q, (hex(x), hex(y), "mul")
        assert int(got[i, 3]) == ((x & 0xFFFFFFFF) * y) % Q, (hex(x), hex(y), "mul_small")
