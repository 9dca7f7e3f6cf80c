"""The tensor-core limb-convolution tile (int8 mma.sync) is exact: every entry
equals the integer convolution numpy computes for the same limbs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_limbconv_tile_is_exact():
    import torch
    from paper_2105_13678_gb300 import _lib
    rng = np.random.default_rng(5)
    nt = 300
    bq = rng.integers(0, 256, size=(nt, 32), dtype=np.uint8)
    a = rng.integers(0, 256, size=(nt, 8, 32), dtype=np.uint8)
    bq[0] = 255
    a[0] = 255  # the largest coefficient: 32 * 255^2
    dbq, da = torch.from_numpy(bq).cuda(), torch.from_numpy(a).cuda()
    out = torch.full((nt, 64, 8), -1, dtype=torch.int32, device="cuda")
    _lib.check(_lib.lib().pa_tc_limbconv_tile(dbq.data_ptr(), da.data_ptr(), out.data_ptr(), nt,
                                              torch.cuda.current_stream().cuda_stream), "limbconv")
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for t in range(nt):
        for c in range(8):
            ref = np.zeros(64, dtype=np.int64)
            ref[:63] = np.convolve(bq[t].astype(np.int64), a[t, c].astype(np.int64))
            assert np.array_equal(got[t, :, c], ref), (t, c)


def test_int8_rate_is_measured():
    from paper_2105_13678_gb300 import _lib
    tops, ms = _lib.tc_int8_rate(2000, 2)
    assert tops > 0 and ms > 0
