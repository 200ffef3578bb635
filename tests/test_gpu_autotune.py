"""The tile-shape autotuner on the device: it picks one of the candidate tile
heights, records it in the cache file, a new context starts from the file,
and a solve with the tuned shape agrees with the default one."""
import numpy as np
import pytest

from paper_2408_00598_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def test_autotune_picks_records_and_reloads(tmp_path):
    from paper_2408_00598_gb300 import hot
    hot.load_library()
    path = str(tmp_path / "tune.txt")
    import torch
    dev = torch.cuda.get_device_name(0).replace(" ", "_")
    S = 64
    mu1, mu2 = syn.make_pair("gauss", S, 3)
    with hot.Context(precision="fp32") as c0:
        r0 = c0.solve(mu1, mu2, tol=1e-6)
        c0.release(r0)
    with hot.Context(precision="fp32", autotune_cache=path.encode()) as c1:
        tr, us = c1.autotune(S)
        assert tr >= 1 and S * tr <= 16384 and us > 0
        r1 = c1.solve(mu1, mu2, tol=1e-6)
        c1.release(r1)
    assert hot.hot_autotune_cache_lookup(path, dev, hot.HOT_FP32_BULK, S)[0] == tr
    with hot.Context(precision="fp32", autotune_cache=path.encode()) as c2:
        r2 = c2.solve(mu1, mu2, tol=1e-6)
        c2.release(r2)
    assert r1["status"] == r2["status"] == r0["status"] == 0
    # the same shape from the file: bit-identical to the tuned context
    assert r2["ot_value"] == r1["ot_value"] and r2["iters"] == r1["iters"]
    # another shape only regroups FP32 sums
    assert abs(r1["dual_value"] - r0["dual_value"]) <= 1e-6 * abs(r0["dual_value"])


def test_autotune_rejects_bad_sizes():
    from paper_2408_00598_gb300 import hot
    with hot.Context(precision="fp32") as c:
        for S in (1, 1025):
            with pytest.raises(hot.HotError):
                c.autotune(S)
