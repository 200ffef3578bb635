"""Host-side logic of the tile-shape autotuner: the cache file format read by
hot_autotune_cache_lookup (no GPU needed)."""
import pytest

from paper_2408_00598_gb300 import hot


def test_cache_lookup(tmp_path):
    f = tmp_path / "tune.txt"
    f.write_text("# device precision S TR us\n"
                 "NVIDIA_GB300 fp32 256 64 80.5\n"
                 "NVIDIA_GB300 fp64 256 16 300.0\n"
                 "Other_GPU fp32 256 32 90.0\n"
                 "garbage line\n"
                 "NVIDIA_GB300 fp32 256 32 78.25\n"      # later entry for the same key wins
                 "NVIDIA_GB300 fp32 128 32 9.5\n")
    assert hot.hot_autotune_cache_lookup(str(f), "NVIDIA_GB300", hot.HOT_FP32_BULK, 256) == (32, 78.25)
    assert hot.hot_autotune_cache_lookup(str(f), "NVIDIA_GB300", hot.HOT_FP64, 256) == (16, 300.0)
    assert hot.hot_autotune_cache_lookup(str(f), "Other_GPU", hot.HOT_FP32_BULK, 256) == (32, 90.0)
    assert hot.hot_autotune_cache_lookup(str(f), "NVIDIA_GB300", hot.HOT_FP32_BULK, 512) is None
    assert hot.hot_autotune_cache_lookup(str(tmp_path / "missing.txt"), "NVIDIA_GB300", hot.HOT_FP32_BULK, 256) is None
