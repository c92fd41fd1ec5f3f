"""The smoke check of the build entry points: one small render, backward,
background loss and contribution sweep on cuda:0 against the FP64 oracle,
with the rasterizer's default configuration (16x16 tiles, four pixels per
thread, persistent queue, two-pass binning)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as entry
    entry.build()
    entry.smoke()
