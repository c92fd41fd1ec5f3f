"""Host logic of bench.py on CPU: the source digest, the rule that a measured
DRAM figure is reported only for the sources and workload it was captured on,
and the per-launch algorithmic byte model of the backward rasterizer."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

ARGS = "--n 500000 --views 16 --tile 16x16 --persistent 1 --ppt 4 --front 0.1"


def _summary(digest: str, args: str) -> str:
    return (f"# DRAM traffic\n\nsources-sha256: {digest}\nworkload-args: {args}\n\n"
            "| kernel | read B | write B | read + write B | ncu time ms | algorithmic B | ratio |\n"
            "|---|---|---|---|---|---|---|\n"
            "| raster_bwd_kernel | 300 | 20 | 320 | 6.8 | 100 | 3.20 |\n"
            "| raster_fwd_kernel (first pass) | 10 | 5 | 15 | 1.8 | | |\n")


def test_digest_is_stable_and_short():
    a, b = bench.sources_digest(), bench.sources_digest()
    assert a == b and len(a) == 16 and all(c in "0123456789abcdef" for c in a)


def test_traffic_only_for_matching_sources_and_workload(tmp_path, monkeypatch):
    path = tmp_path / "traffic.md"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    assert bench.measured_traffic("raster_bwd_kernel", ARGS) is None  # no summary at all
    path.write_text(_summary(bench.sources_digest(), ARGS))
    assert bench.measured_traffic("raster_bwd_kernel", ARGS) == 320  # read + write column
    assert bench.measured_traffic("preprocess_kernel", ARGS) is None  # no row for it
    assert bench.measured_traffic("raster_bwd_kernel", ARGS.replace("0.1", "0.2")) is None  # other workload
    path.write_text(_summary("0" * 16, ARGS))
    assert bench.measured_traffic("raster_bwd_kernel", ARGS) is None  # counters of other sources


def test_backward_byte_model_at_the_measured_workload():
    # 500k surfels x 16 views, 28,331,624 pairs, 16,080,896 pixels: the backward reads the
    # 72-byte record and writes the 80-byte gradient slot of every view-surfel, reads 4 bytes
    # per pair and 40 bytes of pixel state and cotangents per pixel
    N, V, K, P = 500_000, 16, 28_331_624, 16_080_896
    got = bench.algorithmic("raster_bwd", N, V, P, K, T=62_816, E=2_031_239_432, tile_passes=2, kept=0)
    assert got["bytes"] == N * V * (72 + 80) + 4 * K + 40 * P == 1_972_562_336
    assert got["flops"] == 2_031_239_432 * bench.FLOPS_BWD
