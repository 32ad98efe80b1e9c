"""The bench's host-side bookkeeping, on CPU: the roofline's DRAM traffic is
reported only while the kernel's code (comments aside) is the one the ncu
capture was taken on and the timed run uses the captured tiling; the launch count per
frame follows the form's kernels."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_only_for_the_captured_source_and_tiling(monkeypatch):
    c = bench.NCU_TRAFFIC["k_blend"]
    got, why = bench.ncu_traffic("k_blend", tuple(c["tiling"]))
    assert got == c["bytes"] and got > 0, why
    assert bench.ncu_traffic("k_blend", (16, 16, 0))[0] is None  # another tiling
    assert bench.ncu_traffic("k_nothing", tuple(c["tiling"]))[0] is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, "k_blend", dict(c, sha16="0" * 16))  # the source changed
    assert bench.ncu_traffic("k_blend", tuple(c["tiling"]))[0] is None


def test_source_key_ignores_comments_but_not_code(tmp_path):
    f = tmp_path / "k.cu"
    f.write_text("int a = 1;  // one\n\n__global__ void k() {}\n")
    h = bench._src_sha16(str(f))
    f.write_text("// a new header comment\nint a = 1;\n__global__ void k() {}  // edited\n")
    assert bench._src_sha16(str(f)) == h
    f.write_text("int a = 2;\n__global__ void k() {}\n")
    assert bench._src_sha16(str(f)) != h


def test_launches_per_frame_follow_the_form():
    # frame setup, cull (2), plan, tables, derivation, projection, record sort (4 launches), scan,
    # key generation, tile sort (2 for a 12-bit tile key), ranges, blend
    assert bench.launches_per_frame_of("plain", 12) == 17
    assert bench.launches_per_frame_of("bf16_exact", 12) == 17
    # + the cache's free-line scan and assignment (the depth-rule probe runs in the cull)
    assert bench.launches_per_frame_of("cached_bf16_exact", 12) == 19
    # one more tile-sort pass for a tile key of more than 16 bits
    assert bench.launches_per_frame_of("cached_bf16_exact", 16) == 19
    assert bench.launches_per_frame_of("cached_bf16_exact", 17) == 20
