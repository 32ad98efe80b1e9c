"""CPU checks of the boundary: the library builds, loads without a GPU and
exports every symbol its headers declare; the binding's structs match the
C layout."""
import ctypes as C
import subprocess
import numpy as np

import pytest

import paper_2502_14938_b300 as pkg
from paper_2502_14938_b300 import native


def test_library_builds_and_loads():
    from paper_2502_14938_b300 import build
    path = build.build()
    L = pkg.lib()
    assert L.gsc_version() == 1
    assert path.endswith("libgsc.so")


def test_every_declared_symbol_is_exported():
    names = pkg.exported_symbols()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in syms]
    assert not missing, missing
    L = pkg.lib()
    for n in names:
        assert getattr(L, n) is not None


def test_bounds_checked_build_exports_the_same_symbols():
    """The bounds-checked variant (GSC_DEBUG_BOUNDS) is the same ABI."""
    from paper_2502_14938_b300 import build
    path = build.build(checked=True)
    names = pkg.exported_symbols()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert not [n for n in names if n not in syms]


def test_default_config_is_filled_without_gpu():
    c = pkg.default_config()
    assert (c.tile_w, c.tile_h) == (16, 16)
    assert c.pair_capacity == 16 << 20
    assert c.max_depth == 10 and c.use_graph == 1


def test_struct_layouts_match_header(tmp_path):
    """sizeof/offsetof of the header structs, from the C compiler, equal the
    ctypes mirrors of the binding."""
    import os
    inc = os.path.join(os.path.dirname(native.HERE), "include")
    src = tmp_path / "layout.c"
    checks = [("gsc_config", native.Config, ["pair_capacity", "bg", "flags", "blocks_per_sm", "out_format",
                                             "depth_guide"]),
              ("gsc_model_desc", native.ModelDesc, ["pos", "W1", "b2", "level_offset", "lod_blend"]),
              ("gsc_camera", native.Camera, ["fx", "znear", "viewer"]),
              ("gsc_frame_stats", native.FrameStats, ["cache_depth", "ms_stage"])]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gsc.h"', "int main(void){"]
    for cname, _, fields in checks:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    exp = []
    for _, st, fields in checks:
        exp.append(C.sizeof(st))
        exp += [getattr(st, f).offset for f in fields]
    assert got == exp


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = C.c_void_p()
    rc = pkg.lib().gsc_create(C.byref(ctx), None, None)
    assert rc in (-3, -2)  # GSC_ERR_CUDA / GSC_ERR_OOM, no context
    assert not ctx.value


def test_predictor_file_roundtrip(tmp_path):
    from paper_2502_14938_b300 import reuse
    theta = np.random.default_rng(0).standard_normal(native.REUSE_NPARAM).astype(np.float32)
    p = str(tmp_path / "w.gscr")
    reuse.save(p, theta)
    assert np.array_equal(reuse.load(p), theta)
    with open(p, "r+b") as f:
        f.write(b"XXXX")
    with pytest.raises(ValueError):
        reuse.load(p)


def test_autotuner_prefers_one_block_per_tile_within_margin():
    from paper_2502_14938_b300.autotune import order_candidates
    rows = [{"tile_w": 16, "tile_h": 32, "blocks_per_sm": 16, "ms": 0.500},
            {"tile_w": 16, "tile_h": 32, "blocks_per_sm": 0, "ms": 0.505},
            {"tile_w": 16, "tile_h": 16, "blocks_per_sm": 0, "ms": 0.503}]
    assert order_candidates(rows)[0] == rows[1]           # within 2% of the persistent grid
    rows[1]["ms"] = 0.520
    assert order_candidates(rows)[0] == rows[0]           # 4% slower: the persistent grid stays
    only = [{"tile_w": 8, "tile_h": 32, "blocks_per_sm": 4, "ms": 0.4}]
    assert order_candidates(only) == only
    assert order_candidates([]) == []
