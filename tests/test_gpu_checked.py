"""The bounds-checked build of the library (libgsc_checked.so, built with
GSC_DEBUG_BOUNDS): every data-indexed store (compaction offsets, cache lines
and miss lists, scan scatters, sort ranks, tile ranges) tests its index
against the buffer's capacity and, on a miss, flags the frame and skips the
store.  It stands in for a device memory checker.  A child process loads it
(GSC_LIBRARY) and renders the tiny scene, 14 frames of the city path in the
headline form and a batched multi-model frame (13 images, cached BF16 exact
stereo, per-tile and persistent blend); no frame may flag an out-of-range
store, and the images must equal those of the normal build."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKED = os.path.join(ROOT, "paper_2502_14938_b300", "libgsc_checked.so")

RENDER = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import gen, paper_2502_14938_b300 as pkg
from test_gpu_parity import make_renderer, render
out = {{}}
m, cam = gen.tiny_scene(), gen.tiny_camera()
r = make_renderer(m, [cam], pair_capacity=1000)  # grows (re-render) on the first frame
(img,), st = render(r, [cam]); out["tiny"] = img; out["tiny_err"] = st["error_flags"]; r.close()
model, frames = gen.city_workload(n_frames=40)
r = make_renderer(model, list(frames[0]), partners=[1, 0], reuse="depth", stereo_unify="exact", precision="bf16")
r.set_tiling(16, 64, 0)
for f in range(0, 40, 3):
    imgs, st = render(r, list(frames[f]))
    out[f"city{{f}}"] = np.stack(imgs); out[f"city{{f}}_err"] = st["error_flags"]
r.close()
from test_gpu_batched import batched_renderer, render_all
models, viewers, frame_fn = gen.multiviewer_workload(scale=0.02, size_scale=0.25)
images = frame_fn(40)
r, _ = batched_renderer(models, images, stereo_unify="exact", precision="bf16", reuse="depth", tile=(16, 64))
for bps in (0, 4):  # one block per tile, then the persistent blend
    r.set_tiling(16, 64, bps)
    imgs, st = render_all(r, images)
    out[f"batched{{bps}}"] = np.concatenate([i.ravel() for i in imgs]); out[f"batched{{bps}}_err"] = st["error_flags"]
r.close()
np.savez({path!r}, **out)
"""


def run_child(path, lib=None):
    env = dict(os.environ)
    if lib:
        env["GSC_LIBRARY"] = lib
    code = RENDER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), path=path)
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    return dict(np.load(path))


def test_bounds_checked_build_renders_the_same(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    assert os.path.exists(CHECKED), "libgsc_checked.so not built (paper_2502_14938_b300.build.build(checked=True))"
    checked = run_child(str(tmp_path / "checked.npz"), CHECKED)
    normal = run_child(str(tmp_path / "normal.npz"))
    assert set(checked) == set(normal)
    for k in sorted(checked):
        if k.endswith("_err"):
            assert int(checked[k]) == 0, f"{k}: error flags {int(checked[k])}"
        else:
            assert np.array_equal(checked[k], normal[k]), k
