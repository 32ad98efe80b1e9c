"""Programmatic dependent launch in the frame graph: each kernel that follows
a kernel in its stream may be scheduled while that one finishes, and waits
(griddepcontrol.wait) before its first memory access.  The frames must be
bit-for-bit those of the graph without programmatic edges
(FLAG_NO_DEP_LAUNCH), with the same cache decisions and counts, in the
forked cached form (the plan and the tables on a second branch), in the
uncached FP32 form (one stream) and in a batched multi-model frame with the
persistent blend (derivation after derivation)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import gen  # noqa: E402
from test_gpu_parity import make_renderer, render  # noqa: E402

STAT_KEYS = ("visible_anchors", "derived_anchors", "records", "valid_records", "pairs", "cache_depth",
             "error_flags")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _path(flags, model, frames, **kw):
    r = make_renderer(model, list(frames[0]), partners=[1, 0], flags=flags, **kw)
    r.set_tiling(16, 64, 0)
    out = []
    for f in range(0, 30, 2):
        imgs, st = render(r, list(frames[f]))
        out.append((np.stack(imgs), {k: st[k] for k in STAT_KEYS}))
    r.close()
    return out


_city = []


@pytest.mark.parametrize("form", [dict(reuse="depth", stereo_unify="exact", precision="bf16"),
                                  dict(precision="fp32")], ids=["cached_bf16_exact", "plain_fp32"])
def test_dep_launch_frames_equal_plain_graph(form):
    _need_gpu()
    import paper_2502_14938_b300 as pkg
    if not _city:
        _city.append(gen.city_workload(n_frames=30))
    model, frames = _city[0]
    dep = _path(0, model, frames, **form)
    plain = _path(pkg.FLAG_NO_DEP_LAUNCH, model, frames, **form)
    for i, ((a, sa), (b, sb)) in enumerate(zip(dep, plain)):
        assert sa == sb, (i, sa, sb)
        assert sa["error_flags"] == 0
        assert np.array_equal(a, b), f"frame {2 * i}: images differ"


def test_dep_launch_batched_frame_equal():
    _need_gpu()
    import paper_2502_14938_b300 as pkg
    from test_gpu_batched import batched_renderer, render_all
    models, viewers, frame_fn = gen.multiviewer_workload(scale=0.02, size_scale=0.25)
    images = frame_fn(40)
    got = {}
    for flags in (0, pkg.FLAG_NO_DEP_LAUNCH):
        r, _ = batched_renderer(models, images, stereo_unify="exact", precision="bf16", reuse="depth",
                                tile=(16, 64), flags=flags)
        r.set_tiling(16, 64, 4)
        runs = []
        for _ in range(3):  # the cache fills over the repeats
            imgs, st = render_all(r, images)
            assert st["error_flags"] == 0
            runs.append(np.concatenate([i.ravel() for i in imgs]))
        got[flags] = runs
        r.close()
    for a, b in zip(got[0], got[pkg.FLAG_NO_DEP_LAUNCH]):
        assert np.array_equal(a, b)
