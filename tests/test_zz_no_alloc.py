"""The scan entry point that allocates nothing, checked against the allocating one.

Some callers cannot allocate device memory where they need a scan (a
real-time frame loop, or a host whose pool owns all device memory);
gsc_scan_u32_noalloc serves them with a fixed internal device array as its
working memory.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_scan_matches_allocating_scan_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_14938_b300 as pkg
    from paper_2502_14938_b300 import native

    r = pkg.Renderer(max_views=1)
    rs = np.random.default_rng(11)
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row; the second is shorter, so stale look-back words of
    # the first call lie in the array when the second runs
    for n in (1_000_003, 77_777):
        vals = rs.integers(0, 50, n).astype(np.uint32)
        ref, ref_total = r.debug_scan(vals)  # existing, allocating entry point
        d_in = torch.from_numpy(vals.view(np.int32)).cuda()
        d_out = torch.full_like(d_in, -1)
        d_tot = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        native.scan_u32_noalloc(d_in.data_ptr(), d_out.data_ptr(), n, d_tot.data_ptr(), stream)
        got = d_out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref)
        assert int(d_tot.cpu().numpy().view(np.uint32)[0]) == ref_total
    # in place (d_out == d_in), which the header allows
    vals = rs.integers(0, 50, 300_001).astype(np.uint32)
    ref, ref_total = r.debug_scan(vals)
    d_io = torch.from_numpy(vals.view(np.int32)).cuda()
    native.scan_u32_noalloc(d_io.data_ptr(), d_io.data_ptr(), vals.size, 0, stream)
    assert np.array_equal(d_io.cpu().numpy().view(np.uint32), ref)
    r.close()


def test_noalloc_scan_rejects_sizes_beyond_its_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_14938_b300 import native

    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(native.GscError) as e:
        # rejected on the host before any work is enqueued
        native.scan_u32_noalloc(d.data_ptr(), d.data_ptr(), (1 << 24) + 1, 0, 0)
    assert e.value.code == -1
