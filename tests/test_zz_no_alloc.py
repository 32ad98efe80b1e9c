"""The scan entry point that allocates nothing, checked against np.cumsum and
against the allocating scan.

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

MAX_N = 1 << 24  # GSC_NOALLOC_SCAN_MAX_N


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def excl_cumsum(vals):
    c = np.cumsum(vals.astype(np.int64))
    return np.concatenate([[0], c[:-1]]), int(c[-1]) if len(c) else 0


def run_noalloc(vals, stream, in_place=False):
    from paper_2502_14938_b300 import native
    d_in = torch.from_numpy(vals.view(np.int32)).cuda()
    d_out = d_in if in_place else torch.full_like(d_in, -1)
    d_tot = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    native.scan_u32_noalloc(d_in.data_ptr(), d_out.data_ptr(), vals.size, d_tot.data_ptr(), stream)
    return d_out.cpu().numpy().view(np.uint32).astype(np.int64), int(d_tot.cpu().numpy().view(np.uint32)[0])


def test_noalloc_scan_matches_cumsum_and_allocating_scan_on_two_calls():
    import paper_2502_14938_b300 as pkg

    r = pkg.Renderer(max_views=1)
    rs = np.random.default_rng(11)
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row; the second is shorter, so stale look-back words of
    # the first call lie in the array when the second runs
    for n in (1_000_003, 77_777):
        vals = rs.integers(0, 50, n).astype(np.uint32)
        exp, exp_total = excl_cumsum(vals)
        ref, ref_total = r.debug_scan(vals)  # existing, allocating entry point
        got, tot = run_noalloc(vals, stream)
        assert np.array_equal(got, exp) and tot == exp_total
        assert np.array_equal(got, ref.astype(np.int64)) and tot == ref_total
    # in place (d_out == d_in), which the header allows
    vals = rs.integers(0, 50, 300_001).astype(np.uint32)
    exp, exp_total = excl_cumsum(vals)
    got, tot = run_noalloc(vals, stream, in_place=True)
    assert np.array_equal(got, exp) and tot == exp_total
    r.close()


def test_noalloc_scan_edge_sizes():
    """n = 0 writes a zero total; n = the maximum fills every look-back word
    of the array up to its control words; ragged sizes around a tile."""
    from paper_2502_14938_b300 import native
    stream = torch.cuda.current_stream().cuda_stream
    d_tot = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    native.scan_u32_noalloc(d.data_ptr(), d.data_ptr(), 0, d_tot.data_ptr(), stream)
    assert int(d_tot.cpu()[0]) == 0
    rs = np.random.default_rng(12)
    for n in (1, 4095, 4096, 4097, MAX_N):
        vals = rs.integers(0, 60, n).astype(np.uint32)  # max sum 59 * 2^24 < 2^30
        exp, exp_total = excl_cumsum(vals)
        got, tot = run_noalloc(vals, stream)
        assert np.array_equal(got, exp), n
        assert tot == exp_total, n


def test_noalloc_scan_rejects_sums_from_2_pow_30_and_recovers():
    """The look-back words hold 30-bit prefixes: a sum that reaches 2^30 is
    reported as GSC_ERR_INVALID_ARG, and the next call is correct again."""
    from paper_2502_14938_b300 import native
    stream = torch.cuda.current_stream().cuda_stream
    vals = np.full(1 << 22, 256, np.uint32)  # sum exactly 2^30
    with pytest.raises(native.GscError) as e:
        run_noalloc(vals, stream)
    assert e.value.code == -1
    vals = np.full(1 << 22, 255, np.uint32)  # sum 2^30 - 2^22: accepted
    exp, exp_total = excl_cumsum(vals)
    got, tot = run_noalloc(vals, stream)
    assert np.array_equal(got, exp) and tot == exp_total


def test_noalloc_scan_rejects_sizes_beyond_its_maximum():
    from paper_2502_14938_b300 import native

    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(native.GscError) as e:
        # rejected on the host before any work is enqueued
        native.scan_u32_noalloc(d.data_ptr(), d.data_ptr(), MAX_N + 1, 0, 0)
    assert e.value.code == -1


def test_noalloc_scan_refuses_a_capturing_stream():
    """The call synchronises its stream, which a stream under graph capture
    does not allow: it returns GSC_ERR_INVALID_ARG and enqueues nothing."""
    from paper_2502_14938_b300 import native
    d = torch.arange(8, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    code = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            native.scan_u32_noalloc(d.data_ptr(), d.data_ptr(), 8, 0, s.cuda_stream)
        except native.GscError as e:
            code = e.code
        finally:
            g.capture_end()
    torch.cuda.synchronize()
    assert code == -1
    assert np.array_equal(d.cpu().numpy(), np.arange(8))
