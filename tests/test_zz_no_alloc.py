"""trs_search_noalloc, the search entry point for callers that cannot
allocate device memory (graph-capture regions, real-time loops, hosts with
their own pool allocator), must return exactly what trs_search returns.
Two calls in a row on different frames check that the shared scratch array
carries nothing over; a third call with another shape checks the plan swap.
Collected last, so a stop at the first failure has run every other test."""

import numpy as np
import pytest

import synth
from gpu_helpers import SSE_ABS, SSE_REL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tables(dec, plane, times, bd):
    H, W = plane.shape
    raw = np.ascontiguousarray(plane).view(np.uint8)
    luma = torch.from_numpy(raw).cuda()
    st = dec.stats_buffers(W, H)
    dec.texture_map(luma, W, H, raw.strides[0], bd, st)
    tab = dec.tables_buffer(W, H)
    dec.region_tables(st, torch.from_numpy(times).cuda(), W, H, tab)
    return tab, (luma, st)


def _same(a, b):
    ints = ("status", "n_regions", "cols", "rows", "n_tile_cols", "n_tile_rows", "n_windows", "t_min_q",
            "thr_q", "t_q", "q", "tile_row_mask")
    for name in ints:
        assert getattr(a, name) == getattr(b, name), name
    assert a.x_edges() == b.x_edges() and a.band_cuts() == b.band_cuts() and a.regions() == b.regions()
    assert abs(a.sse - b.sse) <= max(SSE_REL * abs(b.sse), SSE_ABS)
    assert a.t == b.t and a.t_min == b.t_min


def test_noalloc_matches_trs_search():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_14792_gb300 import runtime, trs
    dec = runtime.Decider(max_width=3840, max_height=2160, max_regions=16)
    cases = [(synth.SPEC_2160P10, 0, 16), (synth.SPEC_2160P10, 1, 16), (synth.SPEC_1080P10, 2, 8)]
    for spec, seed, n in cases:
        plane, times = synth.make_frame(spec, seed)
        tab, keep = _tables(dec, plane, times, spec.bit_depth)
        W, H = spec.width, spec.height
        ref = dec.search(tab, W, H, n, 0.1)
        got = torch.full((trs.PARTITION_BYTES,), 0xAB, dtype=torch.uint8, device="cuda")
        trs.trs_search_noalloc(tab, W, H, n, 3, 0.1, got)
        torch.cuda.synchronize()
        a, b = dec.partitions(got)[0], dec.partitions(ref)[0]
        assert b.status == 0
        _same(a, b)
    dec.close()


def test_noalloc_rejects_oversize_shape():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_14792_gb300 import trs
    tab = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    out = torch.zeros(trs.PARTITION_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(trs.TrsError) as e:
        trs.trs_search_noalloc(tab, 8192, 4096, 32, 3, 0.1, out)  # plan and scratch exceed the 8 MiB array
    assert e.value.status == trs.ENOMEM
    with pytest.raises(trs.TrsError) as e:
        trs.trs_search_noalloc(tab, 3840, 2160, 0, 3, 0.1, out)
    assert e.value.status == trs.EINVAL
