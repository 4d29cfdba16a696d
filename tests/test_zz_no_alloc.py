"""trs_search_noalloc, the search entry point for callers that cannot
allocate device memory (real-time loops that cannot absorb cudaMalloc's
device synchronisation, hosts whose own pool allocator owns all device
memory), must return exactly what trs_search returns, and the oracle's
decision.  Calls in a row on one shape check that the shared scratch array
carries nothing over; later calls swap shapes, go back to an earlier one,
and cover 832x480, a flat frame whose ties only the canonical code decides,
n = 32 (TRS_MAX_REGIONS) and an area-rule factor k = 2.  Collected last, so
a stop at the first failure has run every other test."""

import numpy as np
import pytest

import synth
from gpu_helpers import SSE_ABS, SSE_REL, assert_partition_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tables(dec, plane, times, bd):
    H, W = plane.shape
    raw = np.ascontiguousarray(plane).view(np.uint8)
    luma = torch.from_numpy(raw).cuda()
    st = dec.stats_buffers(W, H)
    dec.texture_map(luma, W, H, raw.strides[0], bd, st)
    tab = dec.tables_buffer(W, H)
    dec.region_tables(st, torch.from_numpy(np.ascontiguousarray(times)).cuda(), W, H, tab)
    return tab, (luma, st)


def _same(a, b):
    ints = ("status", "n_regions", "cols", "rows", "n_tile_cols", "n_tile_rows", "n_windows", "t_min_q",
            "thr_q", "t_q", "q", "tile_row_mask")
    for name in ints:
        assert getattr(a, name) == getattr(b, name), name
    assert a.x_edges() == b.x_edges() and a.band_cuts() == b.band_cuts() and a.regions() == b.regions()
    assert abs(a.sse - b.sse) <= max(SSE_REL * abs(b.sse), SSE_ABS)
    assert a.t == b.t and a.t_min == b.t_min


def _frame(kind, seed):
    if kind == "flat1080":
        # one sample value everywhere and equal CTU times: Q = 0 and T ties
        return np.full((1080, 1920), 300, np.uint16), np.ones((9, 15), np.float32), 10
    spec = {"480": synth.SPEC_480P8, "1080": synth.SPEC_1080P10, "2160": synth.SPEC_2160P10}[kind]
    plane, times = synth.make_frame(spec, seed)
    return plane, times, spec.bit_depth


# (frame kind, seed, n, k, lambda), in call order
CALLS = [
    ("2160", 0, 16, 3, 0.1), ("2160", 1, 16, 3, 0.1),  # two calls in a row on one shape
    ("1080", 2, 8, 3, 0.1),                             # a swap
    ("2160", 3, 16, 3, 0.1),                            # back to the earlier shape
    ("480", 0, 4, 3, 0.3),
    ("flat1080", 0, 8, 3, 0.0),
    ("1080", 4, 32, 3, 0.1),                            # n = TRS_MAX_REGIONS
    ("480", 1, 6, 2, 0.1), ("1080", 5, 8, 2, 0.0),      # k = 2
    ("1080", 6, 8, 3, 0.1),                             # k back to 3 on a shape seen with k = 2
    ("2160", 7, 16, 3, 0.0),
]


def test_noalloc_matches_trs_search_and_oracle(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_14792_gb300 import runtime, trs
    decs = {k: runtime.Decider(max_width=3840, max_height=2160, max_regions=32, k_area=k) for k in (2, 3)}
    try:
        for kind, seed, n, k, lam in CALLS:
            plane, times, bd = _frame(kind, seed)
            H, W = plane.shape
            dec = decs[k]
            tab, keep = _tables(dec, plane, times, bd)
            ref = dec.search(tab, W, H, n, lam)
            got = torch.full((trs.PARTITION_BYTES,), 0xAB, dtype=torch.uint8, device="cuda")
            trs.trs_search_noalloc(tab, W, H, n, k, lam, got)
            torch.cuda.synchronize()
            a, b = dec.partitions(got)[0], dec.partitions(ref)[0]
            assert b.status == 0, (kind, n, k)
            _same(a, b)
            want, _, _ = oracle.decide(plane, times, bd, n, lam, k_area=k)
            assert_partition_equal(a, want, -(-H // 128))
    finally:
        for d in decs.values():
            d.close()


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
