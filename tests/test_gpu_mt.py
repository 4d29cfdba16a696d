"""Parity of the multi-tile rectangular-slice search (trs_search_mt: slices
of one tile, or rectangles of whole tiles; Sec. 1, Fig. 1b) with the oracle.

Small frames: the whole record (T_min, the Eq. 4 bound, T, Q, the slices and
the list size) equals the oracle's, which enumerates tile grids and groups
their tiles; the library lists partitions of the CTU grid directly.  Full
frames: with two slices the space is every straight cut across the frame,
and up to five slices it is every partition made by recursive full cuts plus
the pinwheels, so T_min and the winner follow from the oracle's rectangle
sums over those sets alone."""

import numpy as np
import pytest

import synth
from gpu_helpers import SSE_ABS, SSE_REL, mt_best

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dec():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_14792_gb300 import runtime
    d = runtime.Decider(max_width=8192, max_height=4096, max_regions=32, max_batch=1)
    yield d
    d.close()


def _tables(dec, plane, times, bd):
    from paper_2012_14792_gb300 import runtime
    H, W = plane.shape
    luma, pitch = runtime.luma_to_device(plane)
    st = dec.stats_buffers(W, H)
    dec.texture_map(luma, W, H, pitch, bd, st)
    tab = dec.tables_buffer(W, H)
    dec.region_tables(st, torch.from_numpy(np.ascontiguousarray(times, np.float32)).cuda(), W, H, tab)
    torch.cuda.synchronize()
    return tab


def _x0x1y0y1(regions):
    """(x0, y0, x1, y1) slices, as the oracle reports them, in the binding's (x0, x1, y0, y1) order."""
    return [(x0, x1, y0, y1) for (x0, y0, x1, y1) in regions]


def _assert_equal(p, ref, count):
    assert p.status == ref["status"], (p.status, ref["status"])
    assert p.candidates == count
    if ref["status"] != 0:
        assert p.winner == -1
        return
    assert (p.t_min_q, p.thr_q, p.t_q, p.q) == (ref["t_min"], ref["thr"], ref["t"], ref["q"])
    assert p.regions() == _x0x1y0y1(ref["regions"])
    assert abs(p.sse - ref["sse"]) <= max(SSE_REL * abs(ref["sse"]), SSE_ABS)
    assert p.t_min == p.t_min_q / 65536.0 and p.t == p.t_q / 65536.0


CASES = [(832, 480, 4, 0.1, 1), (832, 480, 6, 0.1, 2), (640, 640, 5, 0.0, 3), (1024, 512, 4, 0.3, 4),
         (768, 768, 3, 0.1, 5), (300, 200, 3, 0.0, 6), (128, 128, 1, 0.0, 7), (1000, 700, 4, 0.1, 8),
         (129, 385, 2, 0.05, 9), (640, 256, 3, 1.0, 10)]


@pytest.mark.parametrize("W,H,n,lam,seed", CASES)
def test_mt_search_matches_oracle(dec, oracle, W, H, n, lam, seed):
    plane, times = synth.small_frame(W, H, 10, seed)
    tab = _tables(dec, plane, times, 10)
    p = dec.search_mt(tab, W, H, n, lam)
    st = oracle.texture(plane, 10)
    Tq, _ = oracle.time_q(times)
    _assert_equal(p, oracle.mt_search(st, Tq, n, lam), oracle.mt_count(W, H, n))


@pytest.mark.parametrize("W,H,n", [(832, 480, 4), (640, 640, 5), (512, 384, 3)])
def test_mt_search_ties(dec, oracle, W, H, n):
    """Flat texture and times on a coarse grid: ties on T and Q everywhere,
    so the winner is decided by the slice-list order alone."""
    rng = np.random.default_rng(W + H + n)
    plane = np.full((H, W), 300, np.uint16)
    C, R = oracle.grid(W, H)
    times = rng.integers(1, 3, size=(R, C)).astype(np.float32)
    tab = _tables(dec, plane, times, 10)
    st = oracle.texture(plane, 10)
    Tq, _ = oracle.time_q(times)
    for lam in (0.0, 0.5):
        _assert_equal(dec.search_mt(tab, W, H, n, lam), oracle.mt_search(st, Tq, n, lam), oracle.mt_count(W, H, n))


@pytest.mark.parametrize("spec_name", ["SPEC_1080P10", "SPEC_2160P10"])
def test_mt_two_slices_full_frame(dec, oracle, spec_name):
    """n = 2: the partitions are the straight cuts x = 1..C-1 (left, right)
    and y = 1..R-1 (top, bottom); the record must be the best of them."""
    spec = getattr(synth, spec_name)
    W, H = spec.width, spec.height
    plane, times = synth.make_frame(spec, seed=31)
    tab = _tables(dec, plane, times, spec.bit_depth)
    st = oracle.texture(plane, spec.bit_depth)
    Tq, _ = oracle.time_q(times)
    C, R = oracle.grid(W, H)
    px = lambda v, ext: min(v * 128, ext)
    sets = [[(0, 0, C, y), (0, y, C, R)] for y in range(1, R)] + [[(0, 0, x, R), (x, 0, C, R)] for x in range(1, C)]
    cands = []
    for s in sets:
        areas = [(px(x1, W) - px(x0, W)) * (px(y1, H) - px(y0, H)) for (x0, y0, x1, y1) in s]
        if not 3 * min(areas) > max(areas):
            continue
        tq = [oracle.rect(st, Tq, x0, x1, y0, y1) for (x0, y0, x1, y1) in s]
        key = sorted((y0, x0, y1, x1) for (x0, y0, x1, y1) in s)
        cands.append((key, max(t for t, _ in tq), sum(q for _, q in tq), s))
    t_min = min(c[1] for c in cands)
    for lam in (0.0, 0.1):
        lq = oracle.lambda_q(lam)
        thr = t_min * (65536 + lq) // 65536
        best = min((c for c in cands if c[1] <= thr), key=lambda c: (c[2], c[0]))
        p = dec.search_mt(tab, W, H, 2, lam)
        assert p.status == 0 and p.candidates == len(cands)
        assert (p.t_min_q, p.thr_q, p.t_q, p.q) == (t_min, thr, best[1], best[2])
        assert p.regions() == _x0x1y0y1(sorted(best[3], key=lambda r: (r[1], r[0])))


@pytest.mark.parametrize("spec_name,n", [("SPEC_1080P10", 3), ("SPEC_1080P10", 4), ("SPEC_1080P10", 5),
                                         ("SPEC_2160P10", 3), ("SPEC_2160P10", 4), ("SPEC_2160P10", 5)])
def test_mt_full_frames_up_to_five_slices(dec, oracle, spec_name, n):
    """Up to five slices every partition has a full cut or is a pinwheel, so
    those two lists are the whole space at full frame sizes."""
    import bruteforce
    spec = getattr(synth, spec_name)
    W, H = spec.width, spec.height
    plane, times = synth.make_frame(spec, seed=35)
    tab = _tables(dec, plane, times, spec.bit_depth)
    st = oracle.texture(plane, spec.bit_depth)
    Tq, _ = oracle.time_q(times)
    sets = bruteforce.cut_partitions(W, H, n)
    for lam in (0.0, 0.1):
        ref = mt_best(oracle, st, Tq, sets, lam)
        p = dec.search_mt(tab, W, H, n, lam)
        assert p.status == ref["status"] == 0 and p.candidates == ref["count"]
        assert (p.t_min_q, p.thr_q, p.t_q, p.q) == (ref["t_min"], ref["thr"], ref["t"], ref["q"])
        assert p.regions() == _x0x1y0y1(ref["regions"])


@pytest.mark.parametrize("spec_name,n", [("SPEC_1080P10", 6), ("SPEC_1080P10", 7), ("SPEC_2160P10", 5)])
def test_mt_full_frames_six_and_seven_slices(dec, oracle, spec_name, n):
    """The benchmarked 1920x1080 searches (n = 6: 75,106 slice sets, n = 7:
    535,242) against the oracle's search over every partition of the CTU
    grid into n rectangles, evaluated by direct sums."""
    spec = getattr(synth, spec_name)
    W, H = spec.width, spec.height
    plane, times = synth.make_frame(spec, seed=7)
    tab = _tables(dec, plane, times, spec.bit_depth)
    st = oracle.texture(plane, spec.bit_depth)
    Tq, _ = oracle.time_q(times)
    for lam in (0.0, 0.1):
        ref = oracle.mt_search_rects(st, Tq, n, lam)
        _assert_equal(dec.search_mt(tab, W, H, n, lam), ref, ref["count"])


def test_mt_full_frame_eight_slices_golden(dec):
    """The benchmarked 1920x1080 search with n = 8 (3,889,333 slice sets) on
    the same seeded frame, against the oracle's records stored in
    tests/golden/mt_1080p10_n8.json (its enumeration takes about a minute
    per lambda, so the records are written once by make_mt_golden.py)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mt_1080p10_n8.json")) as f:
        g = json.load(f)
    spec = getattr(synth, g["spec"])
    W, H = spec.width, spec.height
    plane, times = synth.make_frame(spec, seed=g["seed"])
    tab = _tables(dec, plane, times, spec.bit_depth)
    for ref in g["records"]:
        ref = dict(ref, regions=[tuple(r) for r in ref["regions"]])
        _assert_equal(dec.search_mt(tab, W, H, g["n"], ref["lambda"]), ref, ref["count"])


@pytest.mark.parametrize("W,H,n,tscale", [(640, 512, 8, 1.0), (896, 512, 8, 4000.0), (768, 640, 9, 1.0),
                                          (768, 512, 10, 4000.0), (640, 640, 12, 1.0)])
def test_mt_eight_and_more_slices(dec, oracle, W, H, n, tscale):
    """Slice counts 8 (the largest with a kernel compiled for its count) and
    9-12 (the generic kernel) against the oracle's rectangle-partition
    search; tscale = 4000 makes the frame's total Q16 time exceed 2^31, so
    the passes read 64-bit times."""
    rng = np.random.default_rng(n * 31 + W)
    plane = rng.integers(0, 1024, (H, W)).astype(np.uint16)
    C, R = -(-W // 128), -(-H // 128)
    times = (rng.uniform(0.5, 2.0, (R, C)) * tscale).astype(np.float32)
    tab = _tables(dec, plane, times, 10)
    st = oracle.texture(plane, 10)
    Tq, _ = oracle.time_q(times)
    assert (int(Tq.astype(np.int64).sum()) >= 2 ** 31) == (tscale > 1.0)
    for lam in (0.0, 0.1):
        ref = oracle.mt_search_rects(st, Tq, n, lam)
        _assert_equal(dec.search_mt(tab, W, H, n, lam), ref, ref["count"])


def test_mt_no_valid_set_and_out_of_range(dec, oracle):
    plane, times = synth.small_frame(256, 256, 10, 1)
    tab = _tables(dec, plane, times, 10)
    p = dec.search_mt(tab, 256, 256, 5, 0.0)             # four CTUs cannot hold five slices
    assert p.status == oracle.EINFEASIBLE and p.candidates == 0 and p.winner == -1
    bad = plane.copy()
    bad[255, 255] = 1024                                 # above the 10-bit range
    p = dec.search_mt(_tables(dec, bad, times, 10), 256, 256, 2, 0.0)
    assert p.status == oracle.ERANGE


def test_mt_invalid_arguments(dec):
    from paper_2012_14792_gb300 import trs
    plane, times = synth.small_frame(256, 256, 10, 1)
    tab = _tables(dec, plane, times, 10)
    out = torch.zeros(trs.MT_PARTITION_BYTES, dtype=torch.uint8, device="cuda")
    for args in [(tab, 256, 256, 0, 0.0), (tab, 256, 256, 33, 0.0), (tab, 256, 256, 2, -1.0),
                 (tab, 256, 256, 2, float("nan")), (tab.data_ptr() + 16, 256, 256, 2, 0.0),
                 (tab, 9000, 256, 2, 0.0), (0, 256, 256, 2, 0.0)]:
        with pytest.raises(trs.TrsError) as e:
            trs.trs_search_mt(dec.ctx, args[0], args[1], args[2], args[3], args[4], out)
        assert e.value.status == trs.EINVAL


def test_mt_cached_lists_repeat(dec, oracle):
    """Alternating shapes reuse each shape's device list; results repeat bit for bit."""
    frames = [(832, 480, 4), (640, 640, 5), (832, 480, 3)]
    first = []
    for W, H, n in frames:
        plane, times = synth.small_frame(W, H, 10, 40 + n)
        tab = _tables(dec, plane, times, 10)
        first.append((tab, bytes(dec.search_mt(tab, W, H, n, 0.1))))
    for (W, H, n), (tab, b) in zip(frames, first):
        assert bytes(dec.search_mt(tab, W, H, n, 0.1)) == b


def test_mt_contains_single_tile_row_space(dec):
    """The multi-tile space holds every single-tile-row partition, so its
    T_min is never above trs_search's."""
    spec = synth.SPEC_1080P10
    plane, times = synth.make_frame(spec, seed=33)
    tab = _tables(dec, plane, times, spec.bit_depth)
    for n in (3, 4, 6):
        one = dec.partitions(dec.search(tab, spec.width, spec.height, n, 0.1))[0]
        mt = dec.search_mt(tab, spec.width, spec.height, n, 0.1)
        assert one.status == 0 and mt.status == 0
        assert mt.t_min_q <= one.t_min_q
        assert mt.candidates >= 1
