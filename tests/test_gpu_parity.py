"""Parity of the CUDA path (through the C ABI) with the oracle: bit-exact
texture statistics, Q16 times, SATs, rectangle tables and partitions; the
reported floating-point SSE within 1e-6 relative."""

import numpy as np
import pytest

import golden_cases
import synth
from gpu_helpers import assert_partition_equal, assert_valid_partition

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dec():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_14792_gb300 import runtime
    d = runtime.Decider(max_width=8192, max_height=4096, max_regions=32, max_batch=64)
    yield d
    d.close()


def _dev(plane, pad_to=None, offset=0):
    """Device copy of a plane with an optional row pitch and byte offset."""
    raw = np.ascontiguousarray(plane).view(np.uint8)
    H, rb = raw.shape
    pitch = rb if pad_to is None else pad_to
    buf = np.zeros(offset + pitch * H + 64, np.uint8)
    for y in range(H):
        buf[offset + y * pitch: offset + y * pitch + rb] = raw[y]
    t = torch.from_numpy(buf).cuda()
    return t, t.data_ptr() + offset, pitch


def _texture(dec, plane, bd, pad_to=None, offset=0):
    H, W = plane.shape
    t, ptr, pitch = _dev(plane, pad_to, offset)
    st = dec.stats_buffers(W, H)
    dec.texture_map(ptr, W, H, pitch, bd, st)
    torch.cuda.synchronize()
    u32 = lambda x: x.cpu().numpy().view(np.uint32)
    return dict(s1=u32(st["s1"]), s2=st["s2"].cpu().numpy().view(np.uint64), count=u32(st["count"]),
                vmax=u32(st["vmax"]), flags=int(u32(st["flags"])[0])), st, t


@pytest.mark.parametrize("W,H,bd,pad,offset", [
    (832, 480, 8, None, 0), (1920, 1080, 10, None, 0), (3840, 2160, 10, None, 0),
    (1000, 700, 10, None, 0), (129, 257, 8, None, 0), (1, 1, 8, None, 0), (130, 3, 12, None, 0),
    (1920, 1080, 10, 4096, 0), (833, 481, 8, 848, 0),        # padded, aligned pitch
    (300, 200, 10, 602, 0), (300, 200, 10, None, 2),          # unaligned pitch / base: scalar path
    (8192, 4096, 10, None, 0),                                # largest frame
])
def test_texture_bit_exact(dec, oracle, W, H, bd, pad, offset):
    rng = np.random.default_rng(W * 7 + H + bd)
    dt = np.uint8 if bd == 8 else np.uint16
    plane = rng.integers(0, 2 ** bd, size=(H, W)).astype(dt)
    got, _, _ = _texture(dec, plane, bd, pad, offset)
    ref = oracle.texture(plane, bd)
    assert (got["s1"] == ref.S1.ravel()).all()
    assert (got["s2"] == ref.S2.ravel()).all()
    assert (got["count"] == ref.N.ravel()).all()
    assert (got["vmax"] == ref.vmax.ravel()).all()
    assert got["flags"] == 0


def test_texture_flags_out_of_range_sample(dec, oracle):
    plane = np.zeros((300, 300), np.uint16)
    plane[299, 299] = 1024
    got, _, _ = _texture(dec, plane, 10)
    assert got["flags"] == 1
    assert oracle.texture(plane, 10).status == oracle.ERANGE


def _check_every_band(oracle, got, ref, Tq):
    """Every slice of every tile column in the GPU's rectangle table (time and
    floor SSE) against the oracle's direct sums of the same rectangle."""
    R, C = Tq.shape
    t_all, q_all = oracle.rect_all(ref, Tq)
    for x0 in range(C):
        for x1 in range(x0 + 1, C + 1):
            b = x0 * (2 * C - x0 + 1) // 2 + (x1 - x0 - 1)
            for d in range(1, R + 1):
                y = np.arange(R - d + 1)
                assert (got["rect_t"][b, d - 1, : R - d + 1] == t_all[x0, x1, y, y + d]).all(), (x0, x1, d)
                assert (got["rect_q"][b, d - 1, : R - d + 1] == q_all[x0, x1, y, y + d]).all(), (x0, x1, d)


@pytest.mark.parametrize("W,H,seed", [(832, 480, 1), (1920, 1080, 2), (3840, 2160, 3), (200, 520, 4)])
def test_tables_bit_exact(dec, oracle, W, H, seed):
    plane, times = synth.small_frame(W, H, 10, seed)
    _, st, _keep = _texture(dec, plane, 10)
    tt = torch.from_numpy(times).cuda()
    tab = dec.tables_buffer(W, H)
    dec.region_tables(st, tt, W, H, tab)
    torch.cuda.synchronize()
    got = dec.read_tables(tab, W, H)
    ref = oracle.texture(plane, 10)
    Tq, s = oracle.time_q(times)
    assert got["status"][0] == 0 and s == 0
    assert (got["tq"] == Tq).all()
    assert (got["sat_s1"] == oracle.sat(ref.S1)).all()
    assert (got["sat_s2"] == oracle.sat(ref.S2)).all()
    assert (got["sat_t"] == oracle.sat(Tq.astype(np.uint64))).all()
    _check_every_band(oracle, got, ref, Tq)


@pytest.mark.parametrize("W,H,pattern", [(8192, 4096, "max"), (8191, 4095, "checker"), (4000, 2200, "coin"),
                                          (129, 131, "checker"), (1, 1, "max")])
def test_tables_extreme_sums_bit_exact(dec, oracle, W, H, pattern):
    """12-bit planes at the sum extremes: S1 up to 4095 * 2^25 and the
    largest slice SSE, on clipped edges too; every Q of every tile column is
    the exact S2 - ceil(S1^2 / N)."""
    rng = np.random.default_rng(W + H)
    if pattern == "max":
        plane = np.full((H, W), 4095, np.uint16)
    elif pattern == "checker":
        plane = ((np.add.outer(np.arange(H), np.arange(W)) & 1) * 4095).astype(np.uint16)
    else:
        plane = (rng.integers(0, 2, (H, W)) * 4095).astype(np.uint16)
    R, C = -(-H // 128), -(-W // 128)
    times = rng.uniform(0.0, 3.0, (R, C)).astype(np.float32)
    _, st, _keep = _texture(dec, plane, 12)
    tab = dec.tables_buffer(W, H)
    dec.region_tables(st, torch.from_numpy(times).cuda(), W, H, tab)
    torch.cuda.synchronize()
    got = dec.read_tables(tab, W, H)
    ref = oracle.texture(plane, 12)
    Tq, _ = oracle.time_q(times)
    _check_every_band(oracle, got, ref, Tq)


@pytest.mark.parametrize("bad", [np.nan, -0.5, 65536.0, np.inf])
def test_tables_bad_time_sets_erange(dec, bad):
    plane, times = synth.small_frame(512, 256, 8, 9)
    times[1, 2] = bad
    _, st, _keep = _texture(dec, plane, 8)
    tab = dec.tables_buffer(512, 256)
    dec.region_tables(st, torch.from_numpy(times).cuda(), 512, 256, tab)
    out = dec.search(tab, 512, 256, 2, 0.0)
    p = dec.partitions(out)[0]
    assert dec.read_tables(tab, 512, 256)["status"][0] == 2
    assert p.status == 2


def _decide(dec, plane, times, bd, n, lam):
    H, W = plane.shape
    luma, ptr, pitch = _dev(plane)
    out = dec.decide(luma, pitch, W, H, bd, torch.from_numpy(np.ascontiguousarray(times, np.float32)).cuda(), n, lam)
    return dec.partitions(out)[0]


@pytest.mark.parametrize("case", golden_cases.cases(), ids=lambda c: c["name"])
def test_hand_worked_cases(dec, case):
    lam = case["lambda_q"] / 65536.0
    p = _decide(dec, golden_cases.plane(case), golden_cases.times(case), case["bit_depth"], case["n"], lam)
    e = case["expect"]
    if e.get("infeasible"):
        assert p.status == 3
        return
    assert p.status == 0
    assert (p.t_min_q, p.t_q, p.q) == (e["t_min"], e["t"], e["q"])
    assert p.x_edges() == e["x_edges"]
    assert p.band_cuts() == golden_cases.band_masks(case)


@pytest.mark.parametrize("seed", range(60))
def test_random_frames_match_oracle(dec, oracle, seed):
    rng = np.random.default_rng(500 + seed)
    W = int(rng.integers(1, 1100))
    H = int(rng.integers(1, 900))
    bd = int(rng.choice([8, 10]))
    n = int(rng.integers(1, 13))
    lam = float(rng.choice([0.0, 0.05, 0.1, 0.3, 1.0]))
    plane, times = synth.small_frame(W, H, bd, seed)
    if seed % 5 == 0:
        times[:] = 1.0  # uniform times: ties on T
    if seed % 7 == 0:
        plane[:] = plane.flat[0]  # flat frame: Q ties, the code decides
    p = _decide(dec, plane, times, bd, n, lam)
    d, st, Tq = oracle.decide(plane, times, bd, n, lam)
    R = st.S1.shape[0]
    assert_partition_equal(p, d, R)
    if W * H < 300 * 300 and n <= 5:
        d1 = oracle.search_enum(st, Tq, n, lam)
        assert_partition_equal(p, d1, R)


@pytest.mark.parametrize("lam", [0.0, 0.1, 0.3])
@pytest.mark.parametrize("n", [4, 8, 16])
def test_480p_matches_oracle(dec, oracle, n, lam):
    for seed in range(3):
        plane, times = synth.make_frame(synth.SPEC_480P8, seed)
        p = _decide(dec, plane, times, 8, n, lam)
        d, st, Tq = oracle.decide(plane, times, 8, n, lam)
        assert_partition_equal(p, d, 4)
        if n <= 8:
            assert_partition_equal(p, oracle.search_enum(st, Tq, n, lam), 4)


@pytest.mark.parametrize("n", [4, 8, 12])
def test_1080p_matches_oracle(dec, oracle, n):
    for seed in range(3):
        plane, times = synth.make_frame(synth.SPEC_1080P10, seed)
        p = _decide(dec, plane, times, 10, n, 0.1)
        d, _, _ = oracle.decide(plane, times, 10, n, 0.1)
        assert_partition_equal(p, d, 9)


def test_2160p_sequence_matches_oracle(dec, oracle):
    """Every 8th frame of the moving-blob UHD sequence, n = 16 and 8."""
    for f, (plane, times) in enumerate(synth.sequence_2160p_blob(64)):
        if f % 8:
            continue
        for n in (16, 8):
            p = _decide(dec, plane, times, 10, n, 0.1)
            d, st, Tq = oracle.decide(plane, times, 10, n, 0.1)
            assert_partition_equal(p, d, 17)
            assert_valid_partition(oracle, p, st, Tq, n)


def test_bench_launch_matches_oracle_on_all_64_frames(dec, oracle):
    """The benchmark's launch: the 64-frame UHD sequence in one captured batch
    (2 pipelined chunks, default launch shapes), replayed, every frame equal
    to the oracle."""
    from paper_2012_14792_gb300 import trs
    frames = list(synth.sequence_2160p_blob(64))
    ins, keep = [], []
    for plane, times in frames:
        luma, ptr, pitch = _dev(plane)
        tt = torch.from_numpy(times).cuda()
        keep += [luma, tt]
        ins.append((ptr, pitch, 3840, 2160, 10, tt, 16, 0.1))
    trs.trs_set_tune(dec.ctx, 2, 2, 4)
    try:
        dec.batch_decide(ins)  # capture
        ps = dec.partitions(dec.batch_decide(ins), 64)  # replay
        assert trs.trs_batch_kernels(dec.ctx) == 18  # 9 kernels per chunk
    finally:
        trs.trs_set_tune(dec.ctx, 4, 4, 8)
    for (plane, times), p in zip(frames, ps):
        d, _, _ = oracle.decide(plane, times, 10, 16, 0.1)
        assert_partition_equal(p, d, 17)


def test_single_slice_and_infeasible(dec, oracle):
    plane, times = synth.small_frame(700, 300, 10, 3)
    p = _decide(dec, plane, times, 10, 1, 0.0)
    d, _, _ = oracle.decide(plane, times, 10, 1, 0.0)
    assert_partition_equal(p, d, 3)
    plane, times = synth.small_frame(256, 128, 8, 3)
    assert _decide(dec, plane, times, 8, 3, 0.0).status == 3


def test_largest_frame_and_n(dec, oracle):
    plane, times = synth.small_frame(8192, 4096, 10, 11)
    p = _decide(dec, plane, times, 10, 32, 0.1)
    d, st, Tq = oracle.decide(plane, times, 10, 32, 0.1)
    assert_partition_equal(p, d, 32)


def test_decide_host_matches_device(dec, oracle):
    plane, times = synth.make_frame(synth.SPEC_1080P10, 5)
    p = dec.decide_host(plane, times, 10, 8, 0.1)
    d, _, _ = oracle.decide(plane, times, 10, 8, 0.1)
    assert_partition_equal(p, d, 9)


def test_invalid_arguments(dec):
    from paper_2012_14792_gb300 import trs
    plane, times = synth.small_frame(256, 256, 8, 1)
    luma, ptr, pitch = _dev(plane)
    tt = torch.from_numpy(times).cuda()
    out = torch.zeros(trs.PARTITION_BYTES, dtype=torch.uint8, device="cuda")
    for args in [(ptr, 256, 256, pitch, 7, tt, 2, 0.0), (ptr, 256, 256, pitch, 8, tt, 0, 0.0),
                 (ptr, 256, 256, pitch, 8, tt, 33, 0.0), (ptr, 256, 256, pitch, 8, tt, 2, -1.0),
                 (ptr, 256, 256, 100, 8, tt, 2, 0.0), (ptr, 9000, 256, 9000, 8, tt, 2, 0.0),
                 (0, 256, 256, pitch, 8, tt, 2, 0.0), (ptr, 256, 256, pitch, 8, tt, 2, float("nan"))]:
        with pytest.raises(trs.TrsError) as e:
            trs.trs_decide(dec.ctx, args[0], args[1], args[2], args[3], args[4], args[5], args[6], args[7], out)
        assert e.value.status == trs.EINVAL


def _batch_inputs(items):
    ins, keep = [], []
    for it in items:
        H, W = it.plane.shape
        luma, ptr, pitch = _dev(it.plane)
        tt = torch.from_numpy(it.times).cuda()
        keep += [luma, tt]
        ins.append((ptr, pitch, W, H, it.spec.bit_depth, tt, it.n_regions, it.lam))
    return ins, keep


def test_batch_matches_plain_and_oracle(dec, oracle):
    items = synth.mixed_batch(256, seed=4)[:40]
    ins, keep = _batch_inputs(items)
    out = dec.batch_decide(ins)
    ps = dec.partitions(out, len(items))
    for it, p, (ptr, pitch, W, H, bd, tt, n, lam) in zip(items, ps, ins):
        q = dec.partitions(dec.decide(ptr, pitch, W, H, bd, tt, n, lam))[0]
        assert bytes(p) == bytes(q)  # identical alone and in the batch
        d, _, _ = oracle.decide(it.plane, it.times, bd, n, lam)
        assert_partition_equal(p, d, it.spec.ctu_rows)


def test_batch_graph_replay_with_new_frames(dec, oracle):
    # same composition twice: the second call replays the captured graph on new inputs
    a = synth.mixed_batch(256, seed=4)[:12]
    b = synth.mixed_batch(256, seed=4)[:12]
    for it, jt in zip(a, b):
        assert it.spec == jt.spec
    for i, jt in enumerate(b):
        jt.plane, jt.times = synth.make_frame(jt.spec, seed=99, frame=i)
    for items in (a, b, a):
        ins, keep = _batch_inputs(items)
        ps = dec.partitions(dec.batch_decide(ins), len(items))
        for it, p in zip(items, ps):
            d, _, _ = oracle.decide(it.plane, it.times, it.spec.bit_depth, it.n_regions, it.lam)
            assert_partition_equal(p, d, it.spec.ctu_rows)


@pytest.mark.parametrize("nf", [1, 7, 8, 9, 33])
def test_batch_chunks_equal_alone(dec, nf):
    """Captured batches run as pipelined chunks on two streams; every
    partition equals the frame decided alone for every chunking, and the
    stage times cover the first chunk."""
    from paper_2012_14792_gb300 import trs
    items = synth.mixed_batch(256, seed=6)[:nf]
    ins, keep = _batch_inputs(items)
    alone = [bytes(dec.partitions(dec.decide(ptr, pitch, W, H, bd, tt, n, lam))[0])
             for (ptr, pitch, W, H, bd, tt, n, lam) in ins]
    try:
        for parts in (2, 1, 3, 4):
            trs.trs_set_batch_parts(dec.ctx, parts)
            P = max(1, min(parts, nf // 4))
            for _ in range(2):  # capture, then replay
                ps = dec.partitions(dec.batch_decide(ins), nf)
                assert trs.trs_batch_stage_frames(dec.ctx) == nf // P
                assert trs.trs_batch_kernels(dec.ctx) == 9 * P
                assert [bytes(p) for p in ps] == alone, parts
    finally:
        trs.trs_set_batch_parts(dec.ctx, 2)
    for bad in (0, 5):
        with pytest.raises(trs.TrsError):
            trs.trs_set_batch_parts(dec.ctx, bad)


def test_two_contexts_in_flight_on_two_streams(dec):
    """Batches of two contexts running at once on two streams (a stream of
    steps with two in flight) decide the same bytes as one context alone."""
    from paper_2012_14792_gb300 import runtime
    items = synth.mixed_batch(256, seed=8)[:24]
    ins, keep = _batch_inputs(items)
    ref = bytes(dec.batch_decide(ins).cpu().numpy())
    other = runtime.Decider(max_width=3840, max_height=2160, max_regions=32, max_batch=24)
    try:
        ctxs = [dec, other]
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        outs = [torch.zeros(24 * 840, dtype=torch.uint8, device="cuda") for _ in range(2)]
        for step in range(6):
            i = step % 2
            with torch.cuda.stream(streams[i]):
                ctxs[i].batch_decide(ins, outs[i])
        torch.cuda.synchronize()
        assert bytes(outs[0].cpu().numpy()) == ref and bytes(outs[1].cpu().numpy()) == ref
    finally:
        other.close()


def test_batch_replay_after_descriptor_growth(dec):
    """A multi-lambda search that needs a larger descriptor buffer drops the
    captured batches that pointed at the old one; replays stay correct."""
    from paper_2012_14792_gb300 import runtime
    fresh = runtime.Decider(max_width=3840, max_height=2160, max_regions=32, max_batch=4)
    try:
        items = synth.mixed_batch(256, seed=7)[:1]
        ins, keep = _batch_inputs(items)
        ref = bytes(dec.batch_decide(ins).cpu().numpy())
        assert bytes(fresh.batch_decide(ins).cpu().numpy()) == ref
        it = items[0]
        W, H = it.spec.width, it.spec.height
        _, st, _keep = _texture(fresh, it.plane, it.spec.bit_depth)
        tab = fresh.tables_buffer(W, H)
        fresh.region_tables(st, torch.from_numpy(it.times).cuda(), W, H, tab)
        fresh.search_lambdas(tab, W, H, it.n_regions, [0.0, 0.05, 0.1, 0.2, 0.3, 0.5, 1.0, 2.0])
        assert bytes(fresh.batch_decide(ins).cpu().numpy()) == ref
    finally:
        fresh.close()


@pytest.mark.parametrize("scale,flag", [(1.0, 1), (2000.0, 0)])
def test_step1_value_width_paths(dec, oracle, scale, flag):
    """Frames whose total Q16 time is below 2^31 run step 1 on 32-bit values,
    others on 64-bit values; both must give the oracle's partition."""
    for seed in range(3):
        plane, times = synth.make_frame(synth.SPEC_1080P10, 40 + seed)
        times = np.minimum(times * np.float32(scale), np.float32(65535.0)).astype(np.float32)
        _, st, _keep = _texture(dec, plane, 10)
        tab = dec.tables_buffer(1920, 1080)
        dec.region_tables(st, torch.from_numpy(times).cuda(), 1920, 1080, tab)
        p = dec.partitions(dec.search(tab, 1920, 1080, 8, 0.1))[0]
        assert int(dec.read_tables(tab, 1920, 1080)["status"][3]) == flag
        d, _, _ = oracle.decide(plane, times, 10, 8, 0.1)
        assert_partition_equal(p, d, 9)


def test_launch_shapes_do_not_change_decisions(dec, oracle):
    """Every launch shape the autotuner may pick gives the same bytes; the
    autotuner picks one of them and keeps the decisions."""
    from paper_2012_14792_gb300 import trs
    items = synth.mixed_batch(256, seed=4)[:16]
    ins, keep = _batch_inputs(items)
    trs.trs_set_tune(dec.ctx, 4, 4, 8)
    ref = bytes(dec.batch_decide(ins).cpu().numpy())
    for bw in (2, 4, 8):
        for cw in (1, 2, 4, 8):
            for cb in (4, 8):
                trs.trs_set_tune(dec.ctx, bw, cw, cb)
                assert bytes(dec.batch_decide(ins).cpu().numpy()) == ref, (bw, cw, cb)
    rep = dec.autotune(ins)
    assert rep["band_warps"] in (2, 4, 8) and rep["col_warps"] in (1, 2, 4) and rep["col_batch"] in (4, 8)
    assert len(rep["candidates"]) == 6 and all(c["rows_ms"] > 0 and c["cols_ms"] > 0 for c in rep["candidates"])
    assert bytes(dec.batch_decide(ins).cpu().numpy()) == ref
    with pytest.raises(trs.TrsError):
        trs.trs_set_tune(dec.ctx, 3, 4, 8)
    trs.trs_set_tune(dec.ctx, 4, 4, 8)


@pytest.mark.parametrize("spec_name,n,lams", [("SPEC_2160P10", 16, [0.0, 0.1, 0.3]),
                                              ("SPEC_1080P10", 8, [0.3, 0.0, 2.0, 0.05, 0.1]),
                                              ("SPEC_480P8", 4, [0.1])])
def test_search_lambdas_equals_separate_searches(dec, oracle, spec_name, n, lams):
    """Step 1 shared across lambdas: every partition equals its own trs_search."""
    spec = getattr(synth, spec_name)
    plane, times = synth.make_frame(spec, seed=21)
    W, H = spec.width, spec.height
    _, st, _keep = _texture(dec, plane, spec.bit_depth)
    tab = dec.tables_buffer(W, H)
    dec.region_tables(st, torch.from_numpy(times).cuda(), W, H, tab)
    many = dec.partitions(dec.search_lambdas(tab, W, H, n, lams), len(lams))
    for lam, p in zip(lams, many):
        one = dec.partitions(dec.search(tab, W, H, n, lam))[0]
        assert bytes(p) == bytes(one)
        d, _, _ = oracle.decide(plane, times, spec.bit_depth, n, lam)
        assert_partition_equal(p, d, spec.ctu_rows)


@pytest.mark.parametrize("spec_name,n,step", [("SPEC_2160P10", 16, 4), ("SPEC_2160P10", 16, 8),
                                              ("SPEC_1080P10", 8, 2), ("SPEC_480P8", 4, 3)])
def test_windowed_search_matches_oracle(dec, oracle, spec_name, n, step):
    from paper_2012_14792_gb300 import trs
    spec = getattr(synth, spec_name)
    trs.trs_set_window_step(dec.ctx, step)
    try:
        for seed in range(2):
            plane, times = synth.make_frame(spec, seed=60 + seed)
            p = _decide(dec, plane, times, spec.bit_depth, n, 0.1)
            st = oracle.texture(plane, spec.bit_depth)
            Tq, _ = oracle.time_q(times)
            d = oracle.search_dp_windows(st, Tq, n, 0.1, window_step=step)
            assert p.n_windows == d.n_windows
            assert_partition_equal(p, d, spec.ctu_rows)
    finally:
        trs.trs_set_window_step(dec.ctx, 1)


@pytest.mark.parametrize("W,H,n,k", [(1, 511, 2, 3), (1, 512, 2, 3), (129, 511, 3, 3), (1, 255, 1, 2),
                                     (255, 1, 1, 2)])
def test_area_rule_edge_frames(oracle, W, H, n, k):
    """Frames where a slice area can equal k*A_min - 1, the largest the rule
    admits (Sec. 2.3): with a slow top CTU row the 1x511 frame's best split is
    128 over 383 = 3*128 - 1 rows of pixels, and 1x512's is 256 over 256; at
    k = 2 the 1x255 frame's one slice of 255 = 2*128 - 1 samples lies in the
    window of area 128.  The GPU partition equals the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2012_14792_gb300 import runtime
    d = runtime.Decider(max_width=512, max_height=512, max_regions=4, max_batch=1, k_area=k)
    try:
        rng = np.random.default_rng(W + H + k)
        plane = rng.integers(0, 1024, size=(H, W)).astype(np.uint16)
        C, R = oracle.grid(W, H)
        times = np.ones((R, C), np.float32)
        times[0, :] = 10.0
        p = _decide(d, plane, times, 10, n, 0.0)
        ref, _, _ = oracle.decide(plane, times, 10, n, 0.0, k_area=k)
        assert ref.status == oracle.OK
        assert_partition_equal(p, ref, R)
    finally:
        d.close()
