"""Continuous-batching server: every decision taken in the mix of concurrent
streams equals the same frame decided alone (bit for bit) and the oracle's
decision for that frame and its co-located time map (Sec. 2.1), admission
is bounded by memory, waits are bounded, and time-map updates take effect."""

import time

import numpy as np
import pytest

import synth
from gpu_helpers import assert_partition_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_14792_gb300 import runtime, trs
    return trs, runtime


def _alone(dec, plane, times, bd, n, lam):
    from paper_2012_14792_gb300 import runtime
    H, W = plane.shape
    luma, pitch = runtime.luma_to_device(plane)
    out = dec.decide(luma, pitch, W, H, bd, torch.from_numpy(times).cuda(), n, lam)
    return dec.partitions(out)[0]


def test_mix_equals_alone(lib, oracle):
    trs, runtime = lib
    srv = trs.trs_server_create(3840, 2160, max_regions=16, max_streams=8, max_batch=8, max_inflight=2)
    dec = runtime.Decider(max_width=3840, max_height=2160, max_regions=16)
    try:
        specs = [(synth.SPEC_1080P10, 8), (synth.SPEC_2160P10, 16)] * 3
        streams, frames = [], {}
        for i, (spec, n) in enumerate(specs):
            sid = trs.trs_server_open_stream(srv, spec.width, spec.height, spec.bit_depth, n, 0.1)
            _, times = synth.make_frame(spec, seed=100 + i, stream=i, workload="serve")
            trs.trs_server_update_times(srv, sid, np.ascontiguousarray(times))
            streams.append((sid, spec, n, times))
        # three frames per stream, interleaved across streams
        queue = []
        for f in range(3):
            for (sid, spec, n, times) in streams:
                plane, _ = synth.make_frame(spec, seed=200 + f, stream=sid, frame=f, workload="serve")
                frames[(sid, f)] = np.ascontiguousarray(plane)
                queue.append((sid, f))
        got = {}
        pending = list(queue)
        deadline = time.time() + 120
        while (pending or len(got) < len(queue)) and time.time() < deadline:
            still = []
            for (sid, f) in pending:
                p = frames[(sid, f)]
                try:
                    trs.trs_server_submit(srv, sid, p, p.strides[0], tag=f)
                except trs.TrsError as e:
                    assert e.status == trs.EBUSY  # both slots of the stream in use: retry later
                    still.append((sid, f))
            pending = still
            for d in trs.trs_server_poll(srv, 64, 2000):
                got[(d.stream_id, int(d.tag))] = d
        assert len(got) == len(queue)
        info = trs.trs_server_info(srv)
        assert info.decided == len(queue) and info.status == 0
        for (sid, spec, n, times) in streams:
            for f in range(3):
                d = got[(sid, f)]
                assert d.status == 0 and d.latency_us > 0
                ref = _alone(dec, frames[(sid, f)], times, spec.bit_depth, n, 0.1)
                assert bytes(d.partition) == bytes(ref)
                want, _, _ = oracle.decide(frames[(sid, f)], times, spec.bit_depth, n, 0.1)
                assert_partition_equal(d.partition, want, spec.ctu_rows)
    finally:
        trs.trs_server_destroy(srv)
        dec.close()


def test_admission_by_memory(lib):
    trs, _ = lib
    budget = 200 << 20
    srv = trs.trs_server_create(3840, 2160, max_regions=16, max_streams=32, max_batch=4, max_inflight=1,
                                mem_budget_bytes=budget)
    try:
        sids = []
        with pytest.raises(trs.TrsError) as e:
            for _ in range(32):
                sids.append(trs.trs_server_open_stream(srv, 3840, 2160, 10, 16, 0.1))
        assert e.value.status == trs.EBUSY
        assert 1 <= len(sids) < 32
        info = trs.trs_server_info(srv)
        assert info.streams_open == len(sids)
        trs.trs_server_close_stream(srv, sids[0])
        sids[0] = trs.trs_server_open_stream(srv, 3840, 2160, 10, 16, 0.1)  # the freed memory admits one again
        with pytest.raises(trs.TrsError):
            trs.trs_server_open_stream(srv, 3840, 2160, 10, 16, 0.1)
    finally:
        trs.trs_server_destroy(srv)


def test_bounded_waits_and_argument_errors(lib):
    trs, _ = lib
    srv = trs.trs_server_create(1920, 1080, max_regions=8, max_streams=2, max_batch=2, max_inflight=1)
    try:
        t0 = time.time()
        assert trs.trs_server_poll(srv, 4, 50_000) == []  # nothing submitted: a bounded, empty wait
        assert time.time() - t0 < 5
        sid = trs.trs_server_open_stream(srv, 1920, 1080, 10, 8, 0.1)
        plane, times = synth.make_frame(synth.SPEC_1080P10, 3)
        with pytest.raises(trs.TrsError) as e:
            trs.trs_server_submit(srv, sid, np.ascontiguousarray(plane), plane.strides[0])  # no time map yet
        assert e.value.status == trs.EINVAL
        with pytest.raises(trs.TrsError) as e:
            trs.trs_server_open_stream(srv, 3840, 2160, 10, 8, 0.1)  # beyond the server's frame size
        assert e.value.status == trs.EINVAL
        with pytest.raises(trs.TrsError):
            trs.trs_server_submit(srv, 5, np.ascontiguousarray(plane), plane.strides[0])  # no such stream
    finally:
        trs.trs_server_destroy(srv)


def test_time_map_update_takes_effect(lib, oracle):
    trs, runtime = lib
    srv = trs.trs_server_create(1920, 1080, max_regions=8, max_streams=1, max_batch=2, max_inflight=2)
    dec = runtime.Decider(max_width=1920, max_height=1080, max_regions=8)
    try:
        sid = trs.trs_server_open_stream(srv, 1920, 1080, 10, 8, 0.0)
        plane, t0 = synth.make_frame(synth.SPEC_1080P10, 5)
        plane = np.ascontiguousarray(plane)
        t1 = np.ascontiguousarray(t0[:, ::-1])  # a different co-located time map
        for times in (t0, t1):
            trs.trs_server_update_times(srv, sid, np.ascontiguousarray(times))
            trs.trs_server_submit(srv, sid, plane, plane.strides[0])
            ds = []
            deadline = time.time() + 30
            while not ds and time.time() < deadline:
                ds = trs.trs_server_poll(srv, 4, 10_000)
            assert len(ds) == 1 and ds[0].status == 0
            assert bytes(ds[0].partition) == bytes(_alone(dec, plane, np.ascontiguousarray(times), 10, 8, 0.0))
            want, _, _ = oracle.decide(plane, np.ascontiguousarray(times), 10, 8, 0.0)
            assert_partition_equal(ds[0].partition, want, 9)
    finally:
        trs.trs_server_destroy(srv)
        dec.close()


def test_temporal_layer_maps_follow_the_co_tl_frame(lib, oracle):
    """One random-access GOP of 16 in coding order: each frame is decided
    with the CTU times of the previous frame of its temporal layer (the co-TL
    frame of Sec. 2.1), or the most recent map before its layer has one."""
    trs, runtime = lib
    srv = trs.trs_server_create(1920, 1080, max_regions=8, max_streams=1, max_batch=4, max_inflight=2)
    dec = runtime.Decider(max_width=1920, max_height=1080, max_regions=8)
    try:
        sid = trs.trs_server_open_stream_layers(srv, 1920, 1080, 10, 8, 0.1, 5)
        spec = synth.SPEC_1080P10
        _, init = synth.make_frame(spec, seed=30, frame=999, workload="serve")
        trs.trs_server_update_times_layer(srv, sid, 0, np.ascontiguousarray(init))
        layer_map, last = {0: init}, init
        for poc in synth.ra_coding_order(16):
            L = synth.ra_temporal_layer(poc)
            plane, encoded_times = synth.make_frame(spec, seed=31, frame=poc, workload="serve")
            plane = np.ascontiguousarray(plane)
            expect = layer_map.get(L, last)
            trs.trs_server_submit_layer(srv, sid, L, plane, plane.strides[0], tag=poc)
            ds = []
            deadline = time.time() + 30
            while not ds and time.time() < deadline:
                ds = trs.trs_server_poll(srv, 4, 10_000)
            assert len(ds) == 1 and ds[0].status == 0 and ds[0].tag == poc
            assert bytes(ds[0].partition) == bytes(_alone(dec, plane, np.ascontiguousarray(expect), 10, 8, 0.1))
            # the oracle, given the co-TL frame's CTU times, takes the same decision
            want, _, _ = oracle.decide(plane, np.ascontiguousarray(expect), 10, 8, 0.1)
            assert_partition_equal(ds[0].partition, want, 9)
            # the frame is encoded: its CTU times become its layer's co-TL map
            trs.trs_server_update_times_layer(srv, sid, L, np.ascontiguousarray(encoded_times))
            layer_map[L] = encoded_times
            last = encoded_times
        with pytest.raises(trs.TrsError):
            trs.trs_server_submit_layer(srv, sid, 5, plane, plane.strides[0])
    finally:
        trs.trs_server_destroy(srv)
        dec.close()
