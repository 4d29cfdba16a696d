"""The packed 10-bit sample format (TRS_PACKED10: four samples in five
bytes, each row a little-endian bit string) through the CUDA path: per-CTU
statistics bit-exact against the oracle reading the same bytes, and
decisions equal to those taken on the same samples in the two-byte form."""

import numpy as np
import pytest

import synth
from gpu_helpers import assert_partition_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dec():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_14792_gb300 import runtime
    d = runtime.Decider(max_width=8192, max_height=4096, max_regions=16, max_batch=8)
    yield d
    d.close()


def _dev_bytes(rows, pitch=None, offset=0):
    """Device copy of uint8 rows with an optional pitch and byte offset."""
    H, rb = rows.shape
    pitch = rb if pitch is None else pitch
    buf = np.zeros(offset + pitch * H + 64, np.uint8)
    for y in range(H):
        buf[offset + y * pitch: offset + y * pitch + rb] = rows[y]
    t = torch.from_numpy(buf).cuda()
    return t, t.data_ptr() + offset, pitch


@pytest.mark.parametrize("W,H,pad,offset", [
    (3840, 2160, None, 0), (1920, 1080, None, 0), (832, 480, None, 0), (8192, 4096, None, 0),
    (129, 257, 176, 0), (300, 200, None, 0), (300, 200, 400, 3), (1, 1, None, 0), (1280, 720, 1616, 0),
])
def test_packed_texture_bit_exact(dec, oracle, W, H, pad, offset):
    from paper_2012_14792_gb300 import trs
    rng = np.random.default_rng(W + 7 * H)
    plane = rng.integers(0, 1024, size=(H, W)).astype(np.uint16)
    packed = synth.pack10(plane)
    t, ptr, pitch = _dev_bytes(packed, pad, offset)
    st = dec.stats_buffers(W, H)
    dec.texture_map(ptr, W, H, pitch, trs.PACKED10, st)
    torch.cuda.synchronize()
    u32 = lambda x: x.cpu().numpy().view(np.uint32)
    ref = oracle.texture(packed, oracle.PACKED10, width=W)
    assert ref.status == oracle.OK
    assert (u32(st["s1"]) == ref.S1.ravel()).all()
    assert (st["s2"].cpu().numpy().view(np.uint64) == ref.S2.ravel()).all()
    assert (u32(st["count"]) == ref.N.ravel()).all()
    assert (u32(st["vmax"]) == ref.vmax.ravel()).all()
    assert int(u32(st["flags"])[0]) == 0


@pytest.mark.parametrize("spec_name,n", [("SPEC_2160P10", 16), ("SPEC_1080P10", 8)])
def test_packed_decisions_equal_two_byte_decisions(dec, oracle, spec_name, n):
    from paper_2012_14792_gb300 import runtime, trs
    spec = getattr(synth, spec_name)
    W, H = spec.width, spec.height
    plane, times = synth.make_frame(spec, seed=51)
    packed = synth.pack10(plane)
    tt = torch.from_numpy(times).cuda()
    luma, pitch = runtime.luma_to_device(plane)
    ref = dec.partitions(dec.decide(luma, pitch, W, H, 10, tt, n, 0.1))[0]
    pl, pptr, ppitch = _dev_bytes(packed)
    got = dec.partitions(dec.decide(pptr, ppitch, W, H, trs.PACKED10, tt, n, 0.1))[0]
    assert bytes(got) == bytes(ref)
    d, _, _ = oracle.decide(packed, times, oracle.PACKED10, n, 0.1, width=W)
    assert_partition_equal(got, d, spec.ctu_rows)
    # from host memory
    got_h = dec.decide_host(packed, times, trs.PACKED10, n, 0.1, width=W)
    assert bytes(got_h) == bytes(ref)


def test_packed_frames_in_a_batch(dec, oracle):
    """Packed and two-byte frames of several shapes in one batched call."""
    from paper_2012_14792_gb300 import runtime, trs
    items = synth.mixed_batch(256, seed=12)[:8]
    ins, keep, refs = [], [], []
    for i, it in enumerate(items):
        W, H = it.spec.width, it.spec.height
        tt = torch.from_numpy(it.times).cuda()
        if it.spec.bit_depth == 10 and i % 2 == 0:
            rows, p_ptr, pitch = _dev_bytes(synth.pack10(it.plane))
            keep += [rows, tt]
            ins.append((p_ptr, pitch, W, H, trs.PACKED10, tt, it.n_regions, it.lam))
        else:
            luma, pitch = runtime.luma_to_device(it.plane)
            keep += [luma, tt]
            ins.append((luma.data_ptr(), pitch, W, H, it.spec.bit_depth, tt, it.n_regions, it.lam))
        d, _, _ = oracle.decide(it.plane, it.times, it.spec.bit_depth, it.n_regions, it.lam)
        refs.append((d, it.spec.ctu_rows))
    assert any(x[4] == trs.PACKED10 for x in ins)
    for _ in range(2):  # capture, then replay
        ps = dec.partitions(dec.batch_decide(ins), len(ins))
        for p, (d, R) in zip(ps, refs):
            assert_partition_equal(p, d, R)


def test_packed_pitch_too_small(dec):
    from paper_2012_14792_gb300 import trs
    rows = np.zeros((4, 10), np.uint8)
    t, ptr, _ = _dev_bytes(rows)
    st = dec.stats_buffers(8, 4)
    with pytest.raises(trs.TrsError) as e:
        dec.texture_map(ptr, 9, 4, 10, trs.PACKED10, st)  # 9 samples need ceil(90 / 8) = 12 bytes
    assert e.value.status == trs.EINVAL
