"""The CUDA path against O1, the oracle's plain enumeration of S(n) in code
order (Sec. 2.3: Eq. 3, then Eq. 2 under Eq. 4, the k*A_min > A_max rule),
with no structured search in between: 3840x2160 frames (30x17 CTUs, the
112-pixel last row), narrow 2160-pixel-high frames, and 1920x1080 up to
n = 12.  Both the one-frame path and a batched launch of frames that share
one plan (the form the benchmark times) are compared."""

import numpy as np
import pytest

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
    d = runtime.Decider(max_width=3840, max_height=2160, max_regions=16, max_batch=16)
    yield d
    d.close()


def _dev(plane):
    from paper_2012_14792_gb300 import runtime
    return runtime.luma_to_device(plane)


def _decide(dec, plane, times, bd, n, lam):
    H, W = plane.shape
    luma, pitch = _dev(plane)
    out = dec.decide(luma, pitch, W, H, bd, torch.from_numpy(np.ascontiguousarray(times, np.float32)).cuda(), n, lam)
    return dec.partitions(out)[0]


def _o1(oracle, plane, times, bd, n, lam):
    st = oracle.texture(plane, bd)
    Tq, s = oracle.time_q(times)
    assert st.status == oracle.OK and s == oracle.OK
    return oracle.search_enum(st, Tq, n, lam), st, Tq


@pytest.mark.parametrize("n,lams", [(4, (0.0, 0.1, 0.3)), (5, (0.1,)), (6, (0.1,)), (8, (0.1,))])
def test_2160p_equals_o1(dec, oracle, n, lams):
    plane, times = synth.make_frame(synth.SPEC_2160P10, 0)
    for lam in lams:
        p = _decide(dec, plane, times, 10, n, lam)
        d, st, Tq = _o1(oracle, plane, times, 10, n, lam)
        assert d.status == oracle.OK
        assert_partition_equal(p, d, 17)
        assert_valid_partition(oracle, p, st, Tq, n)


@pytest.mark.parametrize("W,n", [(640, 2), (640, 3), (640, 4), (640, 5), (640, 6), (640, 8), (1280, 6)])
def test_2160_rows_equals_o1(dec, oracle, W, n):
    for seed in (7, 8):
        plane, times = synth.small_frame(W, 2160, 10, seed)
        for lam in (0.0, 0.1, 0.3):
            p = _decide(dec, plane, times, 10, n, lam)
            d, _, _ = _o1(oracle, plane, times, 10, n, lam)
            assert_partition_equal(p, d, 17)


@pytest.mark.parametrize("W,n", [(384, 3), (384, 5), (640, 6)])
def test_2160_rows_flat_uniform_times_tie_order_equals_o1(dec, oracle, W, n):
    """A flat plane with equal CTU times: every partition has Q = 0 and many
    share T_min, so only the smallest canonical code decides."""
    plane = np.full((2160, W), 512, np.uint16)
    C, R = -(-W // 128), 17
    times = np.ones((R, C), np.float32)
    for lam in (0.0, 0.3):
        p = _decide(dec, plane, times, 10, n, lam)
        d, _, _ = _o1(oracle, plane, times, 10, n, lam)
        assert d.status == oracle.OK and d.q == 0
        assert_partition_equal(p, d, R)


@pytest.mark.parametrize("n,lams", [(8, (0.0, 0.1, 0.3)), (12, (0.1,))])
def test_1080p_equals_o1(dec, oracle, n, lams):
    for seed in ((0, 1) if n == 8 else (0,)):
        plane, times = synth.make_frame(synth.SPEC_1080P10, seed)
        for lam in lams:
            p = _decide(dec, plane, times, 10, n, lam)
            d, _, _ = _o1(oracle, plane, times, 10, n, lam)
            assert_partition_equal(p, d, 9)


def test_batched_2160p_sequence_equals_o1(dec, oracle):
    """Sixteen frames of the moving-blob 3840x2160 sequence in one captured
    batch (one plan shared by every frame), replayed, n = 4: each frame's
    partition equals O1's."""
    frames = [synth.sequence_2160p_frame(f) for f in range(0, 64, 4)]
    ins, keep = [], []
    for plane, times in frames:
        luma, pitch = _dev(plane)
        tt = torch.from_numpy(np.ascontiguousarray(times)).cuda()
        keep += [luma, tt]
        ins.append((luma.data_ptr(), pitch, 3840, 2160, 10, tt, 4, 0.1))
    dec.batch_decide(ins)  # capture
    ps = dec.partitions(dec.batch_decide(ins), len(ins))  # replay
    for (plane, times), p in zip(frames, ps):
        d, _, _ = _o1(oracle, plane, times, 10, 4, 0.1)
        assert_partition_equal(p, d, 17)
