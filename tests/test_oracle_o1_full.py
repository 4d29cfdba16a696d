"""O2 (the exact DP over area windows and tile columns) equals O1 (every
configuration of S(n) enumerated in code order, Sec. 2.3) at the paper's
frame sizes: 832x480 (7x4 CTUs), 1920x1080 (15x9, a clipped 56-pixel last
row) and 3840x2160 (30x17, a clipped 112-pixel last row), for the thread
counts of Table 1 that O1 can enumerate.

The 17-row frames are the geometry of every 3840x2160 decision: the 112-pixel
bottom row, 16 full rows above it and slice heights up to 17 CTU rows.  Narrow
2160-pixel-high frames (640x2160: 5x17 CTUs) reach larger n at small cost.

These cases take O1 over up to 8.9e6 valid configurations (3840x2160, n = 8:
about 17 s on one core), so they sit in their own file, outside the pin set
the mutation test reruns for every planted slip.
"""

import numpy as np
import pytest

import synth


def _frame(oracle, plane, times, bd):
    st = oracle.texture(plane, bd)
    Tq, s = oracle.time_q(times)
    assert st.status == oracle.OK and s == oracle.OK
    return st, Tq


def _same(oracle, st, Tq, n, lam):
    a = oracle.search_enum(st, Tq, n, lam)
    b = oracle.search_dp(st, Tq, n, lam)
    assert a.status == b.status
    if a.status != oracle.OK:
        return a
    assert a.row_mask == 0  # a tile-row cut never gives the smallest code
    assert (a.t_min, a.thr, a.t, a.q) == (b.t_min, b.thr, b.t, b.q)
    assert (a.x_edges, a.band_cuts) == (b.x_edges, b.band_cuts)
    assert abs(a.sse_real - b.sse_real) <= 1e-9 * max(1.0, abs(a.sse_real))
    ev = oracle.evaluate(st, Tq, a.x_edges, a.band_cuts)
    assert ev["n"] == n and ev["t"] == a.t and ev["q"] == a.q and 3 * ev["amin"] > ev["amax"]
    assert a.t * 65536 <= a.t_min * (65536 + oracle.lambda_q(lam))
    return a


@pytest.mark.parametrize("spec_name,n,lams", [
    ("SPEC_1080P10", 8, (0.0, 0.1, 0.3)),
    ("SPEC_1080P10", 12, (0.1,)),
    ("SPEC_2160P10", 4, (0.0, 0.1, 0.3)),
    ("SPEC_2160P10", 8, (0.1,)),
])
def test_o2_equals_o1_table1_sizes(oracle, spec_name, n, lams):
    spec = getattr(synth, spec_name)
    plane, times = synth.make_frame(spec, 0)
    st, Tq = _frame(oracle, plane, times, spec.bit_depth)
    for lam in lams:
        d = _same(oracle, st, Tq, n, lam)
        assert d.status == oracle.OK
        assert d.n_valid > 0


def test_o2_equals_o1_moving_blob_frames(oracle):
    # frames of the 64-frame 3840x2160 sequence (blob at different places), n = 4
    for f in (0, 21, 63):
        plane, times = synth.sequence_2160p_frame(f)
        st, Tq = _frame(oracle, plane, times, 10)
        for lam in (0.0, 0.1):
            assert _same(oracle, st, Tq, 4, lam).status == oracle.OK


@pytest.mark.parametrize("W,n", [(640, 2), (640, 3), (640, 4), (640, 5), (640, 6), (640, 8),
                                 (1280, 6), (3840, 5), (3840, 6)])
def test_o2_equals_o1_2160_rows(oracle, W, n):
    plane, times = synth.small_frame(W, 2160, 10, seed=7)
    st, Tq = _frame(oracle, plane, times, 10)
    for lam in ((0.0, 0.1, 0.3) if W < 3840 else (0.1,)):
        assert _same(oracle, st, Tq, n, lam).status == oracle.OK


def _pixel_counts(W, H):
    C, R = -(-W // 128), -(-H // 128)
    cw = [min(128 * (x + 1), W) - 128 * x for x in range(C)]
    ch = [min(128 * (y + 1), H) - 128 * y for y in range(R)]
    return np.array([[w * h for w in cw] for h in ch], np.uint64)


@pytest.mark.parametrize("seed", range(24))
def test_o2_equals_o1_17_rows_random_stats(oracle, seed):
    """Random statistics on 1-3 CTU columns x 17 rows, the last row clipped to
    112 pixels: flat frames and uniform times make ties everywhere, so the
    tie order of both searches is compared too."""
    rng = np.random.default_rng(17000 + seed)
    C = int(rng.integers(1, 4))
    W = (C - 1) * 128 + int(rng.integers(1, 129))
    H = 2160
    N = _pixel_counts(W, H)
    R = N.shape[0]
    mode = ("random", "flat", "uniform")[seed % 3]
    if mode == "random":
        mu = rng.integers(0, 1024, size=(R, C)).astype(np.uint64)
        S1, S2 = mu * N, mu * mu * N + rng.integers(0, 10 ** 6, size=(R, C)).astype(np.uint64)
        Tq = rng.integers(0, 3 * 65536, size=(R, C)).astype(np.uint32)
    elif mode == "flat":
        S1, S2 = 9 * N, 81 * N
        Tq = (rng.integers(0, 3, size=(R, C)) * 65536).astype(np.uint32)
    else:
        mu = rng.integers(0, 3, size=(R, C)).astype(np.uint64)
        S1, S2 = mu * N, mu * mu * N + rng.integers(0, 40, size=(R, C)).astype(np.uint64)
        Tq = np.full((R, C), 65536, np.uint32)
    from oracle import oracle as O
    st = O.Stats(W, H, S1, S2, N, np.zeros((R, C), np.uint32), 0)
    n = int(rng.integers(2, 9))
    lam = float(rng.choice([0.0, 0.1, 0.3, 1.0]))
    _same(oracle, st, Tq, n, lam)
