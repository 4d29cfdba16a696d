"""Pins of the oracle's Q16 time quantisation (the estimator values of Sec. 2.1
entering Eq. 1) and of its summed-area tables."""

import numpy as np
import pytest


def test_time_q_exact_and_half_even(oracle):
    t = np.array([0.0, 1.0, 3 / 65536, 0.5 / 65536, 1.5 / 65536, 2.5 / 65536, 65535.5], np.float32)
    q, st = oracle.time_q(t)
    assert st == oracle.OK
    assert q.tolist() == [0, 65536, 3, 0, 2, 2, 65535 * 65536 + 32768]


@pytest.mark.parametrize("bad", [np.nan, -1.0, 65536.0, np.inf, -np.inf, -1e-30])
def test_time_q_rejects_out_of_domain(oracle, bad):
    q, st = oracle.time_q(np.array([1.0, bad], np.float32))
    assert st == oracle.ERANGE


def test_negative_zero_is_zero(oracle):
    q, st = oracle.time_q(np.array([-0.0], np.float32))
    assert st == oracle.OK and q[0] == 0


def test_lambda_q(oracle):
    assert oracle.lambda_q(0.0) == 0
    assert oracle.lambda_q(0.1) == 6554      # float32(0.1) * 65536 = 6553.6000...
    assert oracle.lambda_q(0.3) == 19661     # 19660.8000...
    assert oracle.lambda_q(0.5 / 65536) == 0  # half to even
    assert oracle.lambda_q(1.5 / 65536) == 2


@pytest.mark.parametrize("R,C", [(1, 1), (4, 7), (9, 15), (3, 1)])
def test_sat_matches_cumsum_and_rect_sums(oracle, R, C):
    rng = np.random.default_rng(R * 100 + C)
    v = rng.integers(0, 2 ** 40, size=(R, C)).astype(np.uint64)
    s = oracle.sat(v)
    ref = np.zeros((R + 1, C + 1), np.uint64)
    ref[1:, 1:] = np.cumsum(np.cumsum(v, axis=0), axis=1)
    assert (s == ref).all()
    for y0 in range(R):
        for y1 in range(y0 + 1, R + 1):
            for x0 in range(C):
                for x1 in range(x0 + 1, C + 1):
                    rect = int(s[y1, x1]) - int(s[y0, x1]) - int(s[y1, x0]) + int(s[y0, x0])
                    assert rect == int(v[y0:y1, x0:x1].sum())


@pytest.mark.parametrize("W,H", [(300, 520), (128, 128), (1, 700)])
def test_rect_all_matches_written_out_sums(oracle, W, H):
    """Every CTU rectangle's time (Eq. 1) and floor SSE (Eq. 2), against sums
    and an integer ceiling written out here; the unused entries are zero."""
    rng = np.random.default_rng(W + 7 * H)
    C, R = -(-W // 128), -(-H // 128)
    cw = [min(128 * (x + 1), W) - 128 * x for x in range(C)]
    ch = [min(128 * (y + 1), H) - 128 * y for y in range(R)]
    N = np.array([[w * h for w in cw] for h in ch], np.uint64)
    mu = rng.integers(0, 1024, size=(R, C)).astype(np.uint64)
    S1 = mu * N + rng.integers(0, 100, size=(R, C)).astype(np.uint64)
    S2 = mu * mu * N + rng.integers(10 ** 5, 10 ** 7, size=(R, C)).astype(np.uint64)
    Tq = rng.integers(0, 5 * 65536, size=(R, C)).astype(np.uint32)
    st = oracle.Stats(W, H, S1, S2, N, np.zeros((R, C), np.uint32), 0)
    t, q = oracle.rect_all(st, Tq)
    for x0 in range(C + 1):
        for x1 in range(C + 1):
            for y0 in range(R + 1):
                for y1 in range(R + 1):
                    if x0 >= x1 or y0 >= y1:
                        assert t[x0, x1, y0, y1] == 0 and q[x0, x1, y0, y1] == 0
                        continue
                    s1 = sum(int(S1[y, x]) for y in range(y0, y1) for x in range(x0, x1))
                    s2 = sum(int(S2[y, x]) for y in range(y0, y1) for x in range(x0, x1))
                    nn = sum(int(N[y, x]) for y in range(y0, y1) for x in range(x0, x1))
                    tt = sum(int(Tq[y, x]) for y in range(y0, y1) for x in range(x0, x1))
                    assert int(t[x0, x1, y0, y1]) == tt
                    assert int(q[x0, x1, y0, y1]) == s2 - (-(-s1 * s1 // nn))
                    assert (int(t[x0, x1, y0, y1]), int(q[x0, x1, y0, y1])) == oracle.rect(st, Tq, x0, x1, y0, y1)
