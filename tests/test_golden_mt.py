"""The stored multi-tile records of tests/golden/mt_1080p10_n8.json, written
by tests/golden/make_mt_golden.py from the oracle's rectangle-partition
search on the seeded 1920x1080 10-bit frame (seed 7, n = 8; the search the
multi-tile benchmark times), checked here against what holds for any valid
record without rerunning the minute-long enumeration: the stored slices cut
the CTU grid into n rectangles, each CTU once; they meet the area rule
(k * A_min > A_max, luma samples); T and Q are the max (Eq. 1) and sum (Eq. 2)
of the slices' direct sums; T lies within Eq. 4's bound of T_min; and T_min
is no larger than the single-tile-row space's (a subset of this space)."""

import json
import os

import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mt_1080p10_n8.json")


@pytest.fixture(scope="module")
def golden_case(oracle):
    with open(GOLDEN) as f:
        g = json.load(f)
    spec = getattr(synth, g["spec"])
    plane, times = synth.make_frame(spec, seed=g["seed"])
    st = oracle.texture(plane, spec.bit_depth)
    Tq, _ = oracle.time_q(times)
    return g, spec, st, Tq


def test_golden_records_are_valid_decisions(oracle, golden_case):
    g, spec, st, Tq = golden_case
    W, H, n, k = spec.width, spec.height, g["n"], g["k_area"]
    C, R = -(-W // 128), -(-H // 128)
    assert [r["lambda"] for r in g["records"]] == [0.0, 0.1]
    for r in g["records"]:
        assert r["status"] == oracle.OK and r["count"] == 3889333
        regs = r["regions"]
        assert len(regs) == n and regs == sorted(regs, key=lambda v: (v[1], v[0]))  # raster order
        cover = [[0] * C for _ in range(R)]
        areas, ts, qs = [], [], []
        for x0, y0, x1, y1 in regs:
            assert 0 <= x0 < x1 <= C and 0 <= y0 < y1 <= R
            for y in range(y0, y1):
                for x in range(x0, x1):
                    cover[y][x] += 1
            areas.append((min(x1 * 128, W) - x0 * 128) * (min(y1 * 128, H) - y0 * 128))
            t, q = oracle.rect(st, Tq, x0, x1, y0, y1)
            ts.append(t)
            qs.append(q)
        assert all(c == 1 for row in cover for c in row)
        assert sum(areas) == W * H and k * min(areas) > max(areas)
        assert r["t"] == max(ts) and r["q"] == sum(qs)
        lq = oracle.lambda_q(r["lambda"])
        assert r["thr"] == r["t_min"] * (65536 + lq) // 65536
        assert r["t_min"] <= r["t"] <= r["thr"]
        one = oracle.search_dp(st, Tq, n, r["lambda"])
        assert r["t_min"] <= one.t_min
    # lambda = 0 keeps only time-optimal sets; the larger bound can only lower Q
    assert g["records"][0]["t"] == g["records"][0]["t_min"]
    assert g["records"][1]["q"] <= g["records"][0]["q"]
