"""Pins of the oracle's multi-tile slice search (slices of one tile, or
rectangles of two or more whole tiles; Sec. 1, Fig. 1b).

The oracle enumerates tile grids and groups their tiles into rectangles; the
pure-Python brute force instead cuts the CTU grid into every set of n
rectangles and asks whether some tile grid realises it.  The two methods
share nothing but the definition, so equal counts and equal decisions on
tiny frames pin the enumeration.  The single-tile-row space S(n) is a subset:
T_min can only fall, and the space can only grow.
"""

import numpy as np
import pytest

import bruteforce
from test_oracle_search import random_instance, stats_from


@pytest.mark.parametrize("W,H,n", [(256, 256, 2), (384, 256, 3), (384, 384, 3), (512, 256, 4), (300, 200, 3),
                                   (512, 384, 4), (384, 384, 4), (640, 256, 3), (128, 384, 2), (256, 128, 1)])
def test_count_matches_bruteforce(oracle, W, H, n):
    assert oracle.mt_count(W, H, n) == len(bruteforce.mt_partitions(W, H, n))


@pytest.mark.parametrize("seed", range(24))
def test_search_matches_bruteforce(oracle, seed):
    rng = np.random.default_rng(900 + seed)
    W, H = [(384, 384), (512, 256), (300, 200), (512, 384), (640, 256), (384, 300)][seed % 6]
    n = [2, 3, 4][seed % 3]
    mode = ["random", "flat", "uniform"][seed % 3]
    lam = [0.0, 0.1, 0.3][(seed // 3) % 3]
    S1, S2, N, Tq = random_instance(rng, W, H, mode)
    st = stats_from(oracle, W, H, S1, S2, N)
    got = oracle.mt_search(st, Tq, n, lam)
    ref = bruteforce.mt_search(W, H, S1.tolist(), S2.tolist(), Tq.astype(np.int64).tolist(), n,
                               oracle.lambda_q(lam))
    if ref is None:
        assert got["status"] == oracle.EINFEASIBLE
        return
    assert got["status"] == oracle.OK
    assert (got["t_min"], got["t"], got["q"]) == (ref["t_min"], ref["t"], ref["q"])
    # regions: (x0, y0, x1, y1) in raster order vs the brute force's (x0, x1, y0, y1)
    assert got["regions"] == [(r[0], r[2], r[1], r[3]) for r in ref["regions"]]


@pytest.mark.parametrize("W,H,n", [(832, 480, 4), (384, 384, 3), (512, 384, 4)])
def test_single_tile_row_space_is_a_subset(oracle, W, H, n):
    from paper_2012_14792_gb300 import trs
    assert oracle.mt_count(W, H, n) >= trs.trs_count_partitions(W, H, n)
    rng = np.random.default_rng(W + n)
    S1, S2, N, Tq = random_instance(rng, W, H, "random")
    st = stats_from(oracle, W, H, S1, S2, N)
    mt = oracle.mt_search(st, Tq, n, 0.1)
    one = oracle.search_dp(st, Tq, n, 0.1)
    assert mt["t_min"] <= one.t_min


def test_single_slice_and_invalid(oracle):
    rng = np.random.default_rng(5)
    S1, S2, N, Tq = random_instance(rng, 384, 384, "random")
    st = stats_from(oracle, 384, 384, S1, S2, N)
    got = oracle.mt_search(st, Tq, 1, 0.0)
    assert got["status"] == oracle.OK and got["regions"] == [(0, 0, 3, 3)]
    assert got["t_min"] == int(Tq.astype(np.int64).sum())
    assert oracle.mt_search(st, Tq, 10, 0.0)["status"] == oracle.EINFEASIBLE  # 9 CTUs


@pytest.mark.parametrize("W,H,n", [(384, 384, 3), (512, 384, 4), (384, 384, 4), (640, 256, 3), (300, 200, 3),
                                   (512, 512, 4), (256, 128, 1), (128, 384, 2), (384, 384, 5), (512, 384, 5),
                                   (640, 384, 5), (512, 512, 5), (640, 640, 5)])
def test_cut_partitions_give_the_same_space(W, H, n):
    """Up to five slices, recursive full cuts (and the pinwheels at five)
    reach every partition the brute force finds and no other, so they can
    stand in for it on frames far too large for the brute force."""
    got = bruteforce.cut_partitions(W, H, n)
    assert len(got) == len(set(got))
    assert sorted(got) == sorted(bruteforce.mt_partitions(W, H, n))
    if n == 5:
        assert bruteforce.pinwheels(W, H)          # the pinwheels do occur at these sizes


@pytest.mark.parametrize("W,H,n,lam,seed", [(832, 480, 4, 0.1, 1), (640, 640, 4, 0.0, 2), (1024, 512, 3, 0.3, 3),
                                            (768, 768, 4, 0.1, 4), (832, 480, 5, 0.1, 5), (640, 640, 5, 0.0, 6)])
def test_decision_over_guillotine_sets_equals_oracle(oracle, W, H, n, lam, seed):
    from gpu_helpers import mt_best
    import synth
    plane, times = synth.small_frame(W, H, 10, seed)
    st = oracle.texture(plane, 10)
    Tq, _ = oracle.time_q(times)
    got = mt_best(oracle, st, Tq, bruteforce.cut_partitions(W, H, n), lam)
    ref = oracle.mt_search(st, Tq, n, lam)
    assert got["status"] == ref["status"] == oracle.OK
    assert got["count"] == oracle.mt_count(W, H, n)
    assert (got["t_min"], got["thr"], got["t"], got["q"], got["regions"]) == \
        (ref["t_min"], ref["thr"], ref["t"], ref["q"], ref["regions"])


@pytest.mark.parametrize("seed", range(18))
def test_rectangle_search_equals_tile_grid_search(oracle, seed):
    """The same space enumerated two ways: as tile grids whose tiles are
    grouped (oracle_mt_search) and as partitions of the CTU grid into n
    rectangles (oracle_mt_search_rects).  Equal records and counts."""
    rng = np.random.default_rng(4400 + seed)
    W, H, n = [(832, 480, 5), (640, 640, 4), (1000, 700, 3), (513, 385, 6), (768, 512, 5), (384, 300, 4)][seed % 6]
    S1, S2, N, Tq = random_instance(rng, W, H, ["random", "flat", "uniform"][(seed // 3) % 3])
    st = stats_from(oracle, W, H, S1, S2, N)
    for lam in (0.0, 0.1, 0.3):
        a = oracle.mt_search(st, Tq, n, lam)
        b = oracle.mt_search_rects(st, Tq, n, lam)
        assert a["status"] == b["status"]
        if a["status"] == oracle.OK:
            assert (a["t_min"], a["thr"], a["t"], a["q"], a["regions"]) == (b["t_min"], b["thr"], b["t"], b["q"],
                                                                            b["regions"])
            assert abs(a["sse"] - b["sse"]) <= 1e-9 * max(1.0, abs(a["sse"]))
    assert b["count"] == oracle.mt_count(W, H, n)


@pytest.mark.parametrize("seed", range(12))
def test_rectangle_search_matches_bruteforce(oracle, seed):
    rng = np.random.default_rng(4600 + seed)
    W, H = [(384, 384), (512, 256), (300, 200), (512, 384)][seed % 4]
    n = [2, 3, 4][seed % 3]
    S1, S2, N, Tq = random_instance(rng, W, H, ["random", "flat", "uniform"][seed % 3])
    st = stats_from(oracle, W, H, S1, S2, N)
    lam = [0.0, 0.1, 0.3][(seed // 3) % 3]
    got = oracle.mt_search_rects(st, Tq, n, lam)
    ref = bruteforce.mt_search(W, H, S1.tolist(), S2.tolist(), Tq.astype(np.int64).tolist(), n,
                               oracle.lambda_q(lam))
    if ref is None:
        assert got["status"] == oracle.EINFEASIBLE
        return
    assert (got["t_min"], got["t"], got["q"]) == (ref["t_min"], ref["t"], ref["q"])
    assert got["regions"] == [(r[0], r[2], r[1], r[3]) for r in ref["regions"]]
    assert got["count"] == len(bruteforce.mt_partitions(W, H, n))
