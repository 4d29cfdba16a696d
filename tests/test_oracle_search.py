"""Pins of the oracle's search: step 1 (Eq. 3), step 2 (Eq. 2 under Eq. 4), the
k*A_min > A_max rule and the canonical tie-break (Sec. 2.3).

O1 (plain enumeration) is pinned by the closed-form size of the candidate
space, by an independent pure-Python brute force and by hand-worked cases;
O2 (the exact DP) is pinned by equality with O1 on every instance O1 can run.
"""

from math import comb

import numpy as np
import pytest

import bruteforce
import golden_cases


def closed_form_count(C, R, n):
    """|S(n)| without the area rule: choose c-1 of C-1 column lines, r-1 of R-1
    row lines, then n - c*r of the c*(R-r) in-tile lines."""
    tot = 0
    for c in range(1, C + 1):
        for r in range(1, R + 1):
            if c * r <= n:
                tot += comb(C - 1, c - 1) * comb(R - 1, r - 1) * comb(c * (R - r), n - c * r)
    return tot


def stats_from(oracle, W, H, S1, S2, N):
    C, R = oracle.grid(W, H)
    return oracle.Stats(W, H, np.asarray(S1, np.uint64).reshape(R, C), np.asarray(S2, np.uint64).reshape(R, C),
                        np.asarray(N, np.uint64).reshape(R, C), np.zeros((R, C), np.uint32), 0)


def pixel_counts(W, H):
    C, R = -(-W // 128), -(-H // 128)
    cw = [min(128 * (x + 1), W) - 128 * x for x in range(C)]
    ch = [min(128 * (y + 1), H) - 128 * y for y in range(R)]
    return np.array([[w * h for w in cw] for h in ch], np.uint64)


def random_instance(rng, W, H, mode):
    N = pixel_counts(W, H)
    R, C = N.shape
    if mode == "random":
        mu = rng.integers(0, 1024, size=(R, C)).astype(np.uint64)
        S1 = mu * N
        S2 = mu * mu * N + rng.integers(0, 10 ** 6, size=(R, C)).astype(np.uint64)
        Tq = rng.integers(0, 3 * 65536, size=(R, C)).astype(np.uint32)
    elif mode == "flat":
        S1, S2 = 7 * N, 49 * N
        Tq = (rng.integers(0, 4, size=(R, C)) * 65536).astype(np.uint32)
    else:  # uniform times, near-flat texture: ties on T everywhere
        mu = rng.integers(0, 4, size=(R, C)).astype(np.uint64)
        S1 = mu * N
        S2 = mu * mu * N + rng.integers(0, 50, size=(R, C)).astype(np.uint64)
        Tq = np.full((R, C), 65536, np.uint32)
    return S1, S2, N, Tq


@pytest.mark.parametrize("W,H,n", [(832, 480, 4), (832, 480, 8), (832, 480, 16), (1920, 1080, 4),
                                   (384, 384, 3), (640, 256, 5), (128, 128, 1), (256, 640, 6)])
def test_count_matches_closed_form(oracle, W, H, n):
    C, R = oracle.grid(W, H)
    assert oracle.count_enum(W, H, n, area_rule=False) == closed_form_count(C, R, n)


def test_count_at_paper_like_sizes(oracle):
    # the 7x4-CTU (832x480) grid with n = 4 has 271 configurations
    assert oracle.count_enum(832, 480, 4, area_rule=False) == 271


@pytest.mark.parametrize("W,H,n", [(384, 384, 3), (512, 256, 4), (300, 300, 2), (200, 520, 4),
                                   (384, 256, 5), (640, 128, 3)])
def test_constrained_count_matches_bruteforce(oracle, W, H, n):
    assert oracle.count_enum(W, H, n, area_rule=True) == bruteforce.count(W, H, n)


@pytest.mark.parametrize("seed", range(40))
def test_o1_matches_independent_bruteforce(oracle, seed):
    rng = np.random.default_rng(seed)
    C, R = int(rng.integers(1, 4)), int(rng.integers(1, 4))
    W = (C - 1) * 128 + int(rng.integers(1, 129))
    H = (R - 1) * 128 + int(rng.integers(1, 129))
    n = int(rng.integers(1, 6))
    mode = ["random", "flat", "uniform"][seed % 3]
    S1, S2, N, Tq = random_instance(rng, W, H, mode)
    lam_q = int(rng.choice([0, 6554, 19661, 65536]))
    st = stats_from(oracle, W, H, S1, S2, N)
    d = oracle.search_enum(st, Tq, n, lam_q=lam_q)
    ref = bruteforce.search(W, H, S1.tolist(), S2.tolist(), Tq.astype(np.int64).tolist(), n, lam_q)
    if ref is None:
        assert d.status == oracle.EINFEASIBLE
        return
    assert d.status == oracle.OK
    assert (d.t_min, d.t, d.q) == (ref["t_min"], ref["t"], ref["q"])
    assert d.row_mask == sum(1 << (y - 1) for y in ref["row_cuts"])
    assert sorted(d.regions(R)) == sorted(ref["regions"])


@pytest.mark.parametrize("case", golden_cases.cases(), ids=lambda c: c["name"])
@pytest.mark.parametrize("which", ["enum", "dp"])
def test_hand_worked_cases(oracle, case, which):
    st = oracle.texture(golden_cases.plane(case), case["bit_depth"])
    Tq, s = oracle.time_q(golden_cases.times(case))
    assert st.status == oracle.OK and s == oracle.OK
    f = oracle.search_enum if which == "enum" else oracle.search_dp
    d = f(st, Tq, case["n"], lam_q=case["lambda_q"])
    e = case["expect"]
    if e.get("infeasible"):
        assert d.status == oracle.EINFEASIBLE
        return
    assert d.status == oracle.OK
    assert (d.t_min, d.t, d.q) == (e["t_min"], e["t"], e["q"])
    assert d.x_edges == e["x_edges"]
    assert d.band_cuts == golden_cases.band_masks(case)
    assert d.row_mask == 0


def test_single_slice_is_whole_frame(oracle):
    rng = np.random.default_rng(5)
    W, H = 700, 300
    plane = rng.integers(0, 1024, size=(H, W)).astype(np.uint16)
    st = oracle.texture(plane, 10)
    Tq = rng.integers(0, 65536 * 4, size=st.S1.shape).astype(np.uint32)
    for f in (oracle.search_enum, oracle.search_dp):
        d = f(st, Tq, 1)
        assert d.status == oracle.OK and d.c == 1 and d.band_cuts == [0]
        assert d.t == d.t_min == int(Tq.astype(np.uint64).sum())
        s1, s2, nn = int(st.S1.sum()), int(st.S2.sum()), int(st.N.sum())
        assert d.q == s2 - (-(-s1 * s1 // nn))


@pytest.mark.parametrize("C,R,n", [(8, 4, 4), (8, 4, 8), (6, 6, 4), (4, 4, 16), (6, 3, 9)])
def test_uniform_times_divisible_grid(oracle, C, R, n):
    # With equal CTU times t and C*R divisible by n into equal-area slices,
    # T_min = (C*R/n) * t: no slice can be smaller than the mean.
    W, H = 128 * C, 128 * R
    N = pixel_counts(W, H)
    st = stats_from(oracle, W, H, 5 * N, 25 * N, N)
    Tq = np.full((R, C), 3 * 65536, np.uint32)
    for f in (oracle.search_enum, oracle.search_dp):
        d = f(st, Tq, n)
        assert d.status == oracle.OK
        assert d.t_min == (C * R // n) * 3 * 65536


def test_lambda_monotone_and_bound(oracle):
    import synth
    plane, times = synth.small_frame(1100, 700, 10, seed=11)
    st = oracle.texture(plane, 10)
    Tq, _ = oracle.time_q(times)
    prev_q = None
    for lam in [0.0, 0.05, 0.1, 0.3, 1.0, 4.0]:
        d = oracle.search_dp(st, Tq, 6, lam)
        assert d.status == oracle.OK
        assert d.t <= d.thr
        assert d.t * 65536 <= d.t_min * (65536 + oracle.lambda_q(lam))
        if lam == 0.0:
            assert d.t == d.t_min
        if prev_q is not None:
            assert d.q <= prev_q
        prev_q = d.q
        ev = oracle.evaluate(st, Tq, d.x_edges, d.band_cuts)
        assert ev["n"] == 6 and ev["t"] == d.t and ev["q"] == d.q
        assert 3 * ev["amin"] > ev["amax"]


def test_uniform_grid_never_beats_t_min(oracle):
    # The uniform TRS comparator of Sec. 3.2 (a c x r grid of equal slices) is
    # one member of S(n) when it meets the area rule, so T_min <= its time.
    import synth
    plane, times = synth.make_frame(synth.SPEC_1080P10, seed=3)
    st = oracle.texture(plane, 10)
    Tq, _ = oracle.time_q(times)
    C, R = 15, 9
    for n, (c, r) in {4: (2, 2), 8: (4, 2), 12: (4, 3)}.items():
        xs = [i * C // c for i in range(c + 1)]
        cuts = sum(1 << (j * R // r - 1) for j in range(1, r))
        ev = oracle.evaluate(st, Tq, xs, [cuts] * c)
        assert ev["n"] == n
        d = oracle.search_dp(st, Tq, n, 0.0)
        if 3 * ev["amin"] > ev["amax"]:
            assert d.t_min <= ev["t"]


@pytest.mark.parametrize("seed", range(300))
def test_o2_equals_o1_random_tiny(oracle, seed):
    rng = np.random.default_rng(1000 + seed)
    C, R = int(rng.integers(1, 6)), int(rng.integers(1, 6))
    W = (C - 1) * 128 + int(rng.integers(1, 129))
    H = (R - 1) * 128 + int(rng.integers(1, 129))
    n = int(rng.integers(1, 7))
    S1, S2, N, Tq = random_instance(rng, W, H, ["random", "flat", "uniform"][seed % 3])
    st = stats_from(oracle, W, H, S1, S2, N)
    lam_q = int(rng.choice([0, 6554, 19661, 65536]))
    a = oracle.search_enum(st, Tq, n, lam_q=lam_q)
    b = oracle.search_dp(st, Tq, n, lam_q=lam_q)
    assert a.status == b.status
    if a.status == oracle.OK:
        assert (a.t_min, a.thr, a.t, a.q) == (b.t_min, b.thr, b.t, b.q)
        assert a.row_mask == 0  # a tile-row cut never gives the smallest code
        assert a.x_edges == b.x_edges and a.band_cuts == b.band_cuts


def test_o2_equals_o1_ten_thousand_tiny(oracle):
    """O2 equals O1 on 10,000 more seeded tiny instances (grids up to 6 x 6
    CTUs with clipped edges, n up to 8, the three value modes, four lambdas):
    one loop, so a failure names its seed."""
    for seed in range(10_000):
        rng = np.random.default_rng(200_000 + seed)
        C, R = int(rng.integers(1, 7)), int(rng.integers(1, 7))
        W = (C - 1) * 128 + int(rng.integers(1, 129))
        H = (R - 1) * 128 + int(rng.integers(1, 129))
        n = int(rng.integers(1, 9))
        S1, S2, N, Tq = random_instance(rng, W, H, ["random", "flat", "uniform"][seed % 3])
        st = stats_from(oracle, W, H, S1, S2, N)
        lam_q = int(rng.choice([0, 6554, 19661, 65536]))
        a = oracle.search_enum(st, Tq, n, lam_q=lam_q)
        b = oracle.search_dp(st, Tq, n, lam_q=lam_q)
        assert a.status == b.status, seed
        if a.status == oracle.OK:
            assert (a.t_min, a.thr, a.t, a.q, a.x_edges, a.band_cuts) == \
                (b.t_min, b.thr, b.t, b.q, b.x_edges, b.band_cuts), seed


@pytest.mark.parametrize("spec_name,n", [("SPEC_480P8", 4), ("SPEC_480P8", 8), ("SPEC_480P8", 16),
                                         ("SPEC_1080P10", 4)])
def test_o2_equals_o1_paper_sizes(oracle, spec_name, n):
    import synth
    spec = getattr(synth, spec_name)
    for seed in range(2):
        plane, times = synth.make_frame(spec, seed)
        st = oracle.texture(plane, spec.bit_depth)
        Tq, _ = oracle.time_q(times)
        for lam in (0.0, 0.1, 0.3):
            a = oracle.search_enum(st, Tq, n, lam)
            b = oracle.search_dp(st, Tq, n, lam)
            assert a.status == b.status == oracle.OK
            assert (a.t_min, a.t, a.q, a.x_edges, a.band_cuts) == (b.t_min, b.t, b.q, b.x_edges, b.band_cuts)
            assert abs(a.sse_real - b.sse_real) <= 1e-9 * abs(a.sse_real)


def test_infeasible_and_invalid(oracle):
    N = pixel_counts(256, 128)
    st = stats_from(oracle, 256, 128, N, N, N)
    Tq = np.ones((1, 2), np.uint32)
    assert oracle.search_dp(st, Tq, 3).status == oracle.EINFEASIBLE
    assert oracle.search_enum(st, Tq, 3).status == oracle.EINFEASIBLE
    assert oracle.search_dp(st, Tq, 0).status == oracle.EINVAL


def test_random_access_gop_layers():
    import synth
    order = synth.ra_coding_order(16)
    assert order[:6] == [0, 16, 8, 4, 2, 1] and sorted(order) == list(range(17))
    assert [synth.ra_temporal_layer(p) for p in (0, 16, 8, 4, 12, 2, 6, 1, 15)] == [0, 0, 1, 2, 2, 3, 3, 4, 4]


@pytest.mark.parametrize("seed", range(30))
def test_windowed_search_matches_bruteforce(oracle, seed):
    """The lightweight search (every s-th area window) against an independent
    brute force over the configurations that fit a kept window."""
    rng = np.random.default_rng(3000 + seed)
    C, R = int(rng.integers(2, 4)), int(rng.integers(2, 4))
    W = (C - 1) * 128 + int(rng.integers(1, 129))
    H = (R - 1) * 128 + int(rng.integers(1, 129))
    n = int(rng.integers(2, 6))
    step = int(rng.integers(1, 4))
    S1, S2, N, Tq = random_instance(rng, W, H, ["random", "flat", "uniform"][seed % 3])
    st = stats_from(oracle, W, H, S1, S2, N)
    lam_q = int(rng.choice([0, 6554, 65536]))
    d = oracle.search_dp_windows(st, Tq, n, window_step=step, lam_q=lam_q)
    ref = bruteforce.search_in_windows(W, H, S1.tolist(), S2.tolist(), Tq.astype(np.int64).tolist(), n, lam_q, step)
    if ref is None:
        assert d.status == oracle.EINFEASIBLE
        return
    assert d.status == oracle.OK
    assert (d.t_min, d.t, d.q, d.n_windows) == (ref["t_min"], ref["t"], ref["q"], ref["n_windows"])
    assert sorted(d.regions(R)) == sorted(ref["regions"])


def test_windowed_search_step_one_is_exact_and_never_better(oracle):
    import synth
    plane, times = synth.make_frame(synth.SPEC_1080P10, seed=8)
    st = oracle.texture(plane, 10)
    Tq, _ = oracle.time_q(times)
    exact = oracle.search_dp(st, Tq, 8, 0.1)
    one = oracle.search_dp_windows(st, Tq, 8, 0.1, window_step=1)
    assert (one.t_min, one.t, one.q, one.x_edges, one.band_cuts) == (exact.t_min, exact.t, exact.q, exact.x_edges,
                                                                       exact.band_cuts)
    for step in (2, 4, 8):
        h = oracle.search_dp_windows(st, Tq, 8, 0.1, window_step=step)
        assert h.status == oracle.OK and h.t_min >= exact.t_min
        assert h.n_windows == -(-exact.n_windows // step)
        ev = oracle.evaluate(st, Tq, h.x_edges, h.band_cuts)
        assert ev["n"] == 8 and 3 * ev["amin"] > ev["amax"] and ev["t"] == h.t and ev["q"] == h.q


@pytest.mark.parametrize("H,expect_rows", [(511, 1), (512, 2)])
def test_largest_admissible_area_ratio(oracle, H, expect_rows):
    """The area rule admits A_max = k*A_min - 1 and no more (Sec. 2.3, strict
    '>').  A 1-pixel-wide frame of 4 CTU rows split into two slices: with
    H = 511 the top row (128 px) over the rest (383 = 3*128 - 1 px) is valid
    and, with the slow top CTU, the time-optimal split; with H = 512 the rest
    is 384 = 3*128 px, the split is invalid and two rows over two wins."""
    W, n = 1, 2
    N = pixel_counts(W, H)
    S1, S2 = 5 * N, 25 * N
    Tq = (np.array([[10], [1], [1], [1]]) * 65536).astype(np.uint32)
    st = stats_from(oracle, W, H, S1, S2, N)
    ref = bruteforce.search(W, H, S1.tolist(), S2.tolist(), Tq.astype(np.int64).tolist(), n, 0)
    assert ref["t_min"] == (10 if expect_rows == 1 else 11) * 65536
    for d in (oracle.search_enum(st, Tq, n, 0.0), oracle.search_dp(st, Tq, n, 0.0)):
        assert d.status == oracle.OK
        assert (d.t_min, d.t, d.q) == (ref["t_min"], ref["t"], ref["q"])
        assert d.band_cuts[0] == 1 << (expect_rows - 1)


def _exact_sse(plane, W, H, rects):
    """Per slice S2 - S1^2/N as exact rationals, from the samples themselves
    (rects as (x0, x1, y0, y1) in CTUs)."""
    from fractions import Fraction
    out = []
    for x0, x1, y0, y1 in rects:
        blk = plane[y0 * 128:min(y1 * 128, H), x0 * 128:min(x1 * 128, W)].astype(np.int64)
        s1, s2 = int(blk.sum()), int((blk * blk).sum())
        out.append(Fraction(s2) - Fraction(s1 * s1, blk.size))
    return out


@pytest.mark.parametrize("W,H,n,seed", [(300, 200, 3, 1), (832, 480, 4, 2), (640, 384, 5, 3)])
def test_reported_sse_is_exact_sum_of_squared_deviations(oracle, W, H, n, seed):
    """Eq. 2: the reported SSE of the chosen partition is the exact sum over
    its slices of sum (p - mean)^2, and Q is the sum of their floors."""
    import math
    import synth
    plane, times = synth.small_frame(W, H, 10, seed)
    d, _, _ = oracle.decide(plane, times, 10, n, 0.1)
    assert d.status == oracle.OK
    C, R = oracle.grid(W, H)
    parts = _exact_sse(plane, W, H, d.regions(R))
    assert d.q == sum(math.floor(p) for p in parts)
    assert abs(d.sse_real - float(sum(parts))) <= 1e-9 * float(sum(parts))


@pytest.mark.parametrize("W,H,n,seed", [(832, 480, 4, 4), (640, 640, 5, 5)])
def test_multi_tile_reported_sse_is_exact(oracle, W, H, n, seed):
    import math
    import synth
    plane, times = synth.small_frame(W, H, 10, seed)
    st = oracle.texture(plane, 10)
    Tq, _ = oracle.time_q(times)
    r = oracle.mt_search(st, Tq, n, 0.1)
    assert r["status"] == oracle.OK
    parts = _exact_sse(plane, W, H, [(x0, x1, y0, y1) for (x0, y0, x1, y1) in r["regions"]])
    assert r["q"] == sum(math.floor(p) for p in parts)
    assert abs(r["sse"] - float(sum(parts))) <= 1e-9 * float(sum(parts))


@pytest.mark.parametrize("seed", range(40))
def test_evaluate_and_rect_match_direct_sums(oracle, seed):
    """The checkers the GPU tests lean on (oracle_evaluate for a whole
    partition, oracle_rect for one rectangle) against sums written out here
    over random tile columns and slice cuts of random tiny frames: Eq. 1's
    slowest slice, Eq. 2's floored SSE sum, the smallest and largest area."""
    rng = np.random.default_rng(500 + seed)
    C, R = int(rng.integers(1, 6)), int(rng.integers(1, 6))
    W = (C - 1) * 128 + int(rng.integers(1, 129))
    H = (R - 1) * 128 + int(rng.integers(1, 129))
    S1, S2, N, Tq = random_instance(rng, W, H, "random")
    st = stats_from(oracle, W, H, S1, S2, N)
    inner = [x for x in range(1, C) if rng.random() < 0.5]
    x_edges = [0] + inner + [C]
    band_cuts = [int(rng.integers(0, 1 << (R - 1))) if R > 1 else 0 for _ in range(len(x_edges) - 1)]
    slices = []
    for b in range(len(x_edges) - 1):
        y0 = 0
        for y in range(1, R + 1):
            if y == R or (band_cuts[b] >> (y - 1)) & 1:
                slices.append((x_edges[b], x_edges[b + 1], y0, y))
                y0 = y
    terms = []
    for x0, x1, y0, y1 in slices:
        t = int(Tq[y0:y1, x0:x1].astype(np.int64).sum())
        s1, s2, a = (int(v[y0:y1, x0:x1].astype(object).sum()) for v in (S1, S2, N))
        q = s2 - (-(-s1 * s1 // a))
        terms.append((t, q, a))
        assert oracle.rect(st, Tq, x0, x1, y0, y1) == (t, q)
    ev = oracle.evaluate(st, Tq, x_edges, band_cuts)
    assert ev == dict(t=max(t for t, _, _ in terms), q=sum(q for _, q, _ in terms),
                      amin=min(a for _, _, a in terms), amax=max(a for _, _, a in terms), n=len(terms))
