"""A direct check of the exact search (O2) at the benchmarked size, 3840x2160
with n = 16, where the plain enumeration (O1) cannot run (3.6e12
partitions): the decision must be optimal against every partition one local
move away from it, each evaluated by direct sums (oracle_evaluate), not by
the search's window / band / column decomposition.

Moves, all keeping exactly n slices and one tile row: a slice boundary moved
to any free line of any tile column (one removed, one added: this includes
shifting it by one row); a tile-column edge shifted by one CTU; a tile
column split in two, its right part one slice, with one boundary removed
anywhere.  For every neighbour that meets the area rule (k * A_min > A_max,
Sec. 2.3): its time is not below T_min (Eq. 3), and if it meets Eq. 4's
bound its quality term Q (Eq. 2) is not below the decision's."""

import numpy as np
import pytest

import synth

N, K = 16, 3


def _bits(mask: int, R: int) -> list[int]:
    return [y for y in range(1, R) if (mask >> (y - 1)) & 1]


def _neighbours(xe: list[int], cuts: list[int], C: int, R: int):
    c = len(cuts)
    # a boundary removed from one column and added to a free line of any column
    for b in range(c):
        for y in _bits(cuts[b], R):
            base = list(cuts)
            base[b] &= ~(1 << (y - 1))
            for b2 in range(c):
                for y2 in range(1, R):
                    if (b2, y2) != (b, y) and not (base[b2] >> (y2 - 1)) & 1:
                        nc = list(base)
                        nc[b2] |= 1 << (y2 - 1)
                        yield list(xe), nc
    # an inner tile-column edge shifted by one CTU
    for i in range(1, c):
        for dx in (-1, 1):
            x = xe[i] + dx
            if xe[i - 1] < x < xe[i + 1]:
                ne = list(xe)
                ne[i] = x
                yield ne, list(cuts)
    # two boundaries each shifted by one row (in one column or two)
    lines = [(b, y) for b in range(c) for y in _bits(cuts[b], R)]
    for i in range(len(lines)):
        for j in range(i + 1, len(lines)):
            for d1 in (-1, 1):
                for d2 in (-1, 1):
                    nc = list(cuts)
                    ok = True
                    for (b, y), dy in ((lines[i], d1), (lines[j], d2)):
                        nc[b] &= ~(1 << (y - 1))
                    for (b, y), dy in ((lines[i], d1), (lines[j], d2)):
                        y2 = y + dy
                        if not 1 <= y2 < R or (nc[b] >> (y2 - 1)) & 1:
                            ok = False
                            break
                        nc[b] |= 1 << (y2 - 1)
                    if ok:
                        yield list(xe), nc
    # an inner tile-column edge shifted by one CTU and one boundary by one row
    for i in range(1, c):
        for dx in (-1, 1):
            x = xe[i] + dx
            if not xe[i - 1] < x < xe[i + 1]:
                continue
            ne = list(xe)
            ne[i] = x
            for (b, y) in lines:
                for dy in (-1, 1):
                    y2 = y + dy
                    if 1 <= y2 < R and not (cuts[b] >> (y2 - 1)) & 1:
                        nc = list(cuts)
                        nc[b] = (nc[b] & ~(1 << (y - 1))) | (1 << (y2 - 1))
                        yield ne, nc
    # a column split at x (the right part one slice), one boundary removed anywhere
    for b in range(c):
        for x in range(xe[b] + 1, xe[b + 1]):
            ne = xe[:b + 1] + [x] + xe[b + 1:]
            split = cuts[:b + 1] + [0] + cuts[b + 1:]
            for b2 in range(c + 1):
                for y in _bits(split[b2], R):
                    nc = list(split)
                    nc[b2] &= ~(1 << (y - 1))
                    yield ne, nc


@pytest.mark.parametrize("frame", [0, 21, 42, 63])
@pytest.mark.parametrize("lam", [0.0, 0.1])
def test_decision_is_optimal_against_every_local_move(oracle, frame, lam):
    plane, times = synth.sequence_2160p_frame(frame)
    d, st, Tq = oracle.decide(plane, times, 10, N, lam)
    assert d.status == oracle.OK
    C, R = oracle.grid(plane.shape[1], plane.shape[0])
    xe, cuts = list(d.x_edges), list(d.band_cuts)
    own = oracle.evaluate(st, Tq, xe, cuts)
    assert (own["t"], own["q"], own["n"]) == (d.t, d.q, N)
    assert d.thr == d.t_min * (65536 + oracle.lambda_q(lam)) // 65536  # Eq. 4's bound, written out
    assert d.t_min <= d.t <= d.thr
    seen = valid = feasible = 0
    for ne, nc in _neighbours(xe, cuts, C, R):
        seen += 1
        e = oracle.evaluate(st, Tq, ne, nc)
        assert e["n"] == N
        if not K * e["amin"] > e["amax"]:
            continue
        valid += 1
        assert e["t"] >= d.t_min, (ne, nc)
        if e["t"] <= d.thr:
            feasible += 1
            assert e["q"] >= d.q, (ne, nc)
    # the moves reach enough of the space to mean something
    assert seen > 500 and valid > 100 and feasible > 0, (seen, valid, feasible)
