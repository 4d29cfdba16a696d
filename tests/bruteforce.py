"""Independent pure-Python statement of the TRS search, for tiny grids.

It enumerates every subset of tile-row lines, every subset of tile-column
lines and every subset of in-tile slice lines with itertools, keeps the
configurations with exactly n slices, applies the k*A_min > A_max rule
(Sec. 2.3), Eq. 1/3 for the time term, Eq. 4 for the bound and Eq. 2 (floored
per slice) for the quality term, and picks the smallest (Q, code).  It shares
nothing with the C oracle beyond the readings written in its header.
"""

from __future__ import annotations

import itertools

CTU = 128


def _subsets(items):
    items = list(items)
    for r in range(len(items) + 1):
        for c in itertools.combinations(items, r):
            yield frozenset(c)


def geometry(W, H):
    C = -(-W // CTU)
    R = -(-H // CTU)
    cw = [min(CTU * (x + 1), W) - CTU * x for x in range(C)]
    ch = [min(CTU * (y + 1), H) - CTU * y for y in range(R)]
    return C, R, cw, ch


def configurations(W, H, n):
    """Yields (code, regions, row_cuts) for every configuration with n slices."""
    C, R, _, _ = geometry(W, H)
    for Y in _subsets(range(1, R)):
        free = [y for y in range(1, R) if y not in Y]
        for X in _subsets(range(1, C)):
            edges = [0] + sorted(X) + [C]
            nb = len(edges) - 1
            per_band = list(_subsets(free))
            for choice in itertools.product(per_band, repeat=nb):
                total = sum(len(Y) + 1 + len(s) for s in choice)
                if total != n:
                    continue
                code = tuple(1 if y in Y else 0 for y in range(1, R))
                regions = []
                for b in range(nb):
                    code += (edges[b + 1],) + tuple(1 if y in choice[b] else 0 for y in free)
                    cuts = sorted(Y | choice[b])
                    ys = [0] + cuts + [R]
                    for i in range(len(ys) - 1):
                        regions.append((edges[b], edges[b + 1], ys[i], ys[i + 1]))
                yield code, regions, Y


def search(W, H, S1, S2, Tq, n, lam_q, k=3):
    """Returns dict(t_min, t, q, regions, code, row_cuts) or None if S(n) is empty.
    S1, S2, Tq are nested lists [R][C] of ints."""
    C, R, cw, ch = geometry(W, H)

    def rsum(a, r):
        x0, x1, y0, y1 = r
        return sum(a[y][x] for y in range(y0, y1) for x in range(x0, x1))

    def area(r):
        x0, x1, y0, y1 = r
        return sum(cw[x0:x1]) * sum(ch[y0:y1])

    cands = []
    for code, regions, Y in configurations(W, H, n):
        areas = [area(r) for r in regions]
        if not (k * min(areas) > max(areas)):
            continue
        t = max(rsum(Tq, r) for r in regions)
        q = 0
        for r, a in zip(regions, areas):
            s1 = rsum(S1, r)
            s2 = rsum(S2, r)
            q += s2 - (-(-s1 * s1 // a))
        cands.append((code, regions, Y, t, q))
    if not cands:
        return None
    t_min = min(c[3] for c in cands)
    feas = [c for c in cands if c[3] * 65536 <= t_min * (65536 + lam_q)]
    best = min(feas, key=lambda c: (c[4], c[0]))
    return dict(t_min=t_min, t=best[3], q=best[4], regions=best[1], code=best[0], row_cuts=best[2])


def count(W, H, n, k=3, area_rule=True):
    C, R, cw, ch = geometry(W, H)
    c = 0
    for _, regions, _ in configurations(W, H, n):
        if area_rule:
            areas = [sum(cw[r[0]:r[1]]) * sum(ch[r[2]:r[3]]) for r in regions]
            if not (k * min(areas) > max(areas)):
                continue
        c += 1
    return c


def search_in_windows(W, H, S1, S2, Tq, n, lam_q, window_step, k=3):
    """The lightweight search by brute force: the candidates are the
    configurations whose slice areas all fit one kept window [a, k*a-1], the
    kept a being every window_step-th admissible slice area counted from the
    largest."""
    C, R, cw, ch = geometry(W, H)
    A = W * H
    widths = {sum(cw[i:j]) for i in range(C) for j in range(i + 1, C + 1)}
    heights = {sum(ch[i:j]) for i in range(R) for j in range(i + 1, R + 1)}
    wins = sorted({w * h for w in widths for h in heights if w * h * n <= A and (k * w * h - 1) * n >= A})
    kept = [a for i, a in enumerate(wins) if (len(wins) - 1 - i) % window_step == 0]

    def rsum(a, r):
        x0, x1, y0, y1 = r
        return sum(a[y][x] for y in range(y0, y1) for x in range(x0, x1))

    cands = []
    for code, regions, Y in configurations(W, H, n):
        areas = [sum(cw[r[0]:r[1]]) * sum(ch[r[2]:r[3]]) for r in regions]
        if not any(all(a <= x <= k * a - 1 for x in areas) for a in kept):
            continue
        t = max(rsum(Tq, r) for r in regions)
        q = sum(rsum(S2, r) - (-(-rsum(S1, r) ** 2 // ar)) for r, ar in zip(regions, areas))
        cands.append((code, regions, t, q))
    if not cands:
        return None
    t_min = min(c[2] for c in cands)
    feas = [c for c in cands if c[2] * 65536 <= t_min * (65536 + lam_q)]
    best = min(feas, key=lambda c: (c[3], c[0]))
    return dict(t_min=t_min, t=best[2], q=best[3], regions=best[1], n_windows=len(kept))
