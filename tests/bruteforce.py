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


# --- multi-tile rectangular slices (slices of one tile, or unions of whole tiles) ---

def _ctu_rect_partitions(C, R, n):
    """Every partition of the C x R CTU grid into exactly n rectangles
    (x0, x1, y0, y1), built cell by cell from the first free CTU."""
    free = [[True] * C for _ in range(R)]
    out = []

    def rec(acc):
        if len(acc) > n:
            return
        for y in range(R):
            for x in range(C):
                if free[y][x]:
                    for x1 in range(x + 1, C + 1):
                        if not free[y][x1 - 1]:
                            break
                        for y1 in range(y + 1, R + 1):
                            if not all(free[yy][xx] for yy in range(y, y1) for xx in range(x, x1)):
                                break
                            for yy in range(y, y1):
                                for xx in range(x, x1):
                                    free[yy][xx] = False
                            acc.append((x, x1, y, y1))
                            rec(acc)
                            acc.pop()
                            for yy in range(y, y1):
                                for xx in range(x, x1):
                                    free[yy][xx] = True
                    return
        if len(acc) == n:
            out.append(list(acc))

    rec([])
    return out


def _mt_valid(rects, C, R):
    """True if some tile grid makes every rectangle either a run of whole CTU
    rows spanning one tile's width, or a union of whole tiles."""
    for Y in _subsets(range(1, R)):
        ys = [0] + sorted(Y) + [R]
        for X in _subsets(range(1, C)):
            xs = [0] + sorted(X) + [C]
            ok = True
            for i in range(len(xs) - 1):
                for j in range(len(ys) - 1):
                    tx0, tx1, ty0, ty1 = xs[i], xs[i + 1], ys[j], ys[j + 1]
                    inside = [r for r in rects if r[0] < tx1 and r[1] > tx0 and r[2] < ty1 and r[3] > ty0]
                    whole = [r for r in inside if r[0] <= tx0 and r[1] >= tx1 and r[2] <= ty0 and r[3] >= ty1]
                    if whole and (whole[0][1] - whole[0][0], whole[0][3] - whole[0][2]) != (tx1 - tx0, ty1 - ty0):
                        # a union of tiles: its edges on tile lines
                        r = whole[0]
                        if len(inside) != 1 or r[0] not in xs or r[1] not in xs or r[2] not in ys or r[3] not in ys:
                            ok = False
                    elif not all(r[0] == tx0 and r[1] == tx1 and r[2] >= ty0 and r[3] <= ty1 for r in inside):
                        ok = False
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                return True
    return False


def mt_partitions(W, H, n, k=3):
    """Distinct slice sets of the multi-tile space with the area rule, as
    raster-sorted tuples of (x0, x1, y0, y1) in CTUs."""
    C, R, cw, ch = geometry(W, H)
    found = []
    for rects in _ctu_rect_partitions(C, R, n):
        areas = [sum(cw[r[0]:r[1]]) * sum(ch[r[2]:r[3]]) for r in rects]
        if not (k * min(areas) > max(areas)):
            continue
        if _mt_valid(rects, C, R):
            found.append(tuple(sorted(rects, key=lambda r: (r[2], r[0]))))
    return found



def guillotine_partitions(W, H, n, k=3):
    """Partitions of the CTU grid into n rectangles (x0, x1, y0, y1) made by
    full cuts (a cut runs across the whole rectangle being split, and each
    side is split again the same way), with the area rule, as raster-sorted
    tuples.  A partition of a rectangle into at most four rectangles always
    has such a cut (the smallest one without, the pinwheel, has five pieces),
    so for n <= 4 this is the whole multi-tile space, at any frame size;
    with five, the sides of the first cut hold at most four pieces each, so
    only the pinwheels are missing (`cut_partitions` adds them).
    Every slice area a meets A/(n k) < a < k A/n (A the frame's area), which
    bounds the rectangles each sub-problem may hold."""
    from functools import lru_cache
    assert 1 <= n <= 5
    C, R, cw, ch = geometry(W, H)
    px, py = [0], [0]
    for w in cw:
        px.append(px[-1] + w)
    for h in ch:
        py.append(py[-1] + h)
    A = W * H

    def area(x0, x1, y0, y1):
        return (px[x1] - px[x0]) * (py[y1] - py[y0])

    @lru_cache(maxsize=None)
    def parts(x0, x1, y0, y1, j):
        a = area(x0, x1, y0, y1)
        if not (a * n * k > j * A and a * n < j * k * A):
            return frozenset()
        if j == 1:
            return frozenset([((x0, x1, y0, y1),)])
        out = set()
        for j1 in range(1, j):
            for x in range(x0 + 1, x1):
                for left in parts(x0, x, y0, y1, j1):
                    for right in parts(x, x1, y0, y1, j - j1):
                        out.add(tuple(sorted(left + right)))
            for y in range(y0 + 1, y1):
                for top in parts(x0, x1, y0, y, j1):
                    for bottom in parts(x0, x1, y, y1, j - j1):
                        out.add(tuple(sorted(top + bottom)))
        return frozenset(out)

    found = []
    for p in parts(0, C, 0, R, n):
        areas = [area(*r) for r in p]
        if k * min(areas) > max(areas):
            found.append(tuple(sorted(p, key=lambda r: (r[2], r[0]))))
    return found


def pinwheels(W, H, k=3):
    """The five-rectangle partitions without a full cut: a centre rectangle
    [a, b) x [c, d) strictly inside the grid and four arms turning around it,
    clockwise or anticlockwise, with the area rule."""
    C, R, cw, ch = geometry(W, H)
    px, py = [0], [0]
    for w in cw:
        px.append(px[-1] + w)
    for h in ch:
        py.append(py[-1] + h)
    found = []
    for a in range(1, C):
        for b in range(a + 1, C):
            for c in range(1, R):
                for d in range(c + 1, R):
                    centre = (a, b, c, d)
                    turn_cw = [(0, b, 0, c), (b, C, 0, d), (a, C, d, R), (0, a, c, R), centre]
                    turn_ccw = [(0, a, 0, d), (a, C, 0, c), (b, C, c, R), (0, b, d, R), centre]
                    for p in (turn_cw, turn_ccw):
                        areas = [(px[r[1]] - px[r[0]]) * (py[r[3]] - py[r[2]]) for r in p]
                        if k * min(areas) > max(areas):
                            found.append(tuple(sorted(p, key=lambda r: (r[2], r[0]))))
    return found


def cut_partitions(W, H, n, k=3):
    """The whole multi-tile space for n <= 5 at any frame size: full-cut
    partitions, plus the pinwheels when n = 5."""
    found = guillotine_partitions(W, H, n, k)
    return found + pinwheels(W, H, k) if n == 5 else found

def mt_search(W, H, S1, S2, Tq, n, lam_q, k=3):
    """The multi-tile search by brute force: T_min, then the smallest
    (Q, raster-sorted slice list) among slice sets meeting Eq. 4."""
    C, R, cw, ch = geometry(W, H)

    def rsum(a, r):
        return sum(a[y][x] for y in range(r[2], r[3]) for x in range(r[0], r[1]))

    cands = []
    for key in mt_partitions(W, H, n, k):
        t = max(rsum(Tq, r) for r in key)
        q = 0
        for r in key:
            a = sum(cw[r[0]:r[1]]) * sum(ch[r[2]:r[3]])
            s1 = rsum(S1, r)
            q += rsum(S2, r) - (-(-s1 * s1 // a))
        cands.append((key, t, q))
    if not cands:
        return None
    t_min = min(c[1] for c in cands)
    feas = [c for c in cands if c[1] * 65536 <= t_min * (65536 + lam_q)]
    key, t, q = min(feas, key=lambda c: (c[2], [(r[2], r[0], r[3], r[1]) for r in c[0]]))
    return dict(t_min=t_min, t=t, q=q, regions=list(key), count=len(cands))
