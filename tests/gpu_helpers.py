"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare with the oracle."""

import numpy as np

SSE_REL = 1e-6   # relative tolerance on the reported floating-point SSE
SSE_ABS = 1e-3   # absolute floor: the oracle's long double loses a few units at S1^2 > 2^64


def assert_partition_equal(p, d, R):
    """p: trs_partition from the GPU; d: oracle Decision."""
    assert p.status == d.status, (p.status, d.status)
    if d.status != 0:
        return
    assert (p.t_min_q, p.thr_q, p.t_q, p.q) == (d.t_min, d.thr, d.t, d.q)
    assert p.x_edges() == d.x_edges
    assert p.band_cuts() == d.band_cuts
    assert p.tile_row_mask == 0 and d.row_mask == 0
    assert p.n_tile_rows == 1 and p.n_tile_cols == d.c
    assert p.regions() == d.regions(R)
    assert abs(p.sse - d.sse_real) <= max(SSE_REL * abs(d.sse_real), SSE_ABS)
    assert abs(p.t - d.t_real) <= 1e-12 * max(1.0, d.t_real)
    assert abs(p.t_min - d.t_min_real) <= 1e-12 * max(1.0, d.t_min_real)


def assert_valid_partition(oracle, p, st, Tq, n, k=3):
    """Properties any correct answer has: n slices covering every CTU once,
    the area rule, the Eq. 4 bound and objective terms equal to direct sums."""
    assert p.status == 0
    R, C = st.S1.shape
    cover = np.zeros((R, C), np.int32)
    for (x0, x1, y0, y1) in p.regions():
        cover[y0:y1, x0:x1] += 1
    assert (cover == 1).all()
    ev = oracle.evaluate(st, Tq, p.x_edges(), p.band_cuts())
    assert ev["n"] == n
    assert k * ev["amin"] > ev["amax"]
    assert ev["t"] == p.t_q and ev["q"] == p.q
    assert p.t_q <= p.thr_q
    assert p.t_min_q <= p.t_q


def mt_best(oracle, st, Tq, sets, lam):
    """The multi-tile decision over an explicit list of slice sets (each a
    raster-sorted tuple of (x0, x1, y0, y1) CTU rectangles): T_min (Eq. 3),
    the Q16 bound of Eq. 4, then the smallest (Q, slice list as (y0, x0, y1,
    x1) per slice) within it, each slice's time and floored SSE from the
    oracle's direct rectangle sums.  Regions come back as (x0, y0, x1, y1)."""
    cache = {}

    def rect(r):
        if r not in cache:
            cache[r] = oracle.rect(st, Tq, *r)
        return cache[r]

    cands = []
    for s in sets:
        tq = [rect(r) for r in s]
        key = [(r[2], r[0], r[3], r[1]) for r in s]
        cands.append((max(t for t, _ in tq), sum(q for _, q in tq), key, s))
    if not cands:
        return dict(status=oracle.EINFEASIBLE, count=0)
    t_min = min(c[0] for c in cands)
    thr = t_min * (65536 + oracle.lambda_q(lam)) // 65536
    t, q, _, s = min((c for c in cands if c[0] <= thr), key=lambda c: (c[1], c[2]))
    return dict(status=oracle.OK, count=len(cands), t_min=t_min, thr=thr, t=t, q=q,
                regions=[(r[0], r[2], r[1], r[3]) for r in s])
