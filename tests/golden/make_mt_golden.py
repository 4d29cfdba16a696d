"""Writes mt_1080p10_n8.json: the oracle's multi-tile decisions (slices of
one tile, or rectangles of whole tiles; Sec. 1, Fig. 1b) on the seeded
1920x1080 10-bit synthetic frame of seed 7 with n = 8 slices, for
lambda = 0 and 0.1 (Eq. 3, Eq. 4, Eq. 2; k = 3).  That search covers
3,889,333 slice sets and takes the oracle's rectangle-partition
enumeration about a minute per lambda on one core, too long to rerun in
every GPU test, so its records are stored.

Calls only the oracle and the synthetic-input generator:

    python tests/golden/make_mt_golden.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import oracle as O  # noqa: E402

SPEC, SEED, N, LAMBDAS = "SPEC_1080P10", 7, 8, (0.0, 0.1)


def main() -> None:
    spec = getattr(synth, SPEC)
    plane, times = synth.make_frame(spec, seed=SEED)
    st = O.texture(plane, spec.bit_depth)
    Tq, _ = O.time_q(times)
    recs = []
    for lam in LAMBDAS:
        r = O.mt_search_rects(st, Tq, N, lam)
        r["lambda"] = lam
        r["regions"] = [list(x) for x in r["regions"]]
        recs.append(r)
    out = {"about": "oracle_mt_search_rects records (regions as (x0, y0, x1, y1) in CTUs, times in Q16 units) "
                    "on synth.make_frame(synth.%s, seed=%d), n = %d, k = 3; written by make_mt_golden.py"
                    % (SPEC, SEED, N),
           "spec": SPEC, "seed": SEED, "n": N, "k_area": 3, "records": recs}
    with open(os.path.join(HERE, "mt_1080p10_n8.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
