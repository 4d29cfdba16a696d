"""The oracle's pins catch plausible mistakes: each case below plants one slip
in a copy of ``oracle/trs_oracle.c`` (a dropped term, a wrong sign, a bound
off by one, transposed indices, a reversed tie order, a max taken as a sum),
builds it into a library of its own, and runs the oracle pin tests against
it in a child process.  Every mutant must fail at least one pin; the
unmutated copy must pass them all, so a broken harness cannot pass for
caught mutants.  The oracle's own source is read, never changed.

Each slip names the passage whose arithmetic it breaks."""

import concurrent.futures as cf
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "trs_oracle.c")
PINS = ("test_oracle_texture.py", "test_oracle_tables.py", "test_oracle_search.py", "test_oracle_mt.py")

# (name, passage, text in the oracle, planted replacement); each text occurs once
MUTANTS = [
    ("texture_square_dropped", "Eq. 2 (S2)",
     "S2[i] += (uint64_t)p * p;", "S2[i] += (uint64_t)p;"),
    ("texture_big_endian", "sample layout",
     "(uint32_t)row[2 * x] | ((uint32_t)row[2 * x + 1] << 8)",
     "((uint32_t)row[2 * x] << 8) | (uint32_t)row[2 * x + 1]"),
    ("texture_ctu_transposed", "CTU grid",
     "int i = (y / OR_CTU) * C + (x / OR_CTU);", "int i = (x / OR_CTU) * R + (y / OR_CTU);"),
    ("texture_range_off_by_one", "sample range",
     "if (p >> bd) bad = 1;", "if (p >> (bd + 1)) bad = 1;"),
    ("time_truncated", "Sec. 2.1 times in Q16",
     "Tq[i] = (uint32_t)rint(v * 65536.0);", "Tq[i] = (uint32_t)(v * 65536.0);"),
    ("time_domain_inclusive", "Sec. 2.1 times in Q16",
     "!(v < 65536.0)", "!(v <= 65536.0)"),
    ("sat_last_column_dropped", "summed-area table",
     "for (int xx = 0; xx < x; ++xx) s += v[yy * C + xx];",
     "for (int xx = 0; xx + 1 < x; ++xx) s += v[yy * C + xx];"),
    ("lambda_scale", "Eq. 4 lambda in Q16",
     "uint32_t oracle_lambda_q(float lambda) { return (uint32_t)rint((double)lambda * 65536.0); }",
     "uint32_t oracle_lambda_q(float lambda) { return (uint32_t)rint((double)lambda * 65535.0); }"),
    ("sse_floor_instead_of_ceil", "Eq. 2 (floored SSE)",
     "u128 c = (sq + (u128)(N - 1)) / (u128)N;", "u128 c = sq / (u128)N;"),
    ("sse_sign", "Eq. 2",
     "return S2 - (uint64_t)c;", "return S2 + (uint64_t)c;"),
    ("rect_time_overwritten", "Eq. 1",
     "s.T += f->Tq[i];", "s.T = f->Tq[i];"),
    ("eq4_bound_rounded_up", "Eq. 4",
     "u128 q = v / 65536u;", "u128 q = (v + 65535u) / 65536u;"),
    ("enum_area_rule_not_strict", "Sec. 2.3 area rule",
     "return !e->area_rule || (u128)e->k_area * p->amin > (u128)p->amax;",
     "return !e->area_rule || (u128)e->k_area * p->amin >= (u128)p->amax;"),
    ("enum_eq4_exclusive", "Eq. 4",
     "(u128)p->tmax * 65536u <= (u128)e->t_min * (65536u + (u128)e->lambda_q);",
     "(u128)p->tmax * 65536u < (u128)e->t_min * (65536u + (u128)e->lambda_q);"),
    ("enum_time_summed", "Eq. 1 (slowest slice)",
     "if (s.T > p.tmax) p.tmax = s.T;", "p.tmax += s.T;"),
    ("enum_tie_to_last", "tie order",
     "if (!e->have_best || p->q < e->best_q) {", "if (!e->have_best || p->q <= e->best_q) {"),
    ("dp_row_times_summed", "Eq. 1, Eq. 3",
     "uint64_t v = G[yp][k - 1] > s.T ? G[yp][k - 1] : s.T;", "uint64_t v = G[yp][k - 1] + s.T;"),
    ("dp_columns_min_not_max", "Eq. 1, Eq. 3",
     "uint64_t v = F[xp][m - k] > Vb[k] ? F[xp][m - k] : Vb[k];",
     "uint64_t v = F[xp][m - k] > Vb[k] ? Vb[k] : F[xp][m - k];"),
    ("dp_window_top_exclusive", "Sec. 2.3 area rule",
     "if (s.N < d->a_lo || s.N > d->a_hi) return 0;", "if (s.N < d->a_lo || s.N >= d->a_hi) return 0;"),
    ("dp_tie_reversed", "tie order",
     "(q == best.q && code_less(&cur, &best, f.R))", "(q == best.q && code_less(&best, &cur, f.R))"),
    ("mt_area_rule_not_strict", "Sec. 2.3 area rule (multi-tile)",
     "if (!((uint64_t)e->k_area * amin > amax)) return;", "if (!((uint64_t)e->k_area * amin >= amax)) return;"),
    ("mt_eq4_exclusive", "Eq. 4 (multi-tile)",
     "if (tmax > e->thr) return;", "if (tmax >= e->thr) return;"),
    ("time_round_half_away", "Sec. 2.1 times in Q16 (half-even)",
     "Tq[i] = (uint32_t)rint(v * 65536.0);", "Tq[i] = (uint32_t)round(v * 65536.0);"),
    ("light_windows_from_smallest", "Sec. 4 lighter search",
     "if ((nw - 1 - i) % window_step == 0) win[kept++] = win[i];", "if (i % window_step == 0) win[kept++] = win[i];"),
    ("enum_rest_unclipped", "Sec. 2.3 area rule (the rest of the frame, clipped edge CTUs)",
     "int wpx = (x1 * OR_CTU < f->W ? x1 * OR_CTU : f->W);", "int wpx = x1 * OR_CTU;"),
    ("enum_rest_count_off_by_one", "exactly n slices (slices still to come)",
     "u128 left = (u128)(uint64_t)(e->n - used);", "u128 left = (u128)(uint64_t)(e->n - used + 1);"),
    ("enum_line_skipped", "in-tile slice cuts",
     "enum_lines(e, x, x1, y + 1, y, cuts | (1ull << (y - 1)), tile_row ? k : k + 1, used, c);",
     "enum_lines(e, x, x1, y + 2 > f->R ? f->R : y + 2, y, cuts | (1ull << (y - 1)), tile_row ? k : k + 1, used, c);"),
    ("texture_packed_bit_order", "packed 10-bit sample layout",
     "p |= (uint32_t)((row[bit >> 3] >> (bit & 7)) & 1u) << i;",
     "p |= (uint32_t)((row[bit >> 3] >> (bit & 7)) & 1u) << (9 - i);"),
    ("texture_packed_row_bytes", "packed 10-bit sample layout",
     "size_t bit = (size_t)10 * x + i;", "size_t bit = (size_t)10 * x + (i ^ 1);"),
    ("mt_rects_slices_left", "exactly n slices (multi-tile, rectangle partitions)",
     "int left = e->n - e->ns;", "int left = e->n - e->ns - 1;"),
    ("enum_tile_rows_bound", "exactly n slices",
     "if (used + e->r > e->n) return;", "if (used + e->r >= e->n) return;"),
    ("sse_exact_sign", "Eq. 2 (reported SSE)",
     "return (long double)S2 - ((long double)S1 * (long double)S1) / (long double)N;",
     "return (long double)S2 + ((long double)S1 * (long double)S1) / (long double)N;"),
    ("dp_lambda_ignored", "Eq. 4",
     "d.thr = eq4_thr(t_min, lambda_q);", "d.thr = eq4_thr(t_min, 0);"),
    ("dp_step2_bound_exclusive", "Eq. 4",
     "if (step == 2 && s.T > d->thr) return 0;", "if (step == 2 && s.T >= d->thr) return 0;"),
    ("mt_split_all_cuts_dropped", "in-tile slices (multi-tile)",
     "for (uint64_t cm = 0; cm < (1ull << (h - 1)); ++cm) {",
     "for (uint64_t cm = 0; cm + 1 < (1ull << (h - 1)); ++cm) {"),
    ("mt_groups_one_row", "rectangles of whole tiles (multi-tile)",
     "for (int h = 1; ty + h <= e->r; ++h) {", "for (int h = 1; ty + h <= e->r && h < 2; ++h) {"),
    ("texture_vmax_min", "sample range check",
     "if (p > vmax[i]) vmax[i] = p;", "if (p < vmax[i]) vmax[i] = p;"),
    ("texture_pitch_ignored", "sample layout",
     "const uint8_t *row = base + (size_t)y * pitch;",
     "const uint8_t *row = base + (size_t)y * (size_t)W * (size_t)bps;"),
    ("time_nan_accepted", "Sec. 2.1 times in Q16",
     "if (!(v >= 0.0) || !(v < 65536.0)) {", "if (v < 0.0 || v >= 65536.0) {"),
    ("dp_tmin_first_window_only", "Eq. 3",
     "if (t < t_min) t_min = t;", "if (t < t_min && t_min == OR_INF) t_min = t;"),
    ("evaluate_time_summed", "Eq. 1 (checker)",
     "                if (s.T > t) t = s.T;\n                q += sse_floor(s.S1, s.S2, s.N);",
     "                t += s.T;\n                q += sse_floor(s.S1, s.S2, s.N);"),
    ("evaluate_amin_wrong", "Sec. 2.3 area rule (checker)",
     "                if (s.N < amin) amin = s.N;\n                if (s.N > amax) amax = s.N;\n                nreg++;",
     "                if (s.N > amin) amin = s.N;\n                if (s.N > amax) amax = s.N;\n                nreg++;"),
    ("rect_q_is_time", "Eq. 2 (checker)",
     "    *q_out = sse_floor(s.S1, s.S2, s.N);\n    return OR_OK;\n}", "    *q_out = s.T;\n    return OR_OK;\n}"),
]

_DRIVER = r'''
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
from oracle import oracle as O
O._SRC, O._BUILD, O._LIB = {src!r}, {build!r}, {lib!r}
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu", "--rootdir", {root!r}] + {pins!r}))
'''


def _run(tmp_path, name, text):
    d = tmp_path / name
    d.mkdir()
    src = d / "trs_oracle.c"
    src.write_text(text)
    code = _DRIVER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), src=str(src), build=str(d),
                          lib=str(d / "liboracle.so"), pins=[os.path.join(ROOT, "tests", p) for p in PINS])
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900, cwd=str(d))
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    original = open(SRC).read()
    for name, _, old, _ in MUTANTS:
        assert original.count(old) == 1, f"{name}: the mutated text must occur exactly once in the oracle"
    jobs = [("unmutated", original)] + [(name, original.replace(old, new)) for name, _, old, new in MUTANTS]
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = dict(zip([j[0] for j in jobs], ex.map(lambda j: _run(tmp_path, *j), jobs)))
    rc, log = results.pop("unmutated")
    assert rc == 0, "the unmutated oracle copy must pass its pins:\n" + log
    survivors = [name for name, (rc, _) in results.items() if rc == 0]
    assert not survivors, f"mutants no pin catches: {survivors}"
