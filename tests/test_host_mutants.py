"""The host-logic tests of the library catch plausible mistakes: each case
plants one slip in a copy of a host source of the library (the search plan's
pruning and counting in plan.cu, the multi-tile enumeration in mt.cu),
compiles that unit, links it with the other objects of the normal build into
a library of its own, and runs the host-logic ABI tests against it in a
child process.  Every mutant must fail one; the unmutated unit, rebuilt the
same way, must pass them all.  The library's own sources are read, never
changed.  Needs nvcc (no GPU)."""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# fast and sharp first: a killed mutant stops at its first failure
CHECKS = ["test_area_rule_boundary_shapes", "test_count_partitions_matches_brute_force",
          "test_count_partitions_without_the_rule_is_the_closed_form", "test_mt_count_matches_oracle",
          "test_mt_count_limits", "test_mt_list_order_and_validity", "test_mt_list_equals_bruteforce",
          "test_plan_windows_match_oracle", "test_plan_loses_no_partition",
          "test_mt_count_full_frames_matches_cut_partitions", "test_mt_list_full_frames_equals_cut_partitions",
          "test_plan_loses_no_partition_random_shapes"]

# (name, unit, text in it, planted replacement); each text occurs once in its unit
MUTANTS = [
    ("plan_tiling_bound_tight", "plan.cu",
     "kgeo_hi = (int64_t)H / hs[ilo];", "kgeo_hi = (int64_t)H / hs[ihi];"),
    ("plan_reach_right_nonempty", "plan.cu",
     "ok = rest >= 0 && ((Rr >> rest) & 1ull);", "ok = rest > 0 && ((Rr >> rest) & 1ull);"),
    ("plan_window_uniform_dropped", "plan.cu",
     "if (a * (uint64_t)n <= p->A && ((uint64_t)k * a - 1) * (uint64_t)n >= p->A) wins.insert(a);",
     "if (a * (uint64_t)n < p->A && ((uint64_t)k * a - 1) * (uint64_t)n >= p->A) wins.insert(a);"),
    ("plan_heights_top_exclusive", "plan.cu",
     "while (ihi >= 0 && wb * hs[ihi] > hi) --ihi;", "while (ihi >= 0 && wb * hs[ihi] >= hi) --ihi;"),
    ("plan_kset_bottom_exclusive", "plan.cu",
     "if (h >= it.hlo && h <= it.hhi) reach[y] |= (reach[yp] << 1) & full;",
     "if (h > it.hlo && h <= it.hhi) reach[y] |= (reach[yp] << 1) & full;"),
    ("count_min_area_double_counted", "plan.cu",
     "if (i + 1 < a.size() && a[i + 1] <= hi) total -=", "if (i + 1 < a.size() && a[i + 1] < hi) total -="),
    ("plan_kset_largest_count_dropped", "plan.cu",
     "kset[i] = reach[R] & ~1ull & ((2ull << kmax) - 1);", "kset[i] = reach[R] & ~1ull & ((1ull << kmax) - 1);"),
    ("plan_window_single_count_dropped", "plan.cu",
     "if (kmax_w < kmin_w) continue;", "if (kmax_w <= kmin_w) continue;"),
    ("plan_lowest_height_excluded", "plan.cu",
     "it.hlo = hs[ilo];", "it.hlo = hs[ilo] + 1;"),
    ("plan_band_bounds_single_count_dropped", "plan.cu",
     "if (std::max(kmin_w, kgeo_lo) > std::min(kmax_w, kgeo_hi))",
     "if (std::max(kmin_w, kgeo_lo) >= std::min(kmax_w, kgeo_hi))"),
    ("mt_corner_bound_high", "mt.cu",
     "return (corners + 3) / 4;", "return (corners + 4) / 4;"),
    ("mt_area_rule_not_strict", "mt.cu",
     "if ((uint64_t)k * na <= xa) {", "if ((uint64_t)k * na < xa) {"),
    ("mt_pieces_joined_reversed", "mt.cu",
     "for (auto &p : parts) {", "for (auto rp = parts.rbegin(); rp != parts.rend(); ++rp) {\n                    auto &p = *rp;"),
    ("mt_task_bounds_forgotten", "mt.cu",
     "e.rec(tasks[i].ry, tasks[i].amin, tasks[i].amax);", "e.rec(tasks[i].ry, ~0ull, 0);"),
]

_DRIVER = r'''
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import __graft_entry__
__graft_entry__.build = lambda *a, **k: None  # the library under test is already linked
import paper_2012_14792_gb300.build as B
B.LIB = {lib!r}
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu", "--rootdir", {root!r}] + {ids!r}))
'''


def _run(B, tmp_path, name, unit, text):
    d = tmp_path / name
    d.mkdir()
    src = d / unit
    src.write_text(text)
    obj = str(d / (unit[:-3] + ".o"))
    r = subprocess.run([B._nvcc(), *B.ARCH, *B.NVCC_FLAGS, "-I", B.CSRC, "-c", str(src), "-o", obj],
                       capture_output=True, text=True)
    if r.returncode:
        return "compile", r.stderr[-2000:]
    objs = [obj if s == unit else os.path.join(B.BUILD, s[:-3] + ".o") for s in B.SOURCES]
    lib = str(d / "libtrs.so")
    r = subprocess.run([B._nvcc(), *B.ARCH, "-shared", "-o", lib, *objs], capture_output=True, text=True)
    if r.returncode:
        return "link", r.stderr[-2000:]
    ids = [os.path.join(ROOT, "tests", "test_abi.py") + "::" + c for c in CHECKS]
    code = _DRIVER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib, ids=ids)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900, cwd=str(d))
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


def test_every_planted_host_mistake_fails_a_test(tmp_path):
    sys.path.insert(0, ROOT)
    from paper_2012_14792_gb300 import build as B
    if shutil.which(B._nvcc()) is None and not os.path.exists(B._nvcc()):
        pytest.skip("no nvcc")
    B.build()
    sources = {u: open(os.path.join(B.CSRC, u)).read() for u in {m[1] for m in MUTANTS}}
    for name, unit, old, _ in MUTANTS:
        assert sources[unit].count(old) == 1, f"{name}: the mutated text must occur exactly once in {unit}"
    jobs = [("unmutated_" + u[:-3], u, t) for u, t in sources.items()]
    jobs += [(name, unit, sources[unit].replace(old, new)) for name, unit, old, new in MUTANTS]
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = dict(zip([j[0] for j in jobs], ex.map(lambda j: _run(B, tmp_path, *j), jobs)))
    for u in sources:
        rc, log = results.pop("unmutated_" + u[:-3])
        assert rc == 0, f"the unmutated {u} must pass:\n{log}"
    broken = {name: rc for name, (rc, _) in results.items() if rc in ("compile", "link")}
    assert not broken, f"mutants that did not build: {broken}"
    survivors = [name for name, (rc, _) in results.items() if rc == 0]
    assert not survivors, f"mutants no test catches: {survivors}"
