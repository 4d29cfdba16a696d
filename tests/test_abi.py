"""The C ABI library loads without a GPU, exports every entry point that
include/trs.h declares, agrees with the binding on structure sizes, and its
host-side search plan lists the same area windows as the oracle."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def trs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_14792_gb300 import trs as t
    return t


def declared_functions():
    src = open(os.path.join(ROOT, "include", "trs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(trs_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_hot_path(trs):
    names = declared_functions()
    for required in ("trs_texture_map", "trs_region_tables", "trs_search", "trs_batch_decide"):
        assert required in names


def test_every_declared_symbol_is_exported(trs):
    lib = trs.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("name", ["trs_opts", "trs_ctu_stats", "trs_tables_layout", "trs_partition",
                                  "trs_frame_desc", "trs_server_opts", "trs_decision", "trs_server_stats",
                                  "trs_tune_report", "trs_mt_partition"])
def test_struct_sizes_match_binding(trs, name):
    import ctypes
    assert trs.trs_sizeof(name) == ctypes.sizeof(getattr(trs, name))


def test_strerror_and_version(trs):
    assert trs.trs_version() == 1
    assert trs.trs_strerror(0) == "ok"
    assert "area rule" in trs.trs_strerror(trs.EINFEASIBLE)


@pytest.mark.parametrize("W,H,n", [(832, 480, 4), (832, 480, 8), (1920, 1080, 8), (3840, 2160, 16),
                                   (3840, 2160, 8), (1000, 700, 6), (128, 128, 1), (8192, 4096, 32)])
def test_plan_windows_match_oracle(trs, oracle, W, H, n):
    import numpy as np
    nw, ni = trs.trs_plan_stats(W, H, n)
    C, R = oracle.grid(W, H)
    if W * H > 4000 * 2200:
        return  # oracle O2 would take long; the window count is geometry only and checked below
    z = np.zeros((R, C), np.uint64)
    st = oracle.Stats(W, H, z, z, z + 1, np.zeros((R, C), np.uint32), 0)
    d = oracle.search_dp(st, np.zeros((R, C), np.uint32), n)
    assert d.n_windows == nw
    assert ni >= 1 or nw == 0


def test_plan_rejects_oversize(trs):
    with pytest.raises(trs.TrsError):
        trs.trs_plan_stats(8193, 100, 4)
    with pytest.raises(trs.TrsError):
        trs.trs_plan_stats(100, 4097, 4)
    with pytest.raises(trs.TrsError):
        trs.trs_plan_stats(100, 100, 33)


def _brute_partitions(W, H, n, k):
    """Distinct slice sets of S(n) (the rule applied to luma-sample areas),
    by enumerating every code with bruteforce.configurations."""
    import bruteforce
    C, R, cw, ch = bruteforce.geometry(W, H)
    seen = set()
    for _, regions, _ in bruteforce.configurations(W, H, n):
        areas = [sum(cw[r[0]:r[1]]) * sum(ch[r[2]:r[3]]) for r in regions]
        if k * min(areas) > max(areas):
            seen.add(frozenset(regions))
    return len(seen)


@pytest.mark.parametrize("W,H,n", [(384, 384, 3), (512, 256, 4), (500, 300, 4), (640, 384, 5), (300, 520, 3),
                                   (129, 640, 4), (640, 129, 2), (256, 256, 1)])
def test_count_partitions_matches_brute_force(trs, W, H, n):
    assert trs.trs_count_partitions(W, H, n) == _brute_partitions(W, H, n, 3)


@pytest.mark.parametrize("C,R,n", [(7, 4, 4), (15, 9, 8), (30, 17, 16), (5, 5, 1)])
def test_count_partitions_without_the_rule_is_the_closed_form(trs, C, R, n):
    """With k beyond every area ratio the rule admits all: choose c tile
    columns, then n - c of the c(R-1) in-column cut lines."""
    from math import comb
    expect = sum(comb(C - 1, c - 1) * comb(c * (R - 1), n - c) for c in range(1, min(C, n) + 1))
    got = trs.trs_count_partitions(C * 128, R * 128, n, 1 << 20)
    assert got == pytest.approx(float(expect), rel=1e-15)


@pytest.mark.parametrize("W,H,n", [(256, 256, 2), (384, 256, 3), (384, 384, 3), (300, 200, 3), (512, 384, 4),
                                   (640, 256, 3), (256, 128, 1), (832, 480, 4), (1024, 512, 3), (640, 640, 5)])
def test_mt_count_matches_oracle(trs, oracle, W, H, n):
    """The library's host enumeration of the multi-tile space (slices of one
    tile, or rectangles of whole tiles) finds the oracle's set count."""
    assert trs.trs_mt_count(W, H, n) == oracle.mt_count(W, H, n)


def test_mt_count_limits(trs):
    assert trs.trs_mt_count(128, 128, 1) == 1
    assert trs.trs_mt_count(128, 128, 2) == 0          # one CTU cannot hold two slices
    for bad in [(0, 128, 1), (128, 128, 0), (64 * 128 + 1, 128, 1), (128, 128, trs.MAX_REGIONS + 1)]:
        with pytest.raises(trs.TrsError) as e:
            trs.trs_mt_count(*bad)
        assert e.value.status == trs.EINVAL


@pytest.mark.parametrize("W,H,n", [(1920, 1080, 2), (1920, 1080, 3), (1920, 1080, 4), (1920, 1080, 5),
                                   (3840, 2160, 2), (3840, 2160, 3), (3840, 2160, 4), (3840, 2160, 5),
                                   (8192, 4096, 3), (8000, 300, 4), (300, 4000, 3)])
def test_mt_count_full_frames_matches_cut_partitions(trs, W, H, n):
    """At full frame sizes (and the largest, 64 x 32 CTUs) the library's
    count equals the recursive full-cut enumeration plus the pinwheels,
    which is the whole space up to five slices."""
    import bruteforce
    assert trs.trs_mt_count(W, H, n) == len(bruteforce.cut_partitions(W, H, n))


def _mt_sets(arr):
    """trs_mt_list records as a set of tuples of (y0, x0, y1, x1) slices."""
    return {tuple(tuple(int(v) for v in sl) for sl in rec) for rec in arr}


def _cut_sets(parts):
    """Brute-force partitions ((x0, x1, y0, y1) raster-sorted) as the same tuples."""
    return {tuple((r[2], r[0], r[3], r[1]) for r in p) for p in parts}


@pytest.mark.parametrize("W,H,n", [(832, 480, 4), (832, 480, 6), (640, 640, 8), (1280, 720, 6), (300, 200, 3),
                                   (8000, 300, 4), (1920, 1080, 5)])
def test_mt_list_order_and_validity(trs, W, H, n):
    """Records strictly increase (the tie order, no repeats), slices come in
    raster order, every set covers each CTU once, and the area rule holds."""
    import numpy as np
    arr = trs.trs_mt_list(W, H, n)
    assert len(arr) == trs.trs_mt_count(W, H, n)
    flat = arr.reshape(len(arr), -1).astype(np.int16)
    d = flat[1:] - flat[:-1]
    first = np.argmax(d != 0, axis=1)
    assert (d[np.arange(len(d)), first] > 0).all()
    C, R = -(-W // 128), -(-H // 128)
    px = lambda v, ext: min(v * 128, ext)
    for rec in arr:
        cover = np.zeros((R, C), np.int8)
        areas = []
        for y0, x0, y1, x1 in rec.tolist():
            assert 0 <= y0 < y1 <= R and 0 <= x0 < x1 <= C
            cover[y0:y1, x0:x1] += 1
            areas.append((px(x1, W) - px(x0, W)) * (px(y1, H) - px(y0, H)))
        assert (cover == 1).all()
        assert 3 * min(areas) > max(areas)
        starts = [(int(s[0]), int(s[1])) for s in rec]
        assert starts == sorted(starts) and len(set(starts)) == n


@pytest.mark.parametrize("W,H,n", [(384, 384, 3), (512, 384, 4), (640, 384, 5), (512, 512, 5), (512, 384, 6),
                                   (300, 200, 3), (128, 384, 2)])
def test_mt_list_equals_bruteforce(trs, W, H, n):
    import bruteforce
    assert _mt_sets(trs.trs_mt_list(W, H, n)) == _cut_sets(bruteforce.mt_partitions(W, H, n))


@pytest.mark.parametrize("W,H,n", [(1920, 1080, 3), (1920, 1080, 4), (1920, 1080, 5), (3840, 2160, 4),
                                   (3840, 2160, 5), (8192, 4096, 3)])
def test_mt_list_full_frames_equals_cut_partitions(trs, W, H, n):
    """Full frame sizes: the very same slice sets as full cuts plus pinwheels."""
    import bruteforce
    assert _mt_sets(trs.trs_mt_list(W, H, n)) == _cut_sets(bruteforce.cut_partitions(W, H, n))


def test_mt_list_capacity(trs):
    import ctypes
    import numpy as np
    lib = trs.lib()
    c = ctypes.c_int64(-1)
    assert lib.trs_mt_list(832, 480, 4, 3, None, 0, ctypes.byref(c)) == trs.OK and c.value == 106
    buf = np.zeros(106 * 16 - 1, np.uint8)
    c = ctypes.c_int64(-1)
    assert lib.trs_mt_list(832, 480, 4, 3, buf.ctypes.data, buf.nbytes, ctypes.byref(c)) == trs.EINVAL
    assert c.value == 106 and not buf.any()
    assert lib.trs_mt_list(832, 480, 4, 3, None, 0, None) == trs.EINVAL


@pytest.mark.parametrize("W,H,n,k,step", [(832, 480, 4, 3, 1), (1920, 1080, 8, 3, 1), (3840, 2160, 16, 3, 1),
                                          (3840, 2160, 16, 3, 4), (3840, 2160, 16, 3, 8), (8192, 4096, 32, 3, 1),
                                          (1920, 1080, 8, 2, 1), (1920, 1080, 12, 4, 1), (3840, 2160, 4, 3, 1),
                                          (129, 257, 2, 3, 1), (128, 128, 1, 3, 1)])
def test_plan_loses_no_partition(trs, W, H, n, k, step):
    """Every one-tile-row partition whose slice areas fit a window of the
    plan can be formed from the plan's units in that window (the pruning by
    area bounds, tiling bounds and slice-count reachability drops only
    options no partition uses)."""
    windows, short, in_windows = trs.trs_plan_coverage(W, H, n, k, step)
    assert short == 0
    if step == 1:  # and no window is missing: every partition's smallest area is one
        assert windows == trs.trs_plan_stats(W, H, n, k)[0]
        assert in_windows == trs.trs_count_partitions(W, H, n, k)


def test_plan_loses_no_partition_random_shapes(trs):
    import numpy as np
    rng = np.random.default_rng(2012)
    for _ in range(60):
        W, H = int(rng.integers(1, 8193)), int(rng.integers(1, 4097))
        C, R = -(-W // 128), -(-H // 128)
        n = int(rng.integers(1, min(32, C * R) + 1))
        k, step = int(rng.integers(2, 5)), int(rng.integers(1, 5))
        windows, short, in_windows = trs.trs_plan_coverage(W, H, n, k, step)
        assert short == 0, (W, H, n)
        if step == 1:
            assert in_windows == trs.trs_count_partitions(W, H, n, k), (W, H, n, k)


C_CLIENT = r"""
#include <stdio.h>
#include <stddef.h>
#include "trs.h"

#define CHECK_SIZE(T) do { if (trs_sizeof(#T) != sizeof(T)) { \
    printf("size mismatch %s: C %zu, library %zu\n", #T, sizeof(T), trs_sizeof(#T)); return 1; } } while (0)

int main(void) {
    double parts = 0.0;
    int64_t sets = -1;
    int nw = 0, ni = 0;
    CHECK_SIZE(trs_opts);
    CHECK_SIZE(trs_ctu_stats);
    CHECK_SIZE(trs_tables_layout);
    CHECK_SIZE(trs_partition);
    CHECK_SIZE(trs_frame_desc);
    CHECK_SIZE(trs_mt_partition);
    CHECK_SIZE(trs_tune_report);
    CHECK_SIZE(trs_server_opts);
    CHECK_SIZE(trs_decision);
    CHECK_SIZE(trs_server_stats);
    if (trs_version() != 1) return 2;
    if (trs_count_partitions(832, 480, 4, 3, &parts) != TRS_OK) return 3;
    if (trs_mt_count(832, 480, 4, 3, &sets) != TRS_OK) return 4;
    if (trs_plan_stats(3840, 2160, 16, 3, &nw, &ni) != TRS_OK) return 5;
    if (trs_create(NULL, NULL) != TRS_EINVAL) return 6;
    printf("%.0f %lld %d %d %s\n", parts, (long long)sets, nw, ni, trs_strerror(TRS_EINFEASIBLE));
    return 0;
}
"""


def test_header_is_plain_c_and_links(trs, tmp_path):
    """include/trs.h compiles as strict C99, links against the library, and
    the C compiler lays out every structure as the library does."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2012_14792_gb300 import build
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(build.LIB)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(root, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-ltrs", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    parts, sets, nw, ni = r.stdout.split()[:4]
    assert float(parts) == trs.trs_count_partitions(832, 480, 4)
    assert int(sets) == trs.trs_mt_count(832, 480, 4)
    assert (int(nw), int(ni)) == trs.trs_plan_stats(3840, 2160, 16)


@pytest.mark.parametrize("W,H,n,k", [(1, 511, 2, 3), (1, 512, 2, 3), (1, 255, 1, 2), (255, 1, 1, 2),
                                     (1, 383, 1, 3), (129, 511, 3, 3)])
def test_area_rule_boundary_shapes(trs, W, H, n, k):
    """Shapes with a slice area of exactly k*A_min - 1, the largest the rule
    admits (Sec. 2.3): 1x511 splits into 128 over 383 = 3*128 - 1 rows of
    pixels; at k = 2 the 1x255 frame is one slice of 255 = 2*128 - 1 samples,
    the area just above 128.  Counts equal the brute force's, the plan forms
    every partition of each window, and no window is missing."""
    expect = _brute_partitions(W, H, n, k)
    assert trs.trs_count_partitions(W, H, n, k) == expect
    _, short, in_windows = trs.trs_plan_coverage(W, H, n, k, 1)
    assert short == 0 and in_windows == expect


@pytest.mark.parametrize("W,H", [(1, 1), (128, 128), (129, 257), (832, 480), (1920, 1080), (3840, 2160),
                                 (8192, 4096), (8192, 1), (1, 4096)])
def test_tables_layout_holds_every_documented_array(trs, W, H):
    """Each array of the region tables starts on a 256-byte boundary, in the
    documented order, with room for its documented element count, and the
    total covers the last one; the band index formula enumerates every band
    [x0, x1) once."""
    lay = trs.trs_tables_layout_get(W, H)
    C, R = -(-W // 128), -(-H // 128)
    assert (lay.width, lay.height, lay.cols, lay.rows, lay.bands) == (W, H, C, R, C * (C + 1) // 2)
    arrays = [("off_tq", R * C * 4), ("off_sat_s1", (R + 1) * (C + 1) * 8), ("off_sat_s2", (R + 1) * (C + 1) * 8),
              ("off_sat_t", (R + 1) * (C + 1) * 8), ("off_rect_t", lay.bands * R * R * 8),
              ("off_rect_q", lay.bands * R * R * 8), ("off_status", 16)]
    end = 0
    for name, size in arrays:
        off = getattr(lay, name)
        assert off % 256 == 0 and off >= end, name
        end = off + size
    assert lay.bytes >= end and lay.bytes % 256 == 0
    bands = sorted(x0 * (2 * C - x0 + 1) // 2 + (x1 - x0 - 1) for x0 in range(C) for x1 in range(x0 + 1, C + 1))
    assert bands == list(range(lay.bands))


def test_tables_layout_rejects_bad_shapes(trs):
    for W, H in [(0, 10), (10, 0), (8193, 10), (10, 4097)]:
        with pytest.raises(trs.TrsError) as e:
            trs.trs_tables_layout_get(W, H)
        assert e.value.status == trs.EINVAL


def test_missing_library_fails_loudly(tmp_path):
    """Without libtrs.so the binding (and the runtime helper above it)
    refuses to import: there is no CPU fallback."""
    import subprocess
    import sys
    code = (f"import sys; sys.path.insert(0, {ROOT!r})\n"
            "import paper_2012_14792_gb300.build as B\n"
            f"B.LIB = {str(tmp_path / 'absent' / 'libtrs.so')!r}\n"
            "import importlib\n"
            "for mod in ('paper_2012_14792_gb300.trs', 'paper_2012_14792_gb300.runtime'):\n"
            "    try:\n"
            "        importlib.import_module(mod)\n"
            "    except ImportError as e:\n"
            "        assert 'not built' in str(e), e\n"
            "    else:\n"
            "        raise SystemExit(mod + ' imported without the library')\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr


def test_package_never_reaches_the_oracle():
    """No module of the package imports the oracle or names its library."""
    import ast
    pkg = os.path.join(ROOT, "paper_2012_14792_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                tree = ast.parse(open(path).read())
                for node in ast.walk(tree):
                    names = []
                    if isinstance(node, ast.Import):
                        names = [a.name for a in node.names]
                    elif isinstance(node, ast.ImportFrom):
                        names = [node.module or ""]
                    assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (path, names)
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(path).read()
                assert "liboracle" not in text and "trs_oracle" not in text, path


def test_oracle_never_reaches_the_package():
    """The oracle shares no code with the CUDA path: its modules import
    nothing of the package and its C source includes none of the library's
    headers."""
    import ast
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        path = os.path.join(odir, f)
        if f.endswith(".py"):
            for node in ast.walk(ast.parse(open(path).read())):
                if isinstance(node, (ast.Import, ast.ImportFrom)):
                    names = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
                    assert not any(n.startswith("paper_2012_14792_gb300") for n in names), (path, names)
        if f.endswith((".c", ".h")):
            includes = re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(path).read())
            assert not any(i.startswith("trs") or "csrc" in i or i.endswith(".cuh") for i in includes), (path, includes)


def test_every_exported_entry_point_is_declared(trs):
    """No undocumented C entry point: each exported trs_* symbol of the
    library is declared in include/trs.h."""
    import shutil
    import subprocess
    if shutil.which("nm") is None:
        pytest.skip("no nm")
    from paper_2012_14792_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-1].startswith("trs_")}
    assert exported and exported <= set(declared_functions()), sorted(exported - set(declared_functions()))
