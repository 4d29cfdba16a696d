"""Host code under AddressSanitizer, UndefinedBehaviorSanitizer and
ThreadSanitizer.

compute-sanitizer is not available for the device side, so the host side is
checked this way instead:
  * the oracle: a copy of oracle/trs_oracle.c built with
    -fsanitize=address,undefined runs every oracle pin test in a child
    process (the sanitizer runtimes preloaded); any out-of-bounds access,
    use after free, signed overflow or bad shift aborts it.  A second copy
    with one planted off-by-one read must be stopped by AddressSanitizer,
    so a run without a live sanitizer cannot pass;
  * the library's host logic: plan.cu, mt.cu and api.cu rebuilt with the
    same flags (host code only; the device code is unchanged) and linked
    with the other objects of the normal build; the host-logic ABI tests
    run against that library (no GPU is touched);
  * the multi-tile list's enumeration on a pool of host threads: mt.cu
    rebuilt with ThreadSanitizer runs the full-frame enumeration tests
    without a race report, and a copy with one planted race must be
    reported.

Each builds into a temporary folder; the committed sources are read, never
changed."""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")
SAN_FLAGS = ["-fsanitize=address", "-fsanitize=undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
             "-g"]
ORACLE_PINS = ("test_oracle_texture.py", "test_oracle_tables.py", "test_oracle_search.py", "test_oracle_mt.py",
               "test_golden_mt.py")


def _starts(preload: str) -> bool:
    """Whether Python starts with these runtimes preloaded (a sanitizer
    runtime can refuse the process's memory layout on some kernels)."""
    r = subprocess.run([sys.executable, "-c", "pass"], capture_output=True, text=True, timeout=120,
                       env=dict(os.environ, LD_PRELOAD=preload, ASAN_OPTIONS="detect_leaks=0"))
    return r.returncode == 0


def _runtime(*names):
    """The gcc sanitizer runtimes `names` to preload (':'-joined), or None
    when gcc lacks them or they cannot start here."""
    if shutil.which("gcc") is None:
        return None
    libs = []
    for name in names:
        p = subprocess.run(["gcc", "-print-file-name=" + name], capture_output=True, text=True).stdout.strip()
        if not os.path.isabs(p) or not os.path.exists(p):
            return None
        libs.append(p)
    preload = ":".join(libs)
    return preload if _starts(preload) else None


def _runtimes():
    return _runtime("libasan.so", "libubsan.so")


def _child(code: str, cwd: str, preload: str):
    env = dict(os.environ, LD_PRELOAD=preload, ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1200, cwd=cwd,
                          env=env)


_ORACLE_DRIVER = r'''
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
from oracle import oracle as O
O._SRC, O._BUILD, O._LIB = {src!r}, {build!r}, {lib!r}
{body}
'''


def _sanitized_oracle(d, text):
    src = os.path.join(d, "trs_oracle.c")
    with open(src, "w") as f:
        f.write(text)
    lib = os.path.join(d, "liboracle.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-Wall", "-shared", "-fPIC", *SAN_FLAGS, "-o", lib, src, "-lm"])
    return src, lib


def test_oracle_pins_pass_under_asan_and_ubsan(tmp_path):
    preload = _runtimes()
    if preload is None:
        pytest.skip("no usable gcc sanitizer runtimes")
    with open(os.path.join(ROOT, "oracle", "trs_oracle.c")) as f:
        original = f.read()

    # the sanitizer is live: a planted read one word past the input of the
    # summed-area table (last row, last column) must be reported
    old = "for (int xx = 0; xx < x; ++xx) s += v[yy * C + xx];"
    assert original.count(old) == 1
    d = str(tmp_path / "planted")
    os.makedirs(d)
    src, lib = _sanitized_oracle(d, original.replace(old, old.replace("xx < x", "xx <= x")))
    body = "import numpy as np\nO.sat(np.arange(12, dtype=np.uint64).reshape(3, 4))\nprint('no report')"
    r = _child(_ORACLE_DRIVER.format(root=ROOT, tests=TESTS, src=src, build=d, lib=lib, body=body), d, preload)
    assert r.returncode != 0 and "AddressSanitizer" in r.stderr, r.stdout[-1000:] + r.stderr[-2000:]

    # the oracle as committed passes every pin with both sanitizers on
    d = str(tmp_path / "oracle")
    os.makedirs(d)
    src, lib = _sanitized_oracle(d, original)
    pins = [os.path.join(TESTS, p) for p in ORACLE_PINS]
    body = ("import pytest\nsys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', '-m', 'not gpu', "
            f"'--rootdir', {ROOT!r}] + {pins!r}))")
    r = _child(_ORACLE_DRIVER.format(root=ROOT, tests=TESTS, src=src, build=d, lib=lib, body=body), d, preload)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]


_ABI_DRIVER = r'''
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import paper_2012_14792_gb300.build as B
B.LIB = {lib!r}
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu", "--rootdir", {root!r},
                      "-k", {skip!r}, {abi!r}]))
'''

# host units whose logic the ABI tests drive without a GPU
HOST_UNITS = ("plan.cu", "mt.cu", "api.cu")


def test_library_host_logic_passes_under_asan_and_ubsan(tmp_path):
    preload = _runtimes()
    if preload is None:
        pytest.skip("no usable gcc sanitizer runtimes")
    sys.path.insert(0, ROOT)
    from paper_2012_14792_gb300 import build as B
    if shutil.which(B._nvcc()) is None and not os.path.exists(B._nvcc()):
        pytest.skip("no nvcc")
    B.build()
    host = [a for f in SAN_FLAGS for a in ("-Xcompiler", f)]

    def compile_unit(s):
        obj = str(tmp_path / (s[:-3] + ".o"))
        r = subprocess.run([B._nvcc(), *B.ARCH, *B.NVCC_FLAGS, *host, "-I", B.CSRC, "-c",
                            os.path.join(B.CSRC, s), "-o", obj], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(HOST_UNITS)) as ex:
        built = dict(zip(HOST_UNITS, ex.map(compile_unit, HOST_UNITS)))
    objs = [built.get(s, os.path.join(B.BUILD, s[:-3] + ".o")) for s in B.SOURCES]
    lib = str(tmp_path / "libtrs.so")
    r = subprocess.run([B._nvcc(), *B.ARCH, "-shared", "-o", lib, *objs], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    # the host-logic tests (plan windows and pruning, partition counts, plan
    # coverage, the multi-tile list); left out: linking a plain C program
    # against this library (it would need the sanitizer runtimes at link
    # time) and the 60-shape coverage sweep, which runs the same code as the
    # fixed shapes, only longer
    skip = ("(area_rule or count_partitions or plan_ or mt_) and not test_header_is_plain_c_and_links "
            "and not test_plan_loses_no_partition_random_shapes")
    code = _ABI_DRIVER.format(root=ROOT, tests=TESTS, lib=lib, skip=skip, abi=os.path.join(TESTS, "test_abi.py"))
    r = _child(code, str(tmp_path), preload)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]


def _sanitized_library(B, tmp_path, units, flags):
    """libtrs.so with `units` (name -> source text) compiled with the host
    flags `flags`, linked with the other objects of the normal build."""
    host = [a for f in flags for a in ("-Xcompiler", f)]

    def compile_unit(item):
        name, text = item
        src = tmp_path / name
        src.write_text(text)
        obj = str(tmp_path / (name[:-3] + ".o"))
        r = subprocess.run([B._nvcc(), *B.ARCH, *B.NVCC_FLAGS, *host, "-I", B.CSRC, "-c", str(src), "-o", obj],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        return name, obj

    with cf.ThreadPoolExecutor(max_workers=len(units)) as ex:
        built = dict(ex.map(compile_unit, units.items()))
    objs = [built.get(s, os.path.join(B.BUILD, s[:-3] + ".o")) for s in B.SOURCES]
    lib = str(tmp_path / "libtrs.so")
    r = subprocess.run([B._nvcc(), *B.ARCH, "-shared", "-o", lib, *objs], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return lib


def test_multitile_enumeration_threads_under_tsan(tmp_path):
    """The multi-tile list is enumerated on a pool of host threads (mt.cu).
    Rebuilt with ThreadSanitizer, the host-logic tests that enumerate full
    frames run without a race report; a copy with one planted race (every
    thread adding its count into one shared word) must be reported."""
    tsan = _runtime("libtsan.so")
    if tsan is None:
        pytest.skip("no usable gcc ThreadSanitizer runtime")
    sys.path.insert(0, ROOT)
    from paper_2012_14792_gb300 import build as B
    if shutil.which(B._nvcc()) is None and not os.path.exists(B._nvcc()):
        pytest.skip("no nvcc")
    B.build()
    with open(os.path.join(B.CSRC, "mt.cu")) as f:
        mt = f.read()
    flags = ["-fsanitize=thread", "-fno-omit-frame-pointer", "-g"]
    env = dict(os.environ, LD_PRELOAD=tsan, TSAN_OPTIONS="halt_on_error=1 report_signal_unsafe=0")

    def run(lib, select, d):
        # -s: a report is written while a test runs, and the process stops
        # there, so pytest must not be holding the output
        code = _ABI_DRIVER.format(root=ROOT, tests=TESTS, lib=lib, skip=select,
                                  abi=os.path.join(TESTS, "test_abi.py")).replace('"-x", "-q"', '"-x", "-q", "-s"')
        return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1200, cwd=d,
                              env=env)

    old = "wv[t] = e.visits;"
    assert mt.count(old) == 1
    d = tmp_path / "planted"
    d.mkdir()
    lib = _sanitized_library(B, d, {"mt.cu": mt.replace(old, "wv[0] += e.visits;")}, flags)
    r = run(lib, "mt_count_full_frames_matches_cut_partitions and 1920-1080-5", str(d))
    assert r.returncode != 0 and "ThreadSanitizer" in r.stdout + r.stderr, r.stdout[-1000:] + r.stderr[-2000:]

    d = tmp_path / "mt"
    d.mkdir()
    lib = _sanitized_library(B, d, {"mt.cu": mt}, flags)
    r = run(lib, "(mt_count_full_frames or mt_list_full_frames) and 1920", str(d))
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
