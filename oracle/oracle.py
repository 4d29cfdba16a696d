"""Python access to the CPU oracle (``trs_oracle.c``).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.  The CUDA library never
does, and nothing here calls the library.

``build()`` compiles ``trs_oracle.c`` with gcc into ``oracle/_build``.
"""

from __future__ import annotations

import ctypes as ct
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

CTU = 128
OK, EINVAL, ERANGE, EINFEASIBLE, ENOMEM = 0, 1, 2, 3, 4
PACKED10 = 0x10A  # 10-bit samples packed four in five bytes (little-endian bit string per row)
_MAX_C = 64


class _Result(ct.Structure):
    _fields_ = [
        ("status", ct.c_int),
        ("n", ct.c_int),
        ("c", ct.c_int),
        ("r", ct.c_int),
        ("row_mask", ct.c_uint64),
        ("x_edges", ct.c_int * (_MAX_C + 1)),
        ("band_cuts", ct.c_uint64 * _MAX_C),
        ("t_min", ct.c_uint64),
        ("thr", ct.c_uint64),
        ("t", ct.c_uint64),
        ("q", ct.c_uint64),
        ("n_candidates", ct.c_uint64),
        ("n_valid", ct.c_uint64),
        ("n_windows", ct.c_uint64),
        ("t_real", ct.c_double),
        ("t_min_real", ct.c_double),
        ("sse_real", ct.c_double),
    ]


class _MtResult(ct.Structure):
    _fields_ = [
        ("status", ct.c_int),
        ("n", ct.c_int),
        ("t_min", ct.c_uint64),
        ("thr", ct.c_uint64),
        ("t", ct.c_uint64),
        ("q", ct.c_uint64),
        ("n_sets", ct.c_uint64),
        ("region", (ct.c_int16 * 4) * 64),
        ("sse_real", ct.c_double),
    ]


@dataclass
class Decision:
    status: int
    n: int = 0
    c: int = 0
    r: int = 0
    row_mask: int = 0
    x_edges: list = field(default_factory=list)
    band_cuts: list = field(default_factory=list)
    t_min: int = 0
    thr: int = 0
    t: int = 0
    q: int = 0
    n_candidates: int = 0
    n_valid: int = 0
    n_windows: int = 0
    t_real: float = 0.0
    t_min_real: float = 0.0
    sse_real: float = 0.0

    def regions(self, R: int) -> list[tuple[int, int, int, int]]:
        """Slices as (x0, x1, y0, y1) in CTU units, tile columns left to right,
        top to bottom inside each."""
        out = []
        for b in range(self.c):
            y0 = 0
            for y in range(1, R + 1):
                if y == R or (self.band_cuts[b] >> (y - 1)) & 1:
                    out.append((self.x_edges[b], self.x_edges[b + 1], y0, y))
                    y0 = y
        return out


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(build())
        u64p = ct.POINTER(ct.c_uint64)
        u32p = ct.POINTER(ct.c_uint32)
        _lib.oracle_texture.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_size_t, ct.c_int,
                                        u64p, u64p, u64p, u32p]
        _lib.oracle_time_q.argtypes = [ct.POINTER(ct.c_float), ct.c_int, u32p]
        _lib.oracle_lambda_q.argtypes = [ct.c_float]
        _lib.oracle_lambda_q.restype = ct.c_uint32
        _lib.oracle_sat.argtypes = [u64p, ct.c_int, ct.c_int, u64p]
        _lib.oracle_sat.restype = None
        sargs = [ct.c_int, ct.c_int, u64p, u64p, u64p, u32p, ct.c_int, ct.c_int, ct.c_uint32]
        _lib.oracle_search_enum.argtypes = sargs + [ct.c_int, ct.POINTER(_Result)]
        _lib.oracle_search_dp.argtypes = sargs + [ct.POINTER(_Result)]
        _lib.oracle_search_dp_windows.argtypes = sargs + [ct.c_int, ct.POINTER(_Result)]
        _lib.oracle_count_enum.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int, u64p]
        _lib.oracle_evaluate.argtypes = [ct.c_int, ct.c_int, u64p, u64p, u64p, u32p, ct.c_int,
                                         ct.POINTER(ct.c_int), u64p, u64p, u64p, u64p, u64p,
                                         ct.POINTER(ct.c_int)]
        _lib.oracle_rect.argtypes = [ct.c_int, ct.c_int, u64p, u64p, u64p, u32p, ct.c_int, ct.c_int, ct.c_int,
                                     ct.c_int, u64p, u64p]
        _lib.oracle_rect_all.argtypes = [ct.c_int, ct.c_int, u64p, u64p, u64p, u32p, u64p, u64p]
        _lib.oracle_result_size.restype = ct.c_size_t
        assert _lib.oracle_result_size() == ct.sizeof(_Result)
        _lib.oracle_mt_search.argtypes = [ct.c_int, ct.c_int, u64p, u64p, u64p, u32p, ct.c_int, ct.c_int,
                                          ct.c_uint32, ct.POINTER(_MtResult)]
        _lib.oracle_mt_count.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_int, u64p]
        _lib.oracle_mt_search_rects.argtypes = _lib.oracle_mt_search.argtypes
        _lib.oracle_mt_result_size.restype = ct.c_size_t
        assert _lib.oracle_mt_result_size() == ct.sizeof(_MtResult)
    return _lib


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ct.POINTER(ct.c_uint64))


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ct.POINTER(ct.c_uint32))


def grid(width: int, height: int) -> tuple[int, int]:
    return (width + CTU - 1) // CTU, (height + CTU - 1) // CTU


@dataclass
class Stats:
    width: int
    height: int
    S1: np.ndarray   # uint64 [R, C]
    S2: np.ndarray   # uint64 [R, C]
    N: np.ndarray    # uint64 [R, C]
    vmax: np.ndarray  # uint32 [R, C]
    status: int


def texture(plane: np.ndarray, bit_depth: int, pitch: int | None = None, width: int | None = None) -> Stats:
    """Per-CTU S1, S2, N and max sample of a luma plane [H, W] (uint8 or
    uint16), or, with bit_depth == PACKED10, of a packed plane given as
    uint8 rows [H, row bytes] holding `width` samples each."""
    H, W = plane.shape
    if bit_depth == PACKED10:
        W = width
    if pitch is None:
        buf = np.ascontiguousarray(plane)
        pitch = buf.strides[0]
    else:
        # a row-strided view: rows are read in place, `pitch` bytes apart
        if plane.strides[1] != plane.itemsize or plane.strides[0] != pitch:
            raise ValueError("plane strides do not match pitch")
        buf = plane
    C, R = grid(W, H)
    S1 = np.zeros((R, C), np.uint64)
    S2 = np.zeros((R, C), np.uint64)
    N = np.zeros((R, C), np.uint64)
    vmax = np.zeros((R, C), np.uint32)
    st = lib().oracle_texture(buf.ctypes.data, W, H, pitch, bit_depth, _p64(S1), _p64(S2), _p64(N), _p32(vmax))
    return Stats(W, H, S1, S2, N, vmax, st)


def time_q(times: np.ndarray) -> tuple[np.ndarray, int]:
    t = np.ascontiguousarray(times, dtype=np.float32)
    out = np.zeros(t.shape, np.uint32)
    st = lib().oracle_time_q(t.ctypes.data_as(ct.POINTER(ct.c_float)), t.size, _p32(out))
    return out, st


def lambda_q(lam: float) -> int:
    return int(lib().oracle_lambda_q(float(lam)))


def sat(v: np.ndarray) -> np.ndarray:
    R, C = v.shape
    a = np.ascontiguousarray(v, dtype=np.uint64)
    out = np.zeros((R + 1, C + 1), np.uint64)
    lib().oracle_sat(_p64(a), C, R, _p64(out))
    return out


def _decision(r: _Result) -> Decision:
    return Decision(
        status=r.status, n=r.n, c=r.c, r=r.r, row_mask=r.row_mask,
        x_edges=[r.x_edges[i] for i in range(r.c + 1)] if r.status == OK else [],
        band_cuts=[r.band_cuts[i] for i in range(r.c)] if r.status == OK else [],
        t_min=r.t_min, thr=r.thr, t=r.t, q=r.q, n_candidates=r.n_candidates,
        n_valid=r.n_valid, n_windows=r.n_windows, t_real=r.t_real,
        t_min_real=r.t_min_real, sse_real=r.sse_real)


def _search_args(st: Stats, Tq: np.ndarray):
    S1 = np.ascontiguousarray(st.S1, np.uint64)
    S2 = np.ascontiguousarray(st.S2, np.uint64)
    N = np.ascontiguousarray(st.N, np.uint64)
    T = np.ascontiguousarray(Tq, np.uint32)
    return (S1, S2, N, T)


def search_enum(st: Stats, Tq: np.ndarray, n: int, lam: float = 0.0, k_area: int = 3,
                area_rule: bool = True, lam_q: int | None = None) -> Decision:
    """O1: plain enumeration of every TRS configuration (small grids only)."""
    S1, S2, N, T = _search_args(st, Tq)
    lq = lambda_q(lam) if lam_q is None else lam_q
    r = _Result()
    lib().oracle_search_enum(st.width, st.height, _p64(S1), _p64(S2), _p64(N), _p32(T), n, k_area,
                             lq, 1 if area_rule else 0, ct.byref(r))
    return _decision(r)


def search_dp(st: Stats, Tq: np.ndarray, n: int, lam: float = 0.0, k_area: int = 3,
              lam_q: int | None = None) -> Decision:
    """O2: exact dynamic programme with the same result as O1."""
    S1, S2, N, T = _search_args(st, Tq)
    lq = lambda_q(lam) if lam_q is None else lam_q
    r = _Result()
    lib().oracle_search_dp(st.width, st.height, _p64(S1), _p64(S2), _p64(N), _p32(T), n, k_area,
                           lq, ct.byref(r))
    return _decision(r)


def search_dp_windows(st: Stats, Tq: np.ndarray, n: int, lam: float = 0.0, window_step: int = 1,
                      k_area: int = 3, lam_q: int | None = None) -> Decision:
    """O2 over every window_step-th area window (largest kept): the lightweight search."""
    S1, S2, N, T = _search_args(st, Tq)
    lq = lambda_q(lam) if lam_q is None else lam_q
    r = _Result()
    lib().oracle_search_dp_windows(st.width, st.height, _p64(S1), _p64(S2), _p64(N), _p32(T), n, k_area, lq,
                                   window_step, ct.byref(r))
    return _decision(r)


def count_enum(width: int, height: int, n: int, k_area: int = 3, area_rule: bool = True) -> int:
    out = np.zeros(1, np.uint64)
    st = lib().oracle_count_enum(width, height, n, k_area, 1 if area_rule else 0, _p64(out))
    if st != OK:
        raise ValueError(f"oracle_count_enum status {st}")
    return int(out[0])


def evaluate(st: Stats, Tq: np.ndarray, x_edges: list, band_cuts: list) -> dict:
    """Objective terms of a given partition by direct sums."""
    S1, S2, N, T = _search_args(st, Tq)
    c = len(band_cuts)
    xe = (ct.c_int * (c + 1))(*x_edges)
    bc = np.array(band_cuts, dtype=np.uint64)
    o = [np.zeros(1, np.uint64) for _ in range(4)]
    nreg = ct.c_int(0)
    s = lib().oracle_evaluate(st.width, st.height, _p64(S1), _p64(S2), _p64(N), _p32(T), c, xe,
                              _p64(bc), _p64(o[0]), _p64(o[1]), _p64(o[2]), _p64(o[3]), ct.byref(nreg))
    if s != OK:
        raise ValueError(f"oracle_evaluate status {s}")
    return dict(t=int(o[0][0]), q=int(o[1][0]), amin=int(o[2][0]), amax=int(o[3][0]), n=nreg.value)


def rect(st: Stats, Tq: np.ndarray, x0: int, x1: int, y0: int, y1: int) -> tuple[int, int]:
    """(time, floor SSE) of the CTU rectangle [x0,x1) x [y0,y1) by direct sums."""
    S1, S2, N, T = _search_args(st, Tq)
    t, q = np.zeros(1, np.uint64), np.zeros(1, np.uint64)
    s = lib().oracle_rect(st.width, st.height, _p64(S1), _p64(S2), _p64(N), _p32(T), x0, x1, y0, y1, _p64(t), _p64(q))
    if s != OK:
        raise ValueError(f"oracle_rect status {s}")
    return int(t[0]), int(q[0])


def rect_all(st: Stats, Tq: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(time, floor SSE) of every CTU rectangle by direct sums, as two uint64
    arrays indexed [x0, x1, y0, y1] (zero where x0 >= x1 or y0 >= y1)."""
    S1, S2, N, T = _search_args(st, Tq)
    R, C = st.S1.shape
    t = np.zeros((C + 1, C + 1, R + 1, R + 1), np.uint64)
    q = np.zeros_like(t)
    s = lib().oracle_rect_all(st.width, st.height, _p64(S1), _p64(S2), _p64(N), _p32(T), _p64(t), _p64(q))
    if s != OK:
        raise ValueError(f"oracle_rect_all status {s}")
    return t, q


def decide(plane: np.ndarray, times: np.ndarray, bit_depth: int, n: int, lam: float,
           k_area: int = 3, width: int | None = None) -> tuple[Decision, Stats, np.ndarray]:
    """Whole path on the CPU: texture, Q16 times, O2 search (width: the
    samples per row of a PACKED10 plane)."""
    st = texture(plane, bit_depth, width=width)
    Tq, s = time_q(times)
    if st.status != OK:
        return Decision(status=st.status), st, Tq
    if s != OK:
        return Decision(status=s), st, Tq
    return search_dp(st, Tq, n, lam, k_area), st, Tq


# --- multi-tile rectangular slices (enumerated; small frames only) ---

def mt_count(width: int, height: int, n: int, k_area: int = 3) -> int:
    """Distinct slice sets of the multi-tile space that pass the area rule."""
    out = np.zeros(1, np.uint64)
    st = lib().oracle_mt_count(width, height, n, k_area, _p64(out))
    if st != OK:
        raise ValueError(f"oracle_mt_count status {st}")
    return int(out[0])


def mt_search_rects(st: Stats, Tq: np.ndarray, n: int, lam: float = 0.0, k_area: int = 3) -> dict:
    """The multi-tile search over the partitions of the CTU grid into n
    rectangles (the same space as mt_search, enumerated directly; full frame
    sizes for small n).  Adds count = the number of slice sets."""
    S1, S2, N, T = _search_args(st, Tq)
    r = _MtResult()
    lib().oracle_mt_search_rects(st.width, st.height, _p64(S1), _p64(S2), _p64(N), _p32(T), n, k_area,
                                 lambda_q(lam), ct.byref(r))
    regions = [tuple(int(v) for v in r.region[i]) for i in range(n)] if r.status == OK else []
    return dict(status=r.status, t_min=r.t_min, thr=r.thr, t=r.t, q=r.q, regions=regions, sse=r.sse_real,
                count=int(r.n_sets))


def mt_search(st: Stats, Tq: np.ndarray, n: int, lam: float = 0.0, k_area: int = 3) -> dict:
    """The multi-tile search: T_min (Eq. 3), then the smallest (Q, raster-ordered
    slice list) under Eq. 4.  Regions are (x0, y0, x1, y1) in CTUs."""
    S1, S2, N, T = _search_args(st, Tq)
    r = _MtResult()
    lib().oracle_mt_search(st.width, st.height, _p64(S1), _p64(S2), _p64(N), _p32(T), n, k_area,
                           lambda_q(lam), ct.byref(r))
    regions = [tuple(int(v) for v in r.region[i]) for i in range(n)] if r.status == OK else []
    return dict(status=r.status, t_min=r.t_min, thr=r.thr, t=r.t, q=r.q, regions=regions, sse=r.sse_real)
