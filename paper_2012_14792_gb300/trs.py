"""Python binding of the C ABI in include/trs.h (argument marshalling only).

Every function here has the name of the C entry point it calls and only
converts arguments: torch tensors become device pointers, the current torch
stream becomes the cudaStream_t, ctypes structures mirror the C ones.  All of
the computation runs in libtrs.so's CUDA kernels; if the library is missing
the import fails loudly (there is no fallback).
"""

from __future__ import annotations

import ctypes as ct
import os

from . import build as _build

CTU = 128
MAX_COLS = 64
MAX_ROWS = 32
MAX_REGIONS = 32
PACKED10 = 0x10A  # TRS_PACKED10: 10-bit samples packed four in five bytes

OK, EINVAL, ERANGE, EINFEASIBLE, ENOMEM, EBUSY, ETIMEOUT, ECUDA = range(8)


class TrsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.trs_strerror(status).decode()
        last = _lib.trs_last_error().decode()
        super().__init__(f"{where}: {msg}" + (f" ({last})" if status == ECUDA and last else ""))


class trs_opts(ct.Structure):
    _fields_ = [("max_width", ct.c_int), ("max_height", ct.c_int), ("max_regions", ct.c_int),
                ("max_batch", ct.c_int), ("k_area", ct.c_int), ("device", ct.c_int)]


class trs_ctu_stats(ct.Structure):
    _fields_ = [("s1", ct.c_void_p), ("s2", ct.c_void_p), ("count", ct.c_void_p), ("vmax", ct.c_void_p),
                ("flags", ct.c_void_p)]


class trs_tables_layout(ct.Structure):
    _fields_ = [("width", ct.c_int), ("height", ct.c_int), ("cols", ct.c_int), ("rows", ct.c_int),
                ("bands", ct.c_int), ("reserved", ct.c_int), ("bytes", ct.c_size_t), ("off_tq", ct.c_size_t),
                ("off_sat_s1", ct.c_size_t), ("off_sat_s2", ct.c_size_t), ("off_sat_t", ct.c_size_t),
                ("off_rect_t", ct.c_size_t), ("off_rect_q", ct.c_size_t), ("off_status", ct.c_size_t)]


class trs_partition(ct.Structure):
    _fields_ = [("status", ct.c_int32), ("n_regions", ct.c_int32), ("cols", ct.c_int32), ("rows", ct.c_int32),
                ("n_tile_cols", ct.c_int32), ("n_tile_rows", ct.c_int32), ("n_windows", ct.c_int32),
                ("reserved", ct.c_int32), ("t_min_q", ct.c_uint64), ("thr_q", ct.c_uint64), ("t_q", ct.c_uint64),
                ("q", ct.c_uint64), ("t_min", ct.c_double), ("t", ct.c_double), ("sse", ct.c_double),
                ("tile_row_mask", ct.c_uint64), ("col_bd", ct.c_int16 * (MAX_COLS + 1)),
                ("row_bd", ct.c_int16 * (MAX_ROWS + 1)), ("slice_cuts", ct.c_uint32 * MAX_COLS),
                ("region", (ct.c_int16 * 4) * MAX_REGIONS), ("tile_slices", ct.c_uint8 * MAX_REGIONS)]

    def x_edges(self) -> list[int]:
        return [int(self.col_bd[i]) for i in range(self.n_tile_cols + 1)]

    def band_cuts(self) -> list[int]:
        return [int(self.slice_cuts[i]) for i in range(self.n_tile_cols)]

    def regions(self) -> list[tuple[int, int, int, int]]:
        """Slices as (x0, x1, y0, y1) in CTU units."""
        return [(int(r[0]), int(r[2]), int(r[1]), int(r[3])) for r in self.region[: self.n_regions]]


class trs_frame_desc(ct.Structure):
    _fields_ = [("luma_dev", ct.c_void_p), ("ctu_time_dev", ct.c_void_p), ("width", ct.c_int),
                ("height", ct.c_int), ("pitch_bytes", ct.c_size_t), ("bit_depth", ct.c_int),
                ("n_regions", ct.c_int), ("lambda", ct.c_float)]


class trs_server_opts(ct.Structure):
    _fields_ = [("max_width", ct.c_int), ("max_height", ct.c_int), ("max_regions", ct.c_int),
                ("max_streams", ct.c_int), ("max_batch", ct.c_int), ("max_inflight", ct.c_int),
                ("mem_budget_bytes", ct.c_size_t), ("k_area", ct.c_int), ("device", ct.c_int)]


class trs_decision(ct.Structure):
    _fields_ = [("ticket", ct.c_uint64), ("tag", ct.c_uint64), ("stream_id", ct.c_int32), ("status", ct.c_int32),
                ("latency_us", ct.c_double), ("partition", trs_partition)]


class trs_server_stats(ct.Structure):
    _fields_ = [("batches", ct.c_uint64), ("frames", ct.c_uint64), ("decided", ct.c_uint64),
                ("mem_used_bytes", ct.c_size_t), ("streams_open", ct.c_int), ("pending", ct.c_int),
                ("inflight", ct.c_int), ("status", ct.c_int)]


class trs_tune_report(ct.Structure):
    _fields_ = [("band_warps", ct.c_int), ("col_warps", ct.c_int), ("col_batch", ct.c_int),
                ("n_candidates", ct.c_int), ("cand_band_warps", ct.c_int * 6), ("cand_col_warps", ct.c_int * 6),
                ("cand_col_batch", ct.c_int * 6), ("rows_ms", ct.c_float * 6), ("cols_ms", ct.c_float * 6)]

    def as_dict(self) -> dict:
        return {"band_warps": self.band_warps, "col_warps": self.col_warps, "col_batch": self.col_batch,
                "candidates": [{"band_warps": self.cand_band_warps[j], "col_warps": self.cand_col_warps[j],
                                "col_batch": self.cand_col_batch[j], "rows_ms": round(self.rows_ms[j], 4),
                                "cols_ms": round(self.cols_ms[j], 4)} for j in range(self.n_candidates)]}


PARTITION_BYTES = ct.sizeof(trs_partition)


class trs_mt_partition(ct.Structure):
    _fields_ = [("status", ct.c_int32), ("n_regions", ct.c_int32), ("candidates", ct.c_int64),
                ("winner", ct.c_int64), ("t_min_q", ct.c_uint64), ("thr_q", ct.c_uint64), ("t_q", ct.c_uint64),
                ("q", ct.c_uint64), ("t_min", ct.c_double), ("t", ct.c_double), ("sse", ct.c_double),
                ("region", (ct.c_int16 * 4) * MAX_REGIONS)]

    def regions(self) -> list[tuple[int, int, int, int]]:
        """Slices as (x0, x1, y0, y1) in CTUs, as trs_partition.regions(), in
        raster order of their top-left corners."""
        return [(int(r[0]), int(r[2]), int(r[1]), int(r[3])) for r in self.region[: self.n_regions]]


MT_PARTITION_BYTES = ct.sizeof(trs_mt_partition)


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libtrs.so is not built ({path}); run __graft_entry__.build() or "
                          "python -m paper_2012_14792_gb300.build")
    lib = ct.CDLL(path)
    vp, i, sz, f = ct.c_void_p, ct.c_int, ct.c_size_t, ct.c_float
    sig = {
        "trs_version": ([], i),
        "trs_strerror": ([i], ct.c_char_p),
        "trs_last_error": ([], ct.c_char_p),
        "trs_sizeof": ([ct.c_char_p], sz),
        "trs_plan_stats": ([i, i, i, i, ct.POINTER(i), ct.POINTER(i)], i),
        "trs_plan_work": ([i, i, i, i, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)], i),
        "trs_count_partitions": ([i, i, i, i, ct.POINTER(ct.c_double)], i),
        "trs_plan_coverage": ([i, i, i, i, i, ct.POINTER(i), ct.POINTER(i), ct.POINTER(ct.c_double)], i),
        "trs_mt_count": ([i, i, i, i, ct.POINTER(ct.c_int64)], i),
        "trs_mt_list": ([i, i, i, i, vp, sz, ct.POINTER(ct.c_int64)], i),
        "trs_alu_peak": ([i, ct.POINTER(ct.c_double)], i),
        "trs_create": ([ct.POINTER(vp), ct.POINTER(trs_opts)], i),
        "trs_destroy": ([vp], i),
        "trs_ctx_bytes": ([vp], sz),
        "trs_texture_map": ([vp, vp, i, i, sz, i, ct.POINTER(trs_ctu_stats), vp], i),
        "trs_tables_layout_get": ([i, i, ct.POINTER(trs_tables_layout)], i),
        "trs_region_tables": ([vp, ct.POINTER(trs_ctu_stats), vp, i, i, vp, sz, vp], i),
        "trs_search": ([vp, vp, i, i, i, f, vp, vp], i),
        "trs_search_noalloc": ([vp, i, i, i, i, f, vp, vp], i),
        "trs_search_mt": ([vp, vp, i, i, i, f, vp, vp], i),
        "trs_search_lambdas": ([vp, vp, i, i, i, ct.POINTER(ct.c_float), i, vp, vp], i),
        "trs_decide": ([vp, vp, i, i, sz, i, vp, i, f, vp, vp], i),
        "trs_decide_host": ([vp, vp, i, i, sz, i, vp, i, f, ct.POINTER(trs_partition), vp], i),
        "trs_batch_decide": ([vp, ct.POINTER(trs_frame_desc), i, vp, vp], i),
        "trs_batch_decide_host": ([vp, ct.POINTER(trs_frame_desc), i, ct.POINTER(trs_partition), vp], i),
        "trs_batch_stage_ms": ([vp, ct.POINTER(ct.c_float), i], i),
        "trs_batch_stage_frames": ([vp], i),
        "trs_batch_kernels": ([vp], i),
        "trs_set_batch_parts": ([vp, i], i),
        "trs_autotune": ([vp, ct.POINTER(trs_frame_desc), i, ct.POINTER(trs_tune_report), vp], i),
        "trs_set_tune": ([vp, i, i, i], i),
        "trs_set_window_step": ([vp, i], i),
        "trs_server_create": ([ct.POINTER(vp), ct.POINTER(trs_server_opts)], i),
        "trs_server_destroy": ([vp], i),
        "trs_server_open_stream": ([vp, i, i, i, i, f, ct.POINTER(i)], i),
        "trs_server_close_stream": ([vp, i], i),
        "trs_server_update_times": ([vp, i, vp], i),
        "trs_server_submit": ([vp, i, vp, sz, ct.c_uint64, ct.POINTER(ct.c_uint64)], i),
        "trs_server_poll": ([vp, ct.POINTER(trs_decision), i, i, ct.POINTER(i)], i),
        "trs_server_info": ([vp, ct.POINTER(trs_server_stats)], i),
        "trs_server_open_stream_layers": ([vp, i, i, i, i, f, i, ct.POINTER(i)], i),
        "trs_server_update_times_layer": ([vp, i, i, vp], i),
        "trs_server_submit_layer": ([vp, i, i, vp, sz, ct.c_uint64, ct.POINTER(ct.c_uint64)], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def lib():
    return _lib


def _ptr(x) -> int:
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return int(x)


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _check(status: int, where: str) -> None:
    if status != OK:
        raise TrsError(status, where)


def trs_version() -> int:
    return _lib.trs_version()


def trs_strerror(status: int) -> str:
    return _lib.trs_strerror(status).decode()


def trs_sizeof(name: str) -> int:
    return _lib.trs_sizeof(name.encode())


def trs_plan_stats(width: int, height: int, n_regions: int, k_area: int = 3) -> tuple[int, int]:
    nw, ni = ct.c_int(0), ct.c_int(0)
    _check(_lib.trs_plan_stats(width, height, n_regions, k_area, ct.byref(nw), ct.byref(ni)), "trs_plan_stats")
    return nw.value, ni.value


def trs_count_partitions(width: int, height: int, n_regions: int, k_area: int = 3) -> float:
    c = ct.c_double()
    _check(_lib.trs_count_partitions(width, height, n_regions, k_area, ct.byref(c)), "trs_count_partitions")
    return c.value


def trs_plan_coverage(width: int, height: int, n_regions: int, k_area: int = 3,
                      window_step: int = 1) -> tuple[int, int, float]:
    """(windows checked, windows whose plan misses a partition of the window,
    partitions whose smallest slice area is a window of the plan)."""
    nw, bad, inw = ct.c_int(0), ct.c_int(0), ct.c_double(0)
    _check(_lib.trs_plan_coverage(width, height, n_regions, k_area, window_step, ct.byref(nw), ct.byref(bad),
                                  ct.byref(inw)), "trs_plan_coverage")
    return nw.value, bad.value, inw.value


def trs_plan_work(width: int, height: int, n_regions: int, k_area: int = 3) -> tuple[float, float]:
    r, c = ct.c_double(0), ct.c_double(0)
    _check(_lib.trs_plan_work(width, height, n_regions, k_area, ct.byref(r), ct.byref(c)), "trs_plan_work")
    return r.value, c.value


def trs_alu_peak(device: int = 0) -> float:
    v = ct.c_double(0)
    _check(_lib.trs_alu_peak(device, ct.byref(v)), "trs_alu_peak")
    return v.value


def trs_create(max_width: int, max_height: int, max_regions: int = 16, max_batch: int = 1,
               k_area: int = 3, device: int = 0) -> int:
    o = trs_opts(max_width, max_height, max_regions, max_batch, k_area, device)
    h = ct.c_void_p()
    _check(_lib.trs_create(ct.byref(h), ct.byref(o)), "trs_create")
    return h.value


def trs_destroy(ctx: int) -> None:
    _check(_lib.trs_destroy(ctx), "trs_destroy")


def trs_ctx_bytes(ctx: int) -> int:
    return _lib.trs_ctx_bytes(ctx)


def make_stats(s1, s2, count, vmax, flags) -> trs_ctu_stats:
    return trs_ctu_stats(_ptr(s1), _ptr(s2), _ptr(count), _ptr(vmax), _ptr(flags))


def trs_texture_map(ctx, luma, width, height, pitch_bytes, bit_depth, stats: trs_ctu_stats, stream=None) -> None:
    _check(_lib.trs_texture_map(ctx, _ptr(luma), width, height, pitch_bytes, bit_depth, ct.byref(stats),
                                _stream(stream)), "trs_texture_map")


def trs_tables_layout_get(width: int, height: int) -> trs_tables_layout:
    out = trs_tables_layout()
    _check(_lib.trs_tables_layout_get(width, height, ct.byref(out)), "trs_tables_layout_get")
    return out


def trs_region_tables(ctx, stats: trs_ctu_stats, ctu_time, width, height, tables, tables_bytes,
                      stream=None) -> None:
    _check(_lib.trs_region_tables(ctx, ct.byref(stats), _ptr(ctu_time), width, height, _ptr(tables),
                                  tables_bytes, _stream(stream)), "trs_region_tables")


def trs_search(ctx, tables, width, height, n_regions, lam, out, stream=None) -> None:
    _check(_lib.trs_search(ctx, _ptr(tables), width, height, n_regions, lam, _ptr(out), _stream(stream)),
           "trs_search")


def trs_search_lambdas(ctx, tables, width, height, n_regions, lambdas, out, stream=None) -> None:
    arr = (ct.c_float * len(lambdas))(*lambdas)
    _check(_lib.trs_search_lambdas(ctx, _ptr(tables), width, height, n_regions, arr, len(lambdas), _ptr(out),
                                   _stream(stream)), "trs_search_lambdas")


def trs_mt_count(width: int, height: int, n_regions: int, k_area: int = 3) -> int:
    c = ct.c_int64()
    _check(_lib.trs_mt_count(width, height, n_regions, k_area, ct.byref(c)), "trs_mt_count")
    return c.value


def trs_mt_list(width: int, height: int, n_regions: int, k_area: int = 3):
    """The slice-set list of the multi-tile space as a uint8 array of shape
    [count, n_regions, 4] (y0, x0, y1, x1 per slice), in tie order."""
    import numpy as np
    c = ct.c_int64()
    _check(_lib.trs_mt_list(width, height, n_regions, k_area, None, 0, ct.byref(c)), "trs_mt_list")
    out = np.zeros((c.value, n_regions, 4), np.uint8)
    _check(_lib.trs_mt_list(width, height, n_regions, k_area, out.ctypes.data, out.nbytes, ct.byref(c)),
           "trs_mt_list")
    return out


def trs_search_mt(ctx, tables, width, height, n_regions, lam, out, stream=None) -> None:
    _check(_lib.trs_search_mt(ctx, _ptr(tables), width, height, n_regions, lam, _ptr(out), _stream(stream)),
           "trs_search_mt")


def trs_search_noalloc(tables, width, height, n_regions, k_area, lam, out, stream=None) -> None:
    _check(_lib.trs_search_noalloc(_ptr(tables), width, height, n_regions, k_area, lam, _ptr(out),
                                   _stream(stream)), "trs_search_noalloc")


def trs_decide(ctx, luma, width, height, pitch_bytes, bit_depth, ctu_time, n_regions, lam, out,
               stream=None) -> None:
    _check(_lib.trs_decide(ctx, _ptr(luma), width, height, pitch_bytes, bit_depth, _ptr(ctu_time), n_regions,
                           lam, _ptr(out), _stream(stream)), "trs_decide")


def trs_decide_host(ctx, luma_host, width, height, pitch_bytes, bit_depth, ctu_time_host, n_regions, lam,
                    stream=None) -> trs_partition:
    out = trs_partition()
    _check(_lib.trs_decide_host(ctx, _ptr(luma_host), width, height, pitch_bytes, bit_depth,
                                _ptr(ctu_time_host), n_regions, lam, ct.byref(out), _stream(stream)),
           "trs_decide_host")
    return out


def frame_desc(luma, ctu_time, width, height, pitch_bytes, bit_depth, n_regions, lam) -> trs_frame_desc:
    return trs_frame_desc(_ptr(luma), _ptr(ctu_time), width, height, pitch_bytes, bit_depth, n_regions, lam)


def trs_batch_decide(ctx, descs: list[trs_frame_desc], out, stream=None) -> None:
    arr = (trs_frame_desc * len(descs))(*descs)
    _check(_lib.trs_batch_decide(ctx, arr, len(descs), _ptr(out), _stream(stream)), "trs_batch_decide")


def trs_batch_decide_host(ctx, descs: list[trs_frame_desc], stream=None) -> list[trs_partition]:
    """descs point at host memory; returns the partitions (synchronous)."""
    arr = (trs_frame_desc * len(descs))(*descs)
    out = (trs_partition * len(descs))()
    _check(_lib.trs_batch_decide_host(ctx, arr, len(descs), out, _stream(stream)), "trs_batch_decide_host")
    return list(out)


STAGES = ("texture", "tables", "step1_rows", "step1_columns", "step2_rows", "step2_columns", "rebuild", "decode")


def trs_batch_stage_frames(ctx) -> int:
    return _lib.trs_batch_stage_frames(ctx)


def trs_batch_kernels(ctx) -> int:
    return _lib.trs_batch_kernels(ctx)


def trs_set_batch_parts(ctx, parts: int) -> None:
    _check(_lib.trs_set_batch_parts(ctx, parts), "trs_set_batch_parts")


def trs_batch_stage_ms(ctx) -> dict:
    ms = (ct.c_float * len(STAGES))()
    k = _lib.trs_batch_stage_ms(ctx, ms, len(STAGES))
    return {STAGES[i]: float(ms[i]) for i in range(k)}


def trs_autotune(ctx, descs: list[trs_frame_desc], stream=None) -> trs_tune_report:
    arr = (trs_frame_desc * len(descs))(*descs)
    rep = trs_tune_report()
    _check(_lib.trs_autotune(ctx, arr, len(descs), ct.byref(rep), _stream(stream)), "trs_autotune")
    return rep


def trs_set_window_step(ctx, step: int) -> None:
    _check(_lib.trs_set_window_step(ctx, step), "trs_set_window_step")


def trs_set_tune(ctx, band_warps: int, col_warps: int, col_batch: int) -> None:
    _check(_lib.trs_set_tune(ctx, band_warps, col_warps, col_batch), "trs_set_tune")


def partitions_from_bytes(buf: bytes, count: int = 1) -> list[trs_partition]:
    return [trs_partition.from_buffer_copy(buf, i * PARTITION_BYTES) for i in range(count)]


# --- serving ---------------------------------------------------------------

def trs_server_create(max_width, max_height, max_regions=16, max_streams=32, max_batch=64, max_inflight=2,
                      mem_budget_bytes=0, k_area=3, device=0) -> int:
    o = trs_server_opts(max_width, max_height, max_regions, max_streams, max_batch, max_inflight,
                        mem_budget_bytes, k_area, device)
    h = ct.c_void_p()
    _check(_lib.trs_server_create(ct.byref(h), ct.byref(o)), "trs_server_create")
    return h.value


def trs_server_destroy(srv) -> None:
    _check(_lib.trs_server_destroy(srv), "trs_server_destroy")


def trs_server_open_stream(srv, width, height, bit_depth, n_regions, lam) -> int:
    sid = ct.c_int(-1)
    _check(_lib.trs_server_open_stream(srv, width, height, bit_depth, n_regions, lam, ct.byref(sid)),
           "trs_server_open_stream")
    return sid.value


def trs_server_close_stream(srv, sid) -> None:
    _check(_lib.trs_server_close_stream(srv, sid), "trs_server_close_stream")


def trs_server_update_times(srv, sid, times_host) -> None:
    _check(_lib.trs_server_update_times(srv, sid, _ptr(times_host)), "trs_server_update_times")


def trs_server_submit(srv, sid, luma_host, pitch_bytes, tag=0) -> int:
    """Returns the ticket; raises TrsError(EBUSY) when the stream's slots are taken."""
    t = ct.c_uint64(0)
    _check(_lib.trs_server_submit(srv, sid, _ptr(luma_host), pitch_bytes, tag, ct.byref(t)), "trs_server_submit")
    return t.value


def trs_server_poll(srv, max_out=64, timeout_us=1000) -> list:
    buf = (trs_decision * max_out)()
    n = ct.c_int(0)
    st = _lib.trs_server_poll(srv, buf, max_out, timeout_us, ct.byref(n))
    if st not in (OK, ETIMEOUT):
        raise TrsError(st, "trs_server_poll")
    return [buf[i] for i in range(n.value)]


def trs_server_info(srv) -> trs_server_stats:
    out = trs_server_stats()
    _check(_lib.trs_server_info(srv, ct.byref(out)), "trs_server_info")
    return out


def trs_server_open_stream_layers(srv, width, height, bit_depth, n_regions, lam, n_layers) -> int:
    sid = ct.c_int(-1)
    _check(_lib.trs_server_open_stream_layers(srv, width, height, bit_depth, n_regions, lam, n_layers,
                                              ct.byref(sid)), "trs_server_open_stream_layers")
    return sid.value


def trs_server_update_times_layer(srv, sid, layer, times_host) -> None:
    _check(_lib.trs_server_update_times_layer(srv, sid, layer, _ptr(times_host)), "trs_server_update_times_layer")


def trs_server_submit_layer(srv, sid, layer, luma_host, pitch_bytes, tag=0) -> int:
    t = ct.c_uint64(0)
    _check(_lib.trs_server_submit_layer(srv, sid, layer, _ptr(luma_host), pitch_bytes, tag, ct.byref(t)),
           "trs_server_submit_layer")
    return t.value
