"""Torch-facing convenience layer over the binding: owns a context and the
device tensors the C calls write into.  Still marshalling only -- every
number is produced by libtrs.so's kernels."""

from __future__ import annotations

import numpy as np
import torch

from . import trs

CTU = trs.CTU


def grid(width: int, height: int) -> tuple[int, int]:
    return (width + CTU - 1) // CTU, (height + CTU - 1) // CTU


def luma_to_device(plane: np.ndarray, device="cuda") -> tuple[torch.Tensor, int]:
    """Uploads a [H, W] uint8/uint16 plane as raw bytes; returns (tensor, pitch)."""
    raw = np.ascontiguousarray(plane).view(np.uint8)
    t = torch.from_numpy(raw).to(device)
    return t, raw.strides[0]


class Decider:
    def __init__(self, max_width: int = 3840, max_height: int = 2160, max_regions: int = 16,
                 max_batch: int = 1, k_area: int = 3, device: int = 0):
        self.device = torch.device("cuda", device)
        self.ctx = trs.trs_create(max_width, max_height, max_regions, max_batch, k_area, device)

    def close(self):
        if self.ctx:
            trs.trs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- one frame, stage by stage ------------------------------------
    def stats_buffers(self, width: int, height: int) -> dict:
        C, R = grid(width, height)
        d = dict(s1=torch.zeros(R * C, dtype=torch.int32, device=self.device),
                 s2=torch.zeros(R * C, dtype=torch.int64, device=self.device),
                 count=torch.zeros(R * C, dtype=torch.int32, device=self.device),
                 vmax=torch.zeros(R * C, dtype=torch.int32, device=self.device),
                 flags=torch.zeros(4, dtype=torch.int32, device=self.device))
        d["abi"] = trs.make_stats(d["s1"], d["s2"], d["count"], d["vmax"], d["flags"])
        return d

    def texture_map(self, luma: torch.Tensor, width: int, height: int, pitch: int, bit_depth: int,
                    stats: dict) -> None:
        trs.trs_texture_map(self.ctx, luma, width, height, pitch, bit_depth, stats["abi"])

    def tables_buffer(self, width: int, height: int) -> torch.Tensor:
        lay = trs.trs_tables_layout_get(width, height)
        return torch.zeros(lay.bytes, dtype=torch.uint8, device=self.device)

    def region_tables(self, stats: dict, times: torch.Tensor, width: int, height: int,
                      tables: torch.Tensor) -> None:
        trs.trs_region_tables(self.ctx, stats["abi"], times, width, height, tables, tables.numel())

    def search(self, tables: torch.Tensor, width: int, height: int, n: int, lam: float) -> torch.Tensor:
        out = torch.zeros(trs.PARTITION_BYTES, dtype=torch.uint8, device=self.device)
        trs.trs_search(self.ctx, tables, width, height, n, lam, out)
        return out

    def search_mt(self, tables: torch.Tensor, width: int, height: int, n: int, lam: float):
        """Multi-tile rectangular slices (trs_search_mt); the record read back."""
        out = torch.zeros(trs.MT_PARTITION_BYTES, dtype=torch.uint8, device=self.device)
        trs.trs_search_mt(self.ctx, tables, width, height, n, lam, out)
        return trs.trs_mt_partition.from_buffer_copy(out.cpu().numpy().tobytes())

    def search_lambdas(self, tables: torch.Tensor, width: int, height: int, n: int, lams: list) -> torch.Tensor:
        out = torch.zeros(len(lams) * trs.PARTITION_BYTES, dtype=torch.uint8, device=self.device)
        trs.trs_search_lambdas(self.ctx, tables, width, height, n, list(lams), out)
        return out

    # ---- one frame, whole path ------------------------------------------
    def decide(self, luma: torch.Tensor, pitch: int, width: int, height: int, bit_depth: int,
               times: torch.Tensor, n: int, lam: float, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.zeros(trs.PARTITION_BYTES, dtype=torch.uint8, device=self.device)
        trs.trs_decide(self.ctx, luma, width, height, pitch, bit_depth, times, n, lam, out)
        return out

    def decide_host(self, plane: np.ndarray, times: np.ndarray, bit_depth: int, n: int,
                    lam: float, width: int | None = None) -> trs.trs_partition:
        """width: the samples per row of a TRS_PACKED10 plane (uint8 rows)."""
        p = np.ascontiguousarray(plane)
        t = np.ascontiguousarray(times, dtype=np.float32)
        H, W = p.shape
        if width is not None:
            W = width
        return trs.trs_decide_host(self.ctx, p, W, H, p.strides[0], bit_depth, t, n, lam)

    # ---- batched ----------------------------------------------------------
    def batch_decide(self, frames: list, out: torch.Tensor | None = None) -> torch.Tensor:
        """frames: list of (luma tensor, pitch, width, height, bit_depth, times tensor, n, lambda)."""
        descs = [trs.frame_desc(l, t, w, h, p, bd, n, lam) for (l, p, w, h, bd, t, n, lam) in frames]
        if out is None:
            out = torch.zeros(len(frames) * trs.PARTITION_BYTES, dtype=torch.uint8, device=self.device)
        trs.trs_batch_decide(self.ctx, descs, out)
        return out

    def autotune(self, frames: list) -> dict:
        """Picks the search kernels' launch shapes on this batch (see trs_autotune)."""
        descs = [trs.frame_desc(l, t, w, h, p, bd, n, lam) for (l, p, w, h, bd, t, n, lam) in frames]
        return trs.trs_autotune(self.ctx, descs).as_dict()

    # ---- reading results ----------------------------------------------------
    @staticmethod
    def partitions(out: torch.Tensor, count: int = 1) -> list:
        return trs.partitions_from_bytes(out.cpu().numpy().tobytes(), count)

    @staticmethod
    def read_tables(tables: torch.Tensor, width: int, height: int) -> dict:
        lay = trs.trs_tables_layout_get(width, height)
        raw = tables.cpu().numpy()
        C, R, nb = lay.cols, lay.rows, lay.bands

        def arr(off, dtype, count):
            return np.frombuffer(raw[off: off + count * np.dtype(dtype).itemsize].tobytes(), dtype=dtype)

        S = (R + 1) * (C + 1)
        return dict(
            tq=arr(lay.off_tq, np.uint32, R * C).reshape(R, C),
            sat_s1=arr(lay.off_sat_s1, np.uint64, S).reshape(R + 1, C + 1),
            sat_s2=arr(lay.off_sat_s2, np.uint64, S).reshape(R + 1, C + 1),
            sat_t=arr(lay.off_sat_t, np.uint64, S).reshape(R + 1, C + 1),
            rect_t=arr(lay.off_rect_t, np.uint64, nb * R * R).reshape(nb, R, R),
            rect_q=arr(lay.off_rect_q, np.uint64, nb * R * R).reshape(nb, R, R),
            status=arr(lay.off_status, np.int32, 4),
        )
