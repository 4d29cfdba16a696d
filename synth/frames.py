"""Seeded synthetic luma planes and per-CTU encoding-time maps.

Workload recipe (stand-in for the JVET common-test-condition sequences the
paper encodes in Sec. 3.1, which are not available here):

* The plane is tiled by 64x64 patches.  Each patch independently draws a kind:
  flat (40 %), Gaussian noise (40 %) or linear ramp (20 %).  Flat patches take
  a level U[16, 235]; noise patches add N(0, sigma^2) with sigma U[2, 40];
  ramps add slope * (dx*u + dy*v) with slope U[0.1, 2] per sample and a random
  unit direction (dx, dy).  All figures are in 8-bit units and are scaled by
  2^(bd-8) for deeper planes.  Samples are rounded half-to-even and clipped to
  [0, 2^bd - 1].
* Each patch carries a *latent complexity*: 0 for flat patches, sigma^2 for
  noise, slope^2 * (64^2 - 1) / 12 for ramps (the variance of the generating
  process, in 8-bit units).  It is a parameter of the generator, never a
  measurement of the plane.
* The encoding time of a CTU in the co-located previous frame is modelled as
  t = (0.5 + 0.02 * latent) * exp(eps), eps ~ N(0, 0.2^2), stored as float32.
  It stands for the co-TL frame times that Sec. 2.1 feeds to the estimator.
* The 2160p sequence adds a high-detail disk (radius 384 px, sigma 40 noise)
  that moves 32 px per frame; the time map of frame f is drawn from the
  latent complexity of frame f-1 (frame 0 uses its own).

Every draw comes from numpy's PCG64 seeded by a SeedSequence keyed on
(workload id, stream, frame), so inputs are reproducible.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

PATCH = 64
CTU = 128  # CTU grid pitch used to lay out the per-CTU time map


@dataclass(frozen=True)
class FrameSpec:
    name: str
    width: int
    height: int
    bit_depth: int

    @property
    def ctu_cols(self) -> int:
        return (self.width + CTU - 1) // CTU

    @property
    def ctu_rows(self) -> int:
        return (self.height + CTU - 1) // CTU

    @property
    def bytes_per_sample(self) -> int:
        return 1 if self.bit_depth == 8 else 2

    @property
    def frame_bytes(self) -> int:
        return self.width * self.height * self.bytes_per_sample


SPEC_480P8 = FrameSpec("832x480p8", 832, 480, 8)
SPEC_1080P10 = FrameSpec("1920x1080p10", 1920, 1080, 10)
SPEC_2160P10 = FrameSpec("3840x2160p10", 3840, 2160, 10)

_WORKLOAD_IDS = {"single": 1, "seq2160": 2, "mixed": 3, "serve": 4, "test": 5}


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(k) for k in key])))


def _patch_params(rng: np.random.Generator, ph: int, pw: int) -> dict:
    kind = rng.choice(3, size=(ph, pw), p=[0.4, 0.4, 0.2])
    level = rng.uniform(16.0, 235.0, size=(ph, pw))
    sigma = rng.uniform(2.0, 40.0, size=(ph, pw))
    slope = rng.uniform(0.1, 2.0, size=(ph, pw))
    dx = rng.uniform(-1.0, 1.0, size=(ph, pw))
    dy = rng.uniform(-1.0, 1.0, size=(ph, pw))
    norm = np.sqrt(dx * dx + dy * dy)
    norm[norm == 0.0] = 1.0
    return dict(kind=kind, level=level, sigma=sigma, slope=slope, dx=dx / norm, dy=dy / norm)


def _patch_latent(p: dict) -> np.ndarray:
    lat = np.zeros(p["kind"].shape, dtype=np.float64)
    lat = np.where(p["kind"] == 1, p["sigma"] ** 2, lat)
    lat = np.where(p["kind"] == 2, p["slope"] ** 2 * (PATCH * PATCH - 1) / 12.0, lat)
    return lat


def _render(p: dict, spec: FrameSpec, noise_rng: np.random.Generator,
            blob: tuple[float, float, float, float] | None) -> tuple[np.ndarray, np.ndarray]:
    """Returns (plane[H, W], per-pixel latent complexity[H, W] float32)."""
    ph, pw = p["kind"].shape
    u = (np.arange(PATCH, dtype=np.float32) - (PATCH - 1) / 2.0)
    kind = p["kind"][:, None, :, None]
    val = np.broadcast_to(p["level"][:, None, :, None].astype(np.float32), (ph, PATCH, pw, PATCH)).copy()
    z = noise_rng.standard_normal((ph, PATCH, pw, PATCH), dtype=np.float32)
    val += np.where(kind == 1, z * p["sigma"][:, None, :, None].astype(np.float32), np.float32(0))
    ramp = (p["slope"][:, None, :, None] * (p["dx"][:, None, :, None] * u[None, None, None, :]
                                           + p["dy"][:, None, :, None] * u[None, :, None, None]))
    val += np.where(kind == 2, ramp.astype(np.float32), np.float32(0))
    val = val.reshape(ph * PATCH, pw * PATCH)[: spec.height, : spec.width]
    lat = np.broadcast_to(_patch_latent(p)[:, None, :, None], (ph, PATCH, pw, PATCH))
    lat = lat.reshape(ph * PATCH, pw * PATCH)[: spec.height, : spec.width].astype(np.float32)
    if blob is not None:
        cx, cy, radius, sigma = blob
        yy = np.arange(spec.height, dtype=np.float32)[:, None]
        xx = np.arange(spec.width, dtype=np.float32)[None, :]
        inside = (xx - cx) ** 2 + (yy - cy) ** 2 <= radius * radius
        zb = noise_rng.standard_normal((spec.height, spec.width), dtype=np.float32)
        val = np.where(inside, np.float32(128.0) + np.float32(sigma) * zb, val)
        lat = np.where(inside, np.float32(sigma * sigma), lat)
    scale = np.float32(2 ** (spec.bit_depth - 8))
    val = np.rint(val * scale)
    np.clip(val, 0, 2 ** spec.bit_depth - 1, out=val)
    dtype = np.uint8 if spec.bit_depth == 8 else np.uint16
    return val.astype(dtype), lat


def _ctu_mean(lat: np.ndarray, spec: FrameSpec) -> np.ndarray:
    """Mean of the latent map over each (clipped) CTU, float64 [R, C]."""
    R, C = spec.ctu_rows, spec.ctu_cols
    pad = np.zeros((R * CTU, C * CTU), dtype=np.float64)
    cnt = np.zeros_like(pad)
    pad[: spec.height, : spec.width] = lat
    cnt[: spec.height, : spec.width] = 1.0
    s = pad.reshape(R, CTU, C, CTU).sum(axis=(1, 3))
    n = cnt.reshape(R, CTU, C, CTU).sum(axis=(1, 3))
    return s / n


def time_map(latent_ctu: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Co-located CTU encoding times (float32 [R, C]) from a latent map."""
    eps = rng.normal(0.0, 0.2, size=latent_ctu.shape)
    return ((0.5 + 0.02 * latent_ctu) * np.exp(eps)).astype(np.float32)


def make_frame(spec: FrameSpec, seed: int, stream: int = 0, frame: int = 0,
               workload: str = "single") -> tuple[np.ndarray, np.ndarray]:
    """One frame and its co-located time map: (plane[H, W], times[R, C] float32)."""
    wid = _WORKLOAD_IDS[workload]
    ph = (spec.height + PATCH - 1) // PATCH
    pw = (spec.width + PATCH - 1) // PATCH
    p = _patch_params(_rng(wid, seed, stream, frame, 0), ph, pw)
    plane, lat = _render(p, spec, _rng(wid, seed, stream, frame, 1), None)
    times = time_map(_ctu_mean(lat, spec), _rng(wid, seed, stream, frame, 2))
    return plane, times


def _blob_at(f: int) -> tuple[float, float, float, float]:
    # the disk moves 32 px per frame to the right with a slow vertical swing
    # (a triangle wave, integer arithmetic only)
    phase = f % 32
    swing = (phase if phase < 16 else 32 - phase) * 24 - 192
    return (512.0 + 32.0 * f, 1080.0 + float(swing), 384.0, 40.0)


def _latent_map(p: dict, spec: FrameSpec, blob) -> np.ndarray:
    ph, pw = p["kind"].shape
    lat = np.broadcast_to(_patch_latent(p)[:, None, :, None], (ph, PATCH, pw, PATCH))
    lat = lat.reshape(ph * PATCH, pw * PATCH)[: spec.height, : spec.width].astype(np.float32)
    if blob is not None:
        cx, cy, radius, sigma = blob
        yy = np.arange(spec.height, dtype=np.float32)[:, None]
        xx = np.arange(spec.width, dtype=np.float32)[None, :]
        inside = (xx - cx) ** 2 + (yy - cy) ** 2 <= radius * radius
        lat = np.where(inside, np.float32(sigma * sigma), lat)
    return lat


def sequence_2160p_frame(f: int, seed: int = 2160) -> tuple[np.ndarray, np.ndarray]:
    """Frame f of the moving-blob UHD sequence and its time map.

    The patch background is drawn once per sequence; noise is redrawn per
    frame; frame f's time map comes from frame f-1's latent complexity
    (frame 0 uses its own).  Frames can be drawn independently."""
    spec = SPEC_2160P10
    ph = (spec.height + PATCH - 1) // PATCH
    pw = (spec.width + PATCH - 1) // PATCH
    wid = _WORKLOAD_IDS["seq2160"]
    p = _patch_params(_rng(wid, seed, 0, 0, 0), ph, pw)
    plane, _ = _render(p, spec, _rng(wid, seed, 0, f, 1), _blob_at(f))
    src = _latent_map(p, spec, _blob_at(max(f - 1, 0)))
    times = time_map(_ctu_mean(src, spec), _rng(wid, seed, 0, f, 2))
    return plane, times


def sequence_2160p_blob(nframes: int = 64, seed: int = 2160):
    """The moving-blob UHD sequence: yields (plane, times) per frame."""
    for f in range(nframes):
        yield sequence_2160p_frame(f, seed)


@dataclass
class BatchItem:
    spec: FrameSpec
    plane: np.ndarray
    times: np.ndarray
    n_regions: int
    lam: float


def mixed_batch_layout(nframes: int = 256, seed: int = 4) -> list[tuple[FrameSpec, int]]:
    """(spec, n) of each frame of the mixed-resolution batch: 480p8 / 1080p10
    / 2160p10 in ratio 4:2:1 (146 / 73 / 37 of 256), n drawn uniformly from
    {4, 8, 16}, shuffled."""
    n480 = round(nframes * 4 / 7)
    n1080 = round(nframes * 2 / 7)
    n2160 = nframes - n480 - n1080
    specs = [SPEC_480P8] * n480 + [SPEC_1080P10] * n1080 + [SPEC_2160P10] * n2160
    rng = _rng(_WORKLOAD_IDS["mixed"], seed, 0, 0, 3)
    order = rng.permutation(len(specs))
    ns = rng.choice([4, 8, 16], size=len(specs))
    return [(specs[j], int(ns[i])) for i, j in enumerate(order)]


def mixed_batch_frame(i: int, nframes: int = 256, seed: int = 4, lam: float = 0.1) -> BatchItem:
    spec, n = mixed_batch_layout(nframes, seed)[i]
    plane, times = make_frame(spec, seed, stream=0, frame=i, workload="mixed")
    return BatchItem(spec, plane, times, n, lam)


def mixed_batch(nframes: int = 256, seed: int = 4, lam: float = 0.1) -> list[BatchItem]:
    """The whole mixed-resolution batch (see mixed_batch_layout)."""
    out = []
    for i, (spec, n) in enumerate(mixed_batch_layout(nframes, seed)):
        plane, times = make_frame(spec, seed, stream=0, frame=i, workload="mixed")
        out.append(BatchItem(spec, plane, times, n, lam))
    return out


@dataclass
class StreamSpec:
    stream: int
    spec: FrameSpec
    n_regions: int
    fps: float


def serving_streams(nstreams: int = 32, seed: int = 5) -> list[StreamSpec]:
    """Half 1080p10 (n=8), half 2160p10 (n=16); Poisson rates U[30, 60] fps."""
    rng = _rng(_WORKLOAD_IDS["serve"], seed, 0, 0, 4)
    fps = rng.uniform(30.0, 60.0, size=nstreams)
    out = []
    for s in range(nstreams):
        if s % 2 == 0:
            out.append(StreamSpec(s, SPEC_1080P10, 8, float(fps[s])))
        else:
            out.append(StreamSpec(s, SPEC_2160P10, 16, float(fps[s])))
    return out


def poisson_arrivals(streams: list[StreamSpec], duration_s: float, seed: int = 6):
    """Merged arrival list [(t_seconds, stream_index, frame_index)] sorted by time."""
    rng = _rng(_WORKLOAD_IDS["serve"], seed, 0, 0, 5)
    ev = []
    for i, s in enumerate(streams):
        t = 0.0
        f = 0
        while True:
            t += rng.exponential(1.0 / s.fps)
            if t >= duration_s:
                break
            ev.append((t, i, f))
            f += 1
    ev.sort()
    return ev


def small_frame(width: int, height: int, bit_depth: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """A frame of arbitrary size for parity and edge-case tests."""
    spec = FrameSpec(f"{width}x{height}p{bit_depth}", width, height, bit_depth)
    return make_frame(spec, seed, workload="test")


def ra_temporal_layer(poc: int, gop: int = 16) -> int:
    """Temporal layer of a picture in a hierarchical random-access GOP
    (GOP 16: layers 0..4): 0 at multiples of the GOP, then one layer per
    halving of the distance to the nearest anchor."""
    r = poc % gop
    if r == 0:
        return 0
    layer, step = 1, gop // 2
    while r % step:
        step //= 2
        layer += 1
    return layer


def ra_coding_order(gop: int = 16) -> list[int]:
    """POCs of the first GOP in coding order: 0, gop, then each layer's
    pictures depth first (gop/2, gop/4, ... before their right halves)."""
    order = [0, gop]

    def split(lo: int, hi: int):
        if hi - lo < 2:
            return
        mid = (lo + hi) // 2
        order.append(mid)
        split(lo, mid)
        split(mid, hi)

    split(0, gop)
    return order


def pack10(plane: np.ndarray) -> np.ndarray:
    """A [H, W] plane of 10-bit samples in the packed format (four samples in
    five bytes): each row a little-endian bit string with sample x in bits
    [10x, 10x + 10); rows of ceil(10 W / 8) bytes, returned as uint8 [H, bytes]."""
    H, W = plane.shape
    s = np.asarray(plane, np.uint64) & np.uint64(1023)
    Wp = -(-W // 4) * 4
    if Wp != W:
        s = np.concatenate([s, np.zeros((H, Wp - W), np.uint64)], axis=1)
    g = s.reshape(H, Wp // 4, 4)
    v = g[:, :, 0] | (g[:, :, 1] << np.uint64(10)) | (g[:, :, 2] << np.uint64(20)) | (g[:, :, 3] << np.uint64(30))
    out = np.zeros((H, Wp // 4, 5), np.uint8)
    for b in range(5):
        out[:, :, b] = ((v >> np.uint64(8 * b)) & np.uint64(255)).astype(np.uint8)
    return np.ascontiguousarray(out.reshape(H, Wp // 4 * 5)[:, : (10 * W + 7) // 8])
