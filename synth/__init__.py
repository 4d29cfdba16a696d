"""Seeded synthetic inputs shaped like the paper's workloads.

This package only draws random numbers: luma planes made of 64x64 patches
(flat, Gaussian-noise and linear-ramp kinds, plus an optional moving
high-detail disk) and per-CTU co-located encoding-time maps from a
latent-complexity model.  It holds none of the partitioning method's
arithmetic and is shared by the tests, the oracle checks and the benchmark.
"""

from .frames import (  # noqa: F401
    BatchItem,
    FrameSpec,
    SPEC_480P8,
    SPEC_1080P10,
    SPEC_2160P10,
    StreamSpec,
    make_frame,
    mixed_batch,
    mixed_batch_frame,
    mixed_batch_layout,
    pack10,
    poisson_arrivals,
    ra_coding_order,
    ra_temporal_layer,
    sequence_2160p_blob,
    sequence_2160p_frame,
    serving_streams,
    small_frame,
    time_map,
)
