"""The seeded synthetic inputs follow their stated recipe and are
reproducible: the same seed gives the same bytes, so the oracle, the GPU
tests and the benchmark see the same frames.  (The generator only draws
random numbers; none of the partitioning arithmetic is here.)"""

import numpy as np
import pytest

import synth
from synth import frames as F


def test_same_seed_same_frame_other_seed_differs():
    a, b, c = (synth.make_frame(synth.SPEC_480P8, s) for s in (7, 7, 8))
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()
    assert not (a[0] == c[0]).all() and not (a[1] == c[1]).all()


@pytest.mark.parametrize("spec", [synth.SPEC_480P8, synth.SPEC_1080P10, synth.SPEC_2160P10])
def test_shapes_types_and_ranges(spec):
    plane, times = synth.make_frame(spec, 3)
    assert plane.shape == (spec.height, spec.width)
    assert plane.dtype == (np.uint8 if spec.bit_depth == 8 else np.uint16)
    assert int(plane.max()) < 2 ** spec.bit_depth
    assert times.shape == (spec.ctu_rows, spec.ctu_cols) and times.dtype == np.float32
    assert np.isfinite(times).all() and (times > 0).all() and (times < 65536).all()


def test_time_model():
    """t = (0.5 + 0.02 * latent) * exp(eps), eps ~ N(0, 0.2^2)."""
    z = np.log(F.time_map(np.zeros((300, 300)), np.random.default_rng(0)) / 0.5)
    assert abs(z.mean()) < 0.005 and abs(z.std() - 0.2) < 0.005
    t = F.time_map(np.full((300, 300), 100.0), np.random.default_rng(1))
    assert abs(np.median(t) / 2.5 - 1.0) < 0.01


def test_uhd_sequence_is_reproducible_frame_by_frame():
    a = synth.sequence_2160p_frame(3)
    b = list(synth.sequence_2160p_blob(4))[3]
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()
    assert not (a[0] == synth.sequence_2160p_frame(4)[0]).all()  # the disk moves


def test_mixed_batch_layout():
    lay = F.mixed_batch_layout()
    assert len(lay) == 256 and lay == F.mixed_batch_layout()
    counts = {s.name: sum(1 for t, _ in lay if t is s) for s in (synth.SPEC_480P8, synth.SPEC_1080P10,
                                                                 synth.SPEC_2160P10)}
    assert list(counts.values()) == [146, 73, 37]
    assert {n for _, n in lay} == {4, 8, 16}


def test_serving_streams_and_arrivals():
    streams = F.serving_streams()
    assert len(streams) == 32
    assert all(s.spec is (synth.SPEC_1080P10 if s.stream % 2 == 0 else synth.SPEC_2160P10) for s in streams)
    assert all(s.n_regions == (8 if s.stream % 2 == 0 else 16) and 30.0 <= s.fps <= 60.0 for s in streams)
    ev = F.poisson_arrivals(streams, 2.0)
    assert ev == sorted(ev) and all(0.0 < t < 2.0 for t, _, _ in ev)
    for i in range(len(streams)):
        assert [f for _, j, f in ev if j == i] == list(range(sum(1 for _, j, _ in ev if j == i)))
    offered = sum(s.fps for s in streams) * 2.0
    assert abs(len(ev) - offered) < 4 * offered ** 0.5


def test_random_access_gop_16():
    """Layer 0 at multiples of 16, then one layer per halving (8: 1, 4/12: 2,
    even: 3, odd: 4); the coding order starts 0, 16 and codes every picture
    after the two pictures it lies between."""
    assert [F.ra_temporal_layer(p) for p in range(17)] == [0, 4, 3, 4, 2, 4, 3, 4, 1, 4, 3, 4, 2, 4, 3, 4, 0]
    order = F.ra_coding_order()
    assert sorted(order) == list(range(17)) and order[:2] == [0, 16]
    for i, p in enumerate(order[2:], start=2):
        step = 1 << (4 - F.ra_temporal_layer(p))
        assert p - step in order[:i] and p + step in order[:i]
