"""Pins of the oracle's per-CTU texture statistics (S1 = sum p, S2 = sum p^2,
N = samples), the quantities the RS-clustering term of Eq. 2 (Sec. 2.2) needs."""

from fractions import Fraction

import numpy as np
import pytest


def _ctu_sizes(W, H):
    C, R = -(-W // 128), -(-H // 128)
    cw = [min(128 * (x + 1), W) - 128 * x for x in range(C)]
    ch = [min(128 * (y + 1), H) - 128 * y for y in range(R)]
    return C, R, cw, ch


@pytest.mark.parametrize("W,H,bd,v", [(832, 480, 8, 200), (300, 129, 10, 1023), (128, 128, 10, 0),
                                      (1, 1, 8, 255), (257, 200, 12, 4095)])
def test_constant_plane_closed_form(oracle, W, H, bd, v):
    dt = np.uint8 if bd == 8 else np.uint16
    st = oracle.texture(np.full((H, W), v, dt), bd)
    assert st.status == oracle.OK
    C, R, cw, ch = _ctu_sizes(W, H)
    N = np.array([[w * h for w in cw] for h in ch], np.uint64)
    assert (st.N == N).all()
    assert (st.S1 == N * v).all()
    assert (st.S2 == N * v * v).all()
    assert (st.vmax == v).all()


@pytest.mark.parametrize("a,b,W,H", [(3, 5, 512, 256), (1, 0, 200, 130), (7, 2, 130, 64)])
def test_horizontal_ramp_sse_closed_form(oracle, a, b, W, H):
    # p(x, y) = a * (x mod 128) + b: inside a CTU of width w, height h the
    # exact SSE is h * a^2 * w (w^2 - 1) / 12.
    x = np.arange(W) % 128
    plane = np.tile((a * x + b).astype(np.uint16), (H, 1))
    st = oracle.texture(plane, 10)
    C, R, cw, ch = _ctu_sizes(W, H)
    for y in range(R):
        for xx in range(C):
            S1, S2, N = int(st.S1[y, xx]), int(st.S2[y, xx]), int(st.N[y, xx])
            w, h = cw[xx], ch[y]
            sse = Fraction(S2) - Fraction(S1 * S1, N)
            assert sse == Fraction(h * a * a * w * (w * w - 1), 12)


@pytest.mark.parametrize("W,H,bd", [(832, 480, 8), (1000, 700, 10), (129, 257, 10), (64, 64, 12)])
def test_random_plane_matches_block_sums(oracle, W, H, bd):
    rng = np.random.default_rng(W * H + bd)
    dt = np.uint8 if bd == 8 else np.uint16
    plane = rng.integers(0, 2 ** bd, size=(H, W)).astype(dt)
    st = oracle.texture(plane, bd)
    C, R, _, _ = _ctu_sizes(W, H)
    p = plane.astype(np.uint64)
    rows = np.arange(0, H, 128)
    cols = np.arange(0, W, 128)
    s1 = np.add.reduceat(np.add.reduceat(p, rows, axis=0), cols, axis=1)
    s2 = np.add.reduceat(np.add.reduceat(p * p, rows, axis=0), cols, axis=1)
    mx = np.maximum.reduceat(np.maximum.reduceat(plane.astype(np.uint32), rows, axis=0), cols, axis=1)
    assert (st.S1 == s1).all() and (st.S2 == s2).all() and (st.vmax == mx).all()


def test_pitch_padding_is_ignored(oracle):
    rng = np.random.default_rng(1)
    W, H = 300, 140
    plane = rng.integers(0, 1024, size=(H, W)).astype(np.uint16)
    padded = np.full((H, W + 37), 0xFFFF, np.uint16)
    padded[:, :W] = plane
    a = oracle.texture(plane, 10)
    # same bytes, longer pitch, padding holds out-of-range samples that must not be read
    b = oracle.texture(padded[:, :W], 10, pitch=padded.strides[0])
    assert b.status == oracle.OK
    assert (a.S1 == b.S1).all() and (a.S2 == b.S2).all() and (a.N == b.N).all()


def test_little_endian_and_range_check(oracle):
    plane = np.zeros((4, 4), np.uint16)
    plane[0, 0] = 0x0201
    st = oracle.texture(plane, 10)
    assert st.status == oracle.OK and int(st.S1[0, 0]) == 0x0201
    plane[1, 1] = 1024  # >= 2^10
    st = oracle.texture(plane, 10)
    assert st.status == oracle.ERANGE
    assert oracle.texture(np.full((2, 2), 255, np.uint8), 8).status == oracle.OK


def test_packed10_worked_bytes(oracle):
    """Four samples 1, 2, 3, 1023 in five bytes: the 40-bit value
    1 + 2 * 2^10 + 3 * 2^20 + 1023 * 2^30, little endian, is
    01 08 30 C0 FF; the oracle reads them back."""
    import synth
    plane = np.array([[1, 2, 3, 1023]], np.uint16)
    packed = synth.pack10(plane)
    assert packed.tolist() == [[0x01, 0x08, 0x30, 0xC0, 0xFF]]
    st = oracle.texture(packed, oracle.PACKED10, width=4)
    assert st.status == oracle.OK
    assert (int(st.S1[0, 0]), int(st.S2[0, 0]), int(st.N[0, 0]), int(st.vmax[0, 0])) == (
        1029, 1 + 4 + 9 + 1023 * 1023, 4, 1023)


@pytest.mark.parametrize("W,H", [(1, 1), (3, 5), (129, 130), (300, 257), (1920, 1080)])
def test_packed10_equals_two_byte_samples(oracle, W, H):
    """The packed plane of a 10-bit frame has the frame's statistics; ragged
    widths (W not a multiple of 4 or 128) and a padded pitch included."""
    import synth
    rng = np.random.default_rng(W * 3 + H)
    plane = rng.integers(0, 1024, size=(H, W)).astype(np.uint16)
    ref = oracle.texture(plane, 10)
    packed = synth.pack10(plane)
    assert packed.shape == (H, (10 * W + 7) // 8)
    got = oracle.texture(packed, oracle.PACKED10, width=W)
    for a, b in ((got.S1, ref.S1), (got.S2, ref.S2), (got.N, ref.N), (got.vmax, ref.vmax)):
        assert (a == b).all()
    pitch = -(-packed.shape[1] // 16) * 16 + 16
    buf = np.zeros((H, pitch), np.uint8)
    buf[:, : packed.shape[1]] = packed
    got2 = oracle.texture(buf[:, : packed.shape[1]], oracle.PACKED10, pitch=pitch, width=W)
    assert (got2.S2 == ref.S2).all() and (got2.S1 == ref.S1).all()
