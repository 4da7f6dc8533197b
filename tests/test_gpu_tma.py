"""The TMA-staged register-window kernel against the CPU oracle, bit for bit.

Sources whose address and row pitch are multiples of 16 bytes are staged with
2-D tensor copies; every shape below is run with such a pitch (rows padded to
a multiple of 16), so that ragged widths and heights, segments that cross the
left and right edges, bands that cross the top and bottom edges, every border
rule and every output format all go through that kernel.  Strip heights of 4
and 6 rows (tiny bands, many edge items) and the default (tall bands) are
covered; the lane-copy staging is run on the same aligned inputs for
comparison.  Tolerance: zero mismatched elements.
"""
import numpy as np
import pytest

import oracle
import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import run_placed, same_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BORDERS = ("valid", "replicate", "reflect101", "constant0")
FORMATS = ("f32", "u8", "s16x4", "u16", "edge8")
ELEM = {"f32": 4, "u8": 1, "s16x4": 2, "u16": 2, "edge8": 1}
NCPU = oracle.cpu_count()

SHAPES = [(1, 1), (1, 9), (9, 1), (2, 2), (3, 3), (4, 4), (5, 5), (6, 3), (7, 130), (5, 131),
          (8, 127), (9, 128), (10, 129), (11, 133), (12, 255), (13, 256), (17, 257), (33, 300),
          (64, 5), (100, 6), (70, 390), (129, 131), (3, 1000), (200, 261), (261, 389),
          (130, 1029)]


def ceil16(v):
    return (v + 15) // 16 * 16


@pytest.fixture(scope="module")
def handles():
    from paper_2305_00515_gb300 import build
    build.build()
    hs = {}
    for name, variant, R in (("tma", "rg", 0), ("tma_r4", "rg", 4), ("tma_r6", "rg", 6),
                             ("lanecopy", "rg_lanecopy", 0)):
        st, h = pkg.sobel4_create(0, pkg.VARIANTS[variant], rows_per_strip=R)
        assert st == 0, pkg.sobel4_status_string(st)
        hs[name] = h
    yield hs
    for h in hs.values():
        pkg.sobel4_destroy(h)


def assert_same(got, want, what):
    if not same_bits(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {bad[:4].tolist()}")


@pytest.mark.parametrize("HW", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_aligned_rows_every_border_and_format(handles, HW):
    H, W = HW
    rng = np.random.default_rng(7 * H + W)
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    for border in BORDERS:
        if border == "reflect101" and (H < 3 or W < 3):
            continue
        for fmt in FORMATS:
            want = oracle.sobel4(img, border, fmt)
            for name in ("tma", "tma_r4", "tma_r6"):
                got, guards = run_placed(torch, handles[name], img, border, fmt,
                                         src_pitch=ceil16(W), dst_pitch=ceil16(W * ELEM[fmt]))
                assert guards, f"{name} {H}x{W} {border} {fmt}: write outside the payload"
                assert_same(got, want, f"{name} {H}x{W} {border} {fmt}")


@pytest.mark.parametrize("fmt", FORMATS)
def test_aligned_source_unaligned_destination(handles, fmt):
    """Destinations that cannot take vector stores go through the per-element stores."""
    for (H, W) in ((37, 301), (64, 512), (300, 700)):
        img = synth.rects_noise(H, W, 5 + W)
        for border in BORDERS:
            for name in ("tma", "tma_r4"):
                got, guards = run_placed(torch, handles[name], img, border, fmt,
                                         src_pitch=ceil16(W) + 16,
                                         dst_pitch=(W + 3) * ELEM[fmt],
                                         dst_offset=2 * ELEM[fmt] if fmt != "u8" else 3)
                assert guards
                assert_same(got, oracle.sobel4(img, border, fmt), f"{name} {H}x{W} {border}")


@pytest.mark.parametrize("border", BORDERS)
@pytest.mark.parametrize("fmt", FORMATS)
def test_tma_and_lanecopy_agree_2k(handles, border, fmt):
    """A 2048x2176 image: tall bands, interior and edge items, both stagings and the oracle."""
    img = synth.rects_noise(2048, 2176, 21)
    a, ga = run_placed(torch, handles["tma"], img, border, fmt)
    b, gb = run_placed(torch, handles["lanecopy"], img, border, fmt)
    assert ga and gb
    assert_same(a, b, f"tma vs lanecopy {border} {fmt}")
    assert_same(a, oracle.sobel4(img, border, fmt, threads=NCPU), f"tma {border} {fmt}")


def test_device_status_clean_after_runs(handles):
    img = synth.uniform(256, 256, 1)
    for name in ("tma", "tma_r4"):
        run_placed(torch, handles[name], img, "valid", "f32")
        assert pkg.sobel4_device_status(handles[name]) == 0


@pytest.mark.parametrize("fmt", FORMATS)
def test_realigned_stores_every_phase(handles, fmt):
    """Fast-path items into destinations at every sub-vector offset, with a
    pitch that moves the offset from row to row, from aligned and unaligned
    sources: the lane-shifted stores, the head and tail elements of each
    segment and the zeroed frame of the paper's rule."""
    e = ELEM[fmt]
    vec = {"f32": 16, "u8": 4, "s16x4": 8, "u16": 8, "edge8": 4}[fmt]
    for (H, W) in ((40, 256), (33, 384), (70, 517)):
        img = synth.rects_noise(H, W, 3 * W + H)
        for border in BORDERS:
            want = oracle.sobel4(img, border, fmt)
            for doff in range(e, vec, e):
                for (sp, soff) in ((ceil16(W), 0), (W + 1, 3)):
                    for name in ("tma", "tma_r4"):
                        got, guards = run_placed(torch, handles[name], img, border, fmt,
                                                 src_pitch=sp, src_offset=soff,
                                                 dst_pitch=W * e + e, dst_offset=doff)
                        assert guards, f"{name} {H}x{W} {border} doff {doff}: outside payload"
                        assert_same(got, want, f"{name} {H}x{W} {border} doff {doff} sp {sp}")


RAGGED_W = (1, 2, 3, 4, 5, 7, 126, 127, 129, 131, 133, 134, 254, 255, 257, 259, 383)


@pytest.mark.parametrize("fmt", FORMATS)
def test_ragged_last_segment_fast_path(handles, fmt):
    """Widths that end inside a 128-column segment, under the rules the fast
    path serves at any width (VALID; CONSTANT0 from aligned rows): the last
    segment's lanes stop their stores at column W, into vector-aligned and
    lane-shifted destinations, from tensor- and bulk-staged sources, with the
    frame columns W-2 and W-1 zeroed inside that segment.  The guard bytes
    after each row's payload must survive."""
    e = ELEM[fmt]
    for W in RAGGED_W:
        H = 21 + W % 7
        img = np.random.default_rng(W).integers(0, 256, size=(H, W), dtype=np.uint8)
        for border in ("valid", "constant0"):
            want = oracle.sobel4(img, border, fmt)
            for (dp, doff) in ((ceil16(W * e), 0), (W * e + e, e), (ceil16(W * e) + 16, 3 * e)):
                for (sp, soff) in ((ceil16(W), 0), (W + 1, 5)):
                    for name in ("tma", "tma_r4"):
                        got, guards = run_placed(torch, handles[name], img, border, fmt,
                                                 src_pitch=sp, src_offset=soff,
                                                 dst_pitch=dp, dst_offset=doff)
                        what = f"{name} {H}x{W} {border} dp {dp} doff {doff} sp {sp}"
                        assert guards, f"{what}: write outside the payload"
                        assert_same(got, want, what)
