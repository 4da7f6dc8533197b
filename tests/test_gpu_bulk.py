"""The TMA-family kernel with bulk row staging, against the CPU oracle, bit
for bit.

Sources whose address or row pitch is not a multiple of 16 bytes are staged
one image row at a time with 1-D bulk copies of the 16-byte granules that
hold the row's columns; the kernel then reads each row from a per-row byte
offset.  Every shape below is placed at byte offsets 1..15 from a 16-byte
boundary and with odd pitches, so that the granule arithmetic meets every
phase; ragged widths and heights, segments and bands that cross the image
edges, every border rule, every output format, and strip heights of 4, 6 and
the default all go through it.  Tolerance: zero mismatched elements, and no
byte written outside the destination's payload.
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

# (H, W, source offset, extra pitch bytes)
CASES = [(1, 1, 1, 0), (1, 9, 3, 1), (9, 1, 5, 2), (3, 3, 7, 0), (5, 5, 15, 3), (6, 3, 9, 1),
         (7, 130, 1, 1), (5, 131, 2, 0), (8, 127, 13, 5), (9, 128, 4, 1), (10, 129, 8, 7),
         (11, 133, 6, 0), (12, 255, 11, 2), (13, 256, 12, 9), (17, 257, 14, 1),
         (33, 300, 10, 3), (64, 5, 3, 4), (70, 390, 1, 0), (129, 131, 15, 15),
         (3, 1000, 5, 1), (200, 261, 7, 2), (261, 389, 9, 0), (130, 1029, 2, 11),
         (96, 512, 8, 0), (40, 1024, 1, 3)]


@pytest.fixture(scope="module")
def handles():
    from paper_2305_00515_gb300 import build
    build.build()
    hs = {}
    for name, R in (("bulk", 0), ("bulk_r4", 4), ("bulk_r6", 6)):
        st, h = pkg.sobel4_create(0, pkg.VARIANTS["rg"], rows_per_strip=R)
        assert st == 0, pkg.sobel4_status_string(st)
        hs[name] = h
    st, h = pkg.sobel4_create(0, pkg.VARIANTS["rg_lanecopy"])
    assert st == 0
    hs["lanecopy"] = h
    yield hs
    for h in hs.values():
        pkg.sobel4_destroy(h)


def assert_same(got, want, what):
    if not same_bits(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {bad[:4].tolist()}")


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}+{c[2]}p{c[3]}")
def test_unaligned_rows_every_border_and_format(handles, case):
    H, W, off, extra = case
    rng = np.random.default_rng(11 * H + W + off)
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    for border in BORDERS:
        if border == "reflect101" and (H < 3 or W < 3):
            continue
        for fmt in FORMATS:
            want = oracle.sobel4(img, border, fmt)
            for name in ("bulk", "bulk_r4", "bulk_r6"):
                got, guards = run_placed(torch, handles[name], img, border, fmt,
                                         src_pitch=W + extra, src_offset=off)
                assert guards, f"{name} {case} {border} {fmt}: write outside the payload"
                assert_same(got, want, f"{name} {case} {border} {fmt}")


@pytest.mark.parametrize("border", BORDERS)
@pytest.mark.parametrize("fmt", FORMATS)
def test_bulk_and_lanecopy_agree_2k(handles, border, fmt):
    """A 2048x2176 image at byte offset 5 with pitch 2181: tall bands, both kernels, the oracle."""
    img = synth.rects_noise(2048, 2176, 23)
    a, ga = run_placed(torch, handles["bulk"], img, border, fmt, src_pitch=2181, src_offset=5)
    b, gb = run_placed(torch, handles["lanecopy"], img, border, fmt, src_pitch=2181,
                       src_offset=5)
    assert ga and gb
    assert_same(a, b, f"bulk vs lanecopy {border} {fmt}")
    assert_same(a, oracle.sobel4(img, border, fmt, threads=NCPU), f"bulk {border} {fmt}")


def test_every_source_phase_one_shape(handles):
    """One 67x389 image at each of the 16 byte offsets, pitch 389 (odd)."""
    img = synth.rects_noise(67, 389, 3)
    want = {b: oracle.sobel4(img, b, "f32") for b in BORDERS}
    for off in range(16):
        for border in BORDERS:
            got, guards = run_placed(torch, handles["bulk"], img, border, "f32", src_pitch=389,
                                     src_offset=off)
            assert guards
            assert_same(got, want[border], f"offset {off} {border}")
    assert pkg.sobel4_device_status(handles["bulk"]) == 0
