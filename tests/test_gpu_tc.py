"""The tensor-core kernel (VALID, F32, source and destination rows on 16-byte
boundaries, widths that are multiples of 4) against the CPU oracle, bit for
bit.

Shapes cover a single tile, ragged tile rows and columns (heights and widths
that are not multiples of 128 and 64), images narrower than one tile, many
tiles per CTA, and a full-width 8192 image sampled by rows.  Tolerance: zero
mismatched elements and no byte written outside the destination's payload.
The handle (variant TC) reports which kernel serves each shape, so these
tests fail if the images silently take another path.
"""
import numpy as np
import pytest

import oracle
import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import run_placed, same_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Widths that are multiples of 4 run on the tensor-core kernel; the others
# (whose rows do not end on a 16-byte unit of the output) on the
# register-window kernel, which the same handle picks.
SHAPES = [(1, 8), (3, 12), (5, 8), (8, 64), (7, 68), (64, 72), (128, 132), (129, 200),
          (130, 128), (200, 124), (257, 1000), (300, 332), (511, 260), (1000, 76),
          (3, 9), (64, 66), (130, 127)]


def ceil16(v):
    return (v + 15) // 16 * 16


@pytest.fixture(scope="module")
def handle():
    from paper_2305_00515_gb300 import build
    build.build()
    st, h = pkg.sobel4_create(0, pkg.VARIANTS["tc"])
    assert st == 0, pkg.sobel4_status_string(st)
    yield h
    pkg.sobel4_destroy(h)


def assert_same(got, want, what):
    if not same_bits(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {bad[:4].tolist()}")


@pytest.mark.parametrize("HW", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_tc_matches_oracle(handle, HW):
    H, W = HW
    st, kind, _, _ = pkg.sobel4_tune_config(handle, H, W, pkg.FORMATS["f32"])
    assert st == 0 and (kind == 2) == (W % 4 == 0), "the tensor-core kernel serves W % 4 == 0"
    rng = np.random.default_rng(3 * H + W)
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    want = oracle.sobel4(img, "valid", "f32")
    for dst_pitch, dst_off in ((ceil16(4 * W), 0), (ceil16(4 * W) + 16, 16),
                               (ceil16(4 * W) + 48, 32)):
        got, guards = run_placed(torch, handle, img, "valid", "f32", src_pitch=ceil16(W),
                                 dst_pitch=dst_pitch, dst_offset=dst_off)
        assert guards, f"{H}x{W} dst pitch {dst_pitch}: write outside the payload"
        assert_same(got, want, f"{H}x{W} dst pitch {dst_pitch}")
    assert pkg.sobel4_device_status(handle) == 0


def test_tc_extreme_values(handle):
    """Constant, checkerboard and 0/255 step images: the largest responses."""
    H, W = 260, 300  # W % 4 == 0
    yy, xx = np.mgrid[0:H, 0:W]
    imgs = [np.full((H, W), 255, np.uint8), ((yy + xx) % 2 * 255).astype(np.uint8),
            ((xx > yy) * 255).astype(np.uint8), ((xx // 2 + yy // 3) % 2 * 255).astype(np.uint8)]
    for k, img in enumerate(imgs):
        got, guards = run_placed(torch, handle, img, "valid", "f32", src_pitch=ceil16(W))
        assert guards
        assert_same(got, oracle.sobel4(img, "valid", "f32"), f"pattern {k}")


def test_tc_full_width_rows(handle):
    """An 8192 x 8192 image: rows sampled across tile boundaries and the frame."""
    H = W = 8192
    img = synth.rects_noise(H, W, 5)
    src = torch.from_numpy(img).cuda()
    out = torch.full((H, W), -1.0, dtype=torch.float32, device="cuda")
    rc = pkg.sobel4_run(handle, src.data_ptr(), W, out.data_ptr(), 4 * W, H, W,
                        pkg.BORDERS["valid"], pkg.FORMATS["f32"],
                        torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    for y0 in (0, 126, 2047, 4095, 8188):
        rows = slice(max(0, y0 - 2), min(H, y0 + 6))
        want = oracle.sobel4(img[rows], "valid", "f32")
        got = out[rows].cpu().numpy()
        lo = 0 if rows.start == 0 else 2
        hi = want.shape[0] if rows.stop == H else want.shape[0] - 2
        assert_same(got[lo:hi], want[lo:hi], f"rows from {rows.start}")
    assert pkg.sobel4_device_status(handle) == 0


def test_tc_withheld_copy_times_out_and_context_survives(handle):
    img = synth.rects_noise(512, 4096, 9)
    assert pkg.sobel4_inject_stage_loss(handle, 1) == 0
    run_placed(torch, handle, img, "valid", "f32")
    assert pkg.sobel4_device_status(handle) == 5, "the withheld copy must time out"
    got, guards = run_placed(torch, handle, img, "valid", "f32")
    assert guards
    assert_same(got, oracle.sobel4(img, "valid", "f32", threads=oracle.cpu_count()), "after")
    assert pkg.sobel4_device_status(handle) == 0
