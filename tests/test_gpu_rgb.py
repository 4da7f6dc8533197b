"""Colour input through sobel4_run_rgb: the kernel turns interleaved RGB rows
into gray as it reads them (Y = (77 R + 150 G + 29 B + 128) >> 8, the reading
of the paper's host-side grayscale preparation) and runs the operator on Y.
Every output is compared element by element with the CPU oracle's
convert-then-operate (tolerance: 0 mismatched elements), with guard bytes
around every row and buffer."""
import numpy as np
import pytest

import oracle
import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import ELEM, Output, Placed, same_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BORDERS = ("valid", "replicate", "reflect101", "constant0")
FORMATS = ("f32", "u8", "s16x4", "u16", "edge8")
SHAPES = [(1, 1), (3, 5), (5, 5), (7, 130), (37, 61), (64, 128), (130, 257), (200, 261),
          (9, 384), (257, 300)]


def rgb_image(H, W, seed):
    """Three differently seeded rects+noise channels, interleaved."""
    return np.stack([synth.rects_noise(H, W, seed * 3 + c) for c in range(3)], axis=2)


def run_rgb(h, rgb, border, fmt, src_pitch, src_off, dst_pitch, dst_off):
    H, W, _ = rgb.shape
    src = Placed(torch, rgb.reshape(H, 3 * W), src_pitch, src_off)
    out = Output(torch, H, W, fmt, dst_pitch, dst_off)
    rc = pkg.sobel4_run_rgb(h, src.ptr, src.pitch, out.ptr, out.pitch, H, W,
                            pkg.BORDERS[border], pkg.FORMATS[fmt],
                            torch.cuda.current_stream().cuda_stream)
    assert rc == 0, pkg.sobel4_status_string(rc)
    torch.cuda.synchronize()
    return out.read()


@pytest.fixture(scope="module")
def handle():
    from paper_2305_00515_gb300 import build
    build.build()
    st, h = pkg.sobel4_create(0)
    assert st == 0
    yield h
    assert pkg.sobel4_device_status(h) == 0  # no bounded wait ran out
    pkg.sobel4_destroy(h)


@pytest.mark.parametrize("border", BORDERS)
@pytest.mark.parametrize("fmt", FORMATS)
def test_rgb_every_shape_border_format(handle, border, fmt):
    e = ELEM[fmt]
    for i, (H, W) in enumerate(SHAPES):
        if border == "reflect101" and (H < 3 or W < 3):
            continue
        rgb = rgb_image(H, W, 100 + i)
        want = oracle.sobel4_rgb(rgb, border, fmt)
        # tight rows; rows padded to 16 bytes; odd pitch and byte offsets
        layouts = ((3 * W, 0, W * e, 0), ((3 * W + 15) // 16 * 16, 0, (W * e + 15) // 16 * 16, 0),
                   (3 * W + 5, 3, W * e + 2 * e, e))
        for sp, so, dp, do in layouts:
            got, guards = run_rgb(handle, rgb, border, fmt, sp, so, dp, do)
            assert guards, f"{H}x{W} {border} {fmt}: write outside the payload"
            assert same_bits(got, want), f"{H}x{W} {border} {fmt} (pitch {sp}, offset {so})"


def test_rgb_large_images(handle):
    for (H, W, sp, so) in ((1080, 1920, 3 * 1920, 0), (2048, 2176, 3 * 2176 + 7, 5)):
        rgb = rgb_image(H, W, 7)
        got, guards = run_rgb(handle, rgb, "valid", "f32", sp, so, 4 * W, 0)
        assert guards and same_bits(got, oracle.sobel4_rgb(rgb, "valid", "f32",
                                                           threads=oracle.cpu_count()))


def test_rgb_8192_sampled_rows(handle):
    H = W = 8192
    rgb = rgb_image(H, W, 3)
    src = torch.from_numpy(rgb).cuda()
    with pkg.Sobel4(0) as s:
        out = s.run_rgb(src)
        torch.cuda.synchronize()
    for y0 in (0, 2, 4091, H - 10):
        band = rgb[max(0, y0 - 2):y0 + 12]
        want = oracle.sobel4_rgb(band, "valid", "f32")
        off = y0 - max(0, y0 - 2)
        rows = range(max(y0, 2), min(y0 + 10, H - 2))
        for y in rows:
            assert same_bits(out[y].cpu().numpy(), want[y - y0 + off]), y
    assert same_bits(out[:2].cpu().numpy(), np.zeros((2, W), np.float32))


def test_rgb_gray_input_equals_gray_operator(handle):
    img = synth.rects_noise(301, 517, 9)
    rgb = np.repeat(img[:, :, None], 3, axis=2)
    with pkg.Sobel4(0) as s:
        a = s.run_rgb(torch.from_numpy(rgb).cuda(), border="replicate")
        b = s.run(torch.from_numpy(img).cuda(), border="replicate")
        torch.cuda.synchronize()
    assert same_bits(a.cpu().numpy(), b.cpu().numpy())


def test_rgb_rejects(handle):
    dst = torch.empty((8, 16), dtype=torch.float32, device="cuda")
    src = torch.zeros((8, 48), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    # pitch below 3 * width
    assert pkg.sobel4_run_rgb(handle, src.data_ptr(), 40, dst.data_ptr(), 64, 8, 16, 0, 0,
                              st) == 1
    # runtime weights are served by other kernels only
    ok, h2 = pkg.sobel4_create(0)
    assert pkg.sobel4_set_weights(h2, 2, 1, 2, 2) == 0
    assert pkg.sobel4_run_rgb(h2, src.data_ptr(), 48, dst.data_ptr(), 64, 8, 16, 0, 0, st) == 2
    pkg.sobel4_destroy(h2)
