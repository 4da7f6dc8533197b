"""The persistent batched kernel: every image of a ragged batch equals its
single-image output and the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import Output, Placed, same_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NCPU = oracle.cpu_count()


@pytest.fixture(scope="module")
def h():
    from paper_2305_00515_gb300 import build
    build.build()
    st, h = pkg.sobel4_create(0)
    assert st == 0
    yield h
    pkg.sobel4_destroy(h)


def run_batch(h, imgs, border, fmt, layout=None):
    elem = {"f32": 4, "u8": 1, "s16x4": 2, "u16": 2, "edge8": 1}[fmt]
    srcs, outs, descs = [], [], []
    for i, img in enumerate(imgs):
        H, W = img.shape
        spx, so, dpx, do = layout[i] if layout else (0, 0, 0, 0)
        s = Placed(torch, img, W + spx, so)
        o = Output(torch, H, W, fmt, (W + dpx) * elem, do)
        srcs.append(s)
        outs.append(o)
        descs.append(pkg.Image(s.ptr, s.pitch, o.ptr, o.pitch, H, W))
    rc = pkg.sobel4_run_batched(h, descs, pkg.BORDERS[border], pkg.FORMATS[fmt],
                                torch.cuda.current_stream().cuda_stream)
    assert rc == 0, pkg.sobel4_status_string(rc)
    torch.cuda.synchronize()
    return [o.read() for o in outs]


def test_ragged_512_batch_matches_oracle(h):
    """The 512-image ragged batch (sides U{37..2048}, seed 1) in one persistent launch."""
    imgs = synth.batch_images(512, 1)
    res = run_batch(h, imgs, "valid", "f32")
    for i, (img, (got, guards)) in enumerate(zip(imgs, res)):
        assert guards, f"image {i}: write outside its output"
        want = oracle.sobel4(img, "valid", "f32", threads=NCPU)
        assert same_bits(got, want), f"image {i} {img.shape} differs from the oracle"


def test_ragged_512_batch_at_the_tuned_configuration():
    """The configuration the bench times: sobel4_tune_batched on the 512-image
    batch, then the batch again; every image against the oracle."""
    imgs = synth.batch_images(512, 1)
    st, ht = pkg.sobel4_create(0)
    assert st == 0
    try:
        srcs = [Placed(torch, img, img.shape[1], 0) for img in imgs]
        outs = [Output(torch, *img.shape, "f32", 4 * img.shape[1], 0) for img in imgs]
        descs = [pkg.Image(s.ptr, s.pitch, o.ptr, o.pitch, *img.shape)
                 for s, o, img in zip(srcs, outs, imgs)]
        st, us = pkg.sobel4_tune_batched(ht, descs, 0, 0)
        assert st == 0 and us > 0
        for o in outs:  # the tuning runs wrote results; start from other bytes (tight rows)
            o.buf[o.offset:o.offset + o.H * o.pitch].fill_(0x7F)
        rc = pkg.sobel4_run_batched(ht, descs, 0, 0, torch.cuda.current_stream().cuda_stream)
        assert rc == 0, pkg.sobel4_status_string(rc)
        torch.cuda.synchronize()
        for i, (img, o) in enumerate(zip(imgs, outs)):
            got, guards = o.read()
            assert guards, f"image {i}: write outside its output"
            want = oracle.sobel4(img, "valid", "f32", threads=NCPU)
            assert same_bits(got, want), f"image {i} {img.shape} differs at the tuned configuration"
        assert pkg.sobel4_device_status(ht) == 0
    finally:
        pkg.sobel4_destroy(ht)


def test_batch_equals_single_runs_all_modes(h):
    rng = np.random.default_rng(3)
    shapes = [(int(a), int(b)) for a, b in rng.integers(3, 400, size=(24, 2))] + [(3, 3), (1000, 7)]
    imgs = [synth.uniform(a, b, i) for i, (a, b) in enumerate(shapes)]
    layout = [(int(rng.integers(0, 9)), int(rng.integers(0, 4)), int(rng.integers(0, 5)),
               4 * int(rng.integers(0, 4))) for _ in imgs]
    for border in ("valid", "replicate", "reflect101", "constant0"):
        for fmt in ("f32", "u8", "s16x4", "u16", "edge8"):
            res = run_batch(h, imgs, border, fmt, layout)
            for img, (got, guards) in zip(imgs, res):
                assert guards
                assert same_bits(got, oracle.sobel4(img, border, fmt)), (img.shape, border, fmt)


def test_batch_of_one_and_shared_input(h):
    img = synth.rects_noise(200, 300, 5)
    (got, guards), = run_batch(h, [img], "replicate", "f32")
    assert guards and same_bits(got, oracle.sobel4(img, "replicate", "f32"))
    # the same input read by two images of one batch is allowed
    s = Placed(torch, img, 300, 0)
    o1 = Output(torch, 200, 300, "u8", 300, 0)
    o2 = Output(torch, 200, 300, "u8", 300, 0)
    descs = [pkg.Image(s.ptr, 300, o1.ptr, 300, 200, 300), pkg.Image(s.ptr, 300, o2.ptr, 300, 200, 300)]
    assert pkg.sobel4_run_batched(h, descs, 0, 1, torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    want = oracle.sobel4(img, "valid", "u8")
    assert same_bits(o1.read()[0], want) and same_bits(o2.read()[0], want)


def test_back_to_back_batches_reuse_slots(h):
    """More batches in flight than descriptor slots: results must not mix."""
    imgs = [synth.uniform(50 + 7 * i, 60 + 11 * i, i) for i in range(6)]
    outs = []
    keep = []
    stream = torch.cuda.current_stream().cuda_stream
    for k in range(10):
        img = imgs[k % len(imgs)]
        s = Placed(torch, img, img.shape[1], 0)
        o = Output(torch, img.shape[0], img.shape[1], "f32", img.shape[1] * 4, 0)
        keep.append(s)
        outs.append((img, o))
        assert pkg.sobel4_run_batched(h, [pkg.Image(s.ptr, s.pitch, o.ptr, o.pitch, *img.shape)],
                                      0, 0, stream) == 0
    torch.cuda.synchronize()
    for img, o in outs:
        got, guards = o.read()
        assert guards and same_bits(got, oracle.sobel4(img))


def test_mixed_staging_batch_all_modes(h):
    """Images with 16-byte aligned rows (TMA-staged batch kernel) and tight rows
    (lane-copy batch kernel) in one call: every border rule and format."""
    rng = np.random.default_rng(11)
    shapes = [(int(a), int(b)) for a, b in rng.integers(3, 300, size=(14, 2))]
    shapes += [(700, 1300), (129, 257), (37, 128), (300, 640)]
    imgs = [synth.rects_noise(a, b, 40 + i) for i, (a, b) in enumerate(shapes)]
    layout = []
    for i, (H, W) in enumerate(shapes):
        if i % 2 == 0:
            layout.append(((-W) % 16, 0, (-W) % 4, 0))          # aligned source and output rows
        else:
            layout.append((int(rng.integers(0, 5)), int(rng.integers(0, 3)), 1, 4))
    for border in ("valid", "replicate", "reflect101", "constant0"):
        for fmt in ("f32", "u8", "s16x4"):
            res = run_batch(h, imgs, border, fmt, layout)
            for img, (got, guards) in zip(imgs, res):
                assert guards, (img.shape, border, fmt)
                assert same_bits(got, oracle.sobel4(img, border, fmt)), (img.shape, border, fmt)


def test_aligned_frames_batch_like_serving(h):
    """A batch of serving-sized frames (all rows 16-byte aligned) against the oracle."""
    sizes = [(480, 640), (720, 1280), (1080, 1920), (480, 640), (2160, 3840), (720, 1280)]
    imgs = [synth.rects_noise(a, b, 60 + i) for i, (a, b) in enumerate(sizes)]
    res = run_batch(h, imgs, "valid", "f32")
    for img, (got, guards) in zip(imgs, res):
        assert guards
        assert same_bits(got, oracle.sobel4(img, "valid", "f32", threads=NCPU)), img.shape
