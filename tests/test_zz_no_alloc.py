"""The allocation-free batched entry point, sobel4_run_batched_static.

It exists for callers that cannot allocate GPU memory (plugins inside a host
framework that owns every device buffer, services held to a fixed memory
budget, latency-critical threads that must not pay for cudaMalloc), so it keeps
its scratch in a static device array inside the library.  Every output is
compared element by element with the CPU oracle (tolerance: 0 mismatched
elements) and with the handle-based sobel4_run_batched.  This file is named to
be collected last: if it fails, a run that stops at the first failure has
already run every other test.  It passes alone in a fresh process and after
the rest of the suite.
"""
import numpy as np
import pytest

import oracle
import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import ELEM, Output, Placed, same_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# descriptors per parameter upload launch (31744-byte blocks of 64-byte descriptors)
UPLOAD_CHUNK = 496


def make_batch(seed, n, lo, hi, fmt="f32"):
    rng = np.random.default_rng(seed)
    imgs, srcs, outs, descs = [], [], [], []
    e = ELEM[fmt]
    for i in range(n):
        H, W = (int(v) for v in rng.integers(lo, hi + 1, size=2))
        img = synth.rects_noise(H, W, seed * 1000 + i)
        s = Placed(torch, img, W + int(rng.integers(0, 5)), int(rng.integers(0, 4)))
        o = Output(torch, H, W, fmt, e * (W + int(rng.integers(0, 3))), e * int(rng.integers(0, 4)))
        imgs.append(img)
        srcs.append(s)
        outs.append(o)
        descs.append(pkg.Image(s.ptr, s.pitch, o.ptr, o.pitch, H, W))
    return imgs, srcs, outs, descs


def run_and_compare(h, imgs, outs, descs, border, fmt, stream):
    """Runs the static entry point, then sobel4_run_batched into fresh buffers,
    and checks every image against the oracle and the two runs against each other."""
    b, f = pkg.BORDERS[border], pkg.FORMATS[fmt]
    ref = [Output(torch, o.H, o.W, fmt, o.pitch, o.offset) for o in outs]
    ref_descs = [pkg.Image(d.src, d.src_pitch, r.ptr, r.pitch, d.height, d.width)
                 for d, r in zip(descs, ref)]
    rc = pkg.sobel4_run_batched_static(descs, b, f, stream)
    assert rc == 0, pkg.sobel4_status_string(rc)
    assert pkg.sobel4_run_batched(h, ref_descs, b, f, stream) == 0
    torch.cuda.synchronize()
    for img, o, r in zip(imgs, outs, ref):
        got, guards = o.read()
        assert guards, "write outside an output payload"
        want = oracle.sobel4(img, border, fmt)
        assert same_bits(got, want), f"{img.shape} {border} {fmt} differs from the oracle"
        other, _ = r.read()
        assert same_bits(got, other)


@pytest.fixture(scope="module")
def handle():
    from paper_2305_00515_gb300 import build
    build.build()
    torch.cuda.init()
    st, h = pkg.sobel4_create(0)
    assert st == 0
    yield h
    pkg.sobel4_destroy(h)


def test_static_batched_matches_oracle_twice_in_a_row(handle):
    stream = torch.cuda.current_stream().cuda_stream
    for call, (seed, n) in enumerate(((11, 37), (12, 64))):
        imgs, srcs, outs, descs = make_batch(seed, n, 3, 700)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = pkg.sobel4_run_batched_static(descs, 0, 0, stream)
        assert rc == 0, pkg.sobel4_status_string(rc)
        torch.cuda.synchronize()
        if call == 1:
            # after the first call on the device, a call takes no device memory
            assert torch.cuda.mem_get_info()[0] == free_before
        for img, o in zip(imgs, outs):
            got, guards = o.read()
            assert guards, "write outside an output payload"
            assert same_bits(got, oracle.sobel4(img, "valid", "f32"))  # 0 mismatches
    run_and_compare(handle, imgs, outs, descs, "valid", "f32", stream)


@pytest.mark.parametrize("fmt", ["f32", "u8", "s16x4"])
@pytest.mark.parametrize("border", ["valid", "replicate", "reflect101", "constant0"])
def test_static_batched_every_border_and_format(handle, border, fmt):
    seed = 100 + 10 * pkg.BORDERS[border] + pkg.FORMATS[fmt]
    imgs, srcs, outs, descs = make_batch(seed, 12, 3, 200, fmt)
    run_and_compare(handle, imgs, outs, descs, border, fmt,
                    torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("n", [UPLOAD_CHUNK + 1, 1024])
def test_static_batched_several_uploads_and_the_cap(handle, n):
    # n = 497 needs two descriptor uploads (the second starts one image in);
    # n = 1024 is the largest batch the static array holds.
    imgs, srcs, outs, descs = make_batch(200 + n, n, 3, 64)
    run_and_compare(handle, imgs, outs, descs, "replicate", "f32",
                    torch.cuda.current_stream().cuda_stream)


def test_static_batched_rejects_oversize_and_bad_args():
    img = pkg.Image(0x10000000, 100, 0x20000000, 400, 50, 100)
    assert pkg.sobel4_run_batched_static([], 0, 0, None) == 1
    too_many = [pkg.Image(0x10000000 + 10000 * i, 100, 0x80000000 + 40000 * i, 400, 50, 100)
                for i in range(1025)]
    assert pkg.sobel4_run_batched_static(too_many, 0, 0, None) == 2
    assert pkg.sobel4_run_batched_static([img], 7, 0, None) == 1
    assert pkg.sobel4_run_batched_static([img], 0, pkg.FORMATS["u16"], None) == 2
    # overlapping outputs are rejected before anything is enqueued
    twin = [img, pkg.Image(0x30000000, 100, 0x20000000 + 400, 400, 50, 100)]
    assert pkg.sobel4_run_batched_static(twin, 0, 0, None) == 1
