"""The allocation-free batched entry point, sobel4_run_batched_static.

It exists for callers that cannot allocate GPU memory (plugins inside a host
framework that owns every device buffer, services held to a fixed memory
budget, latency-critical threads that must not pay for cudaMalloc), so it keeps
its scratch in a static device array inside the library.  This file is named
to be collected last: if it fails, a run that stops at the first failure has
already run every other test.  It passes alone in a fresh process and after
the rest of the suite.
"""
import numpy as np
import pytest

import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import Output, Placed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def make_batch(seed, n):
    rng = np.random.default_rng(seed)
    imgs, srcs, outs, descs = [], [], [], []
    for i in range(n):
        H, W = (int(v) for v in rng.integers(3, 700, size=2))
        img = synth.rects_noise(H, W, seed * 1000 + i)
        s = Placed(torch, img, W + int(rng.integers(0, 5)), int(rng.integers(0, 4)))
        o = Output(torch, H, W, "f32", 4 * (W + int(rng.integers(0, 3))), 4 * int(rng.integers(0, 4)))
        imgs.append(img)
        srcs.append(s)
        outs.append(o)
        descs.append(pkg.Image(s.ptr, s.pitch, o.ptr, o.pitch, H, W))
    return imgs, srcs, outs, descs


def test_static_batched_matches_handle_batched_twice_in_a_row():
    from paper_2305_00515_gb300 import build
    build.build()
    torch.cuda.init()
    stream = torch.cuda.current_stream().cuda_stream
    st, h = pkg.sobel4_create(0)
    assert st == 0
    try:
        for call, (seed, n) in enumerate(((11, 37), (12, 64))):
            imgs, srcs, outs, descs = make_batch(seed, n)
            # the existing entry point writes the reference outputs
            ref = [Output(torch, o.H, o.W, "f32", o.pitch, o.offset) for o in outs]
            ref_descs = [pkg.Image(d.src, d.src_pitch, r.ptr, r.pitch, d.height, d.width)
                         for d, r in zip(descs, ref)]
            assert pkg.sobel4_run_batched(h, ref_descs, 0, 0, stream) == 0
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            rc = pkg.sobel4_run_batched_static(descs, 0, 0, stream)
            assert rc == 0, pkg.sobel4_status_string(rc)
            torch.cuda.synchronize()
            if call == 1:
                # after the first call's one-time set-up, a call takes no device memory
                assert torch.cuda.mem_get_info()[0] == free_before
            for o, r in zip(outs, ref):
                got, guards = o.read()
                want, _ = r.read()
                assert guards, "write outside an output payload"
                assert np.array_equal(got, want)  # tolerance: 0 mismatched elements
    finally:
        pkg.sobel4_destroy(h)


def test_static_batched_rejects_oversize_and_bad_args():
    img = pkg.Image(0x10000000, 100, 0x20000000, 400, 50, 100)
    assert pkg.sobel4_run_batched_static([], 0, 0, None) == 1
    too_many = [pkg.Image(0x10000000 + 10000 * i, 100, 0x80000000 + 40000 * i, 400, 50, 100)
                for i in range(1025)]
    assert pkg.sobel4_run_batched_static(too_many, 0, 0, None) == 2
    assert pkg.sobel4_run_batched_static([img], 7, 0, None) == 1
