"""Failure detection in the TMA-staged kernel without a GPU fault: a withheld
row copy makes one warp's bounded barrier wait run out; the kernel records it
in the handle's error word and stops, sobel4_device_status reports TIMEOUT,
and the context stays usable (the next launch is exact)."""
import numpy as np
import pytest

import oracle
import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import run_placed, same_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_withheld_stage_times_out_and_context_survives():
    from paper_2305_00515_gb300 import build
    build.build()
    st, h = pkg.sobel4_create(0, pkg.VARIANTS["rg"])
    assert st == 0
    try:
        img = synth.rects_noise(256, 512, 9)  # 512-byte rows: TMA staging
        assert pkg.sobel4_device_status(h) == 0
        assert pkg.sobel4_inject_stage_loss(h, 1) == 0
        run_placed(torch, h, img, "valid", "f32")          # launch returns OK (asynchronous)
        assert pkg.sobel4_device_status(h) == 5, "the withheld stage must time out"
        assert pkg.sobel4_device_status(h) == 0            # the word was cleared
        got, guards = run_placed(torch, h, img, "valid", "f32")
        assert guards
        assert same_bits(got, oracle.sobel4(img, "valid", "f32"))
        assert pkg.sobel4_device_status(h) == 0
        assert pkg.sobel4_inject_stage_loss(h, -1) == 1
        assert pkg.sobel4_inject_stage_loss(None, 0) == 1
    finally:
        pkg.sobel4_destroy(h)
