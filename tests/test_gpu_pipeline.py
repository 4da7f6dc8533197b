"""The graph-captured video pipeline: every frame that streams through the
slots comes out equal to the oracle, frames of different slots overlap, and a
slot cannot be resubmitted before it is waited for."""
import numpy as np
import pytest

import oracle
import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import same_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fmt,border", [("f32", "valid"), ("u8", "replicate"),
                                        ("s16x4", "reflect101")])
def test_pipeline_frames_match_oracle(fmt, border):
    H, W = 130, 333
    bg = synth.video_background(H, W, 5)
    frames = [synth.video_frame(bg, k, H, W, 5) for k in range(9)]
    with pkg.Sobel4(0) as s:
        n0 = s.launches
        pipe = pkg.Pipeline(s, H, W, border, fmt, slots=3)
        assert s.launches == n0  # capture is not a launch
        results = {}
        for k, frame in enumerate(frames):
            slot = k % 3
            pipe.wait(slot)
            if k >= 3:
                results[k - 3] = pipe.outputs[slot].copy()
            pipe.inputs[slot][:] = frame
            pipe.submit(slot)
            if k == 0:
                with pytest.raises(pkg.Sobel4Error):
                    pipe.submit(slot)  # not waited for
        for k in range(len(frames) - 3, len(frames)):
            pipe.wait(k % 3)
            results[k] = pipe.outputs[k % 3].copy()
        assert s.launches == n0 + len(frames)
        pipe.close()
    for k, frame in enumerate(frames):
        assert same_bits(results[k], oracle.sobel4(frame, border, fmt)), k


def test_pipeline_rejects_bad_arguments():
    with pkg.Sobel4(0) as s:
        st, p = pkg.sobel4_pipeline_create(s.handle, 10, 10, 0, 0, 1)
        assert st == 1 and not p.value
        st, p = pkg.sobel4_pipeline_create(s.handle, 10, 10, 0, 0, 2)
        assert st == 0
        assert pkg.sobel4_pipeline_submit(p, 5) == 1
        assert pkg.sobel4_pipeline_wait(p, -1) == 1
        assert pkg.sobel4_pipeline_destroy(p) == 0
