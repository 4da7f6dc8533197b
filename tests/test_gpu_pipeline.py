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


def test_pipeline_submit_from_caller_buffers():
    """Each frame from its own host buffer (pinned by cudaHostAlloc, or a numpy
    array registered with cudaHostRegister), results into caller buffers:
    pinned ones, which the kernel writes itself, and one pageable buffer,
    which gets the staged kernel and a download."""
    H, W = 120, 256
    bg = synth.video_background(H, W, 8)
    frames = [synth.video_frame(bg, k, H, W, 8) for k in range(6)]
    pinned_in = [torch.from_numpy(f).pin_memory() for f in frames[:3]]
    ring = np.stack(frames[3:])  # registered page-locked numpy memory
    cudart = torch.cuda.cudart()
    assert int(cudart.cudaHostRegister(ring.ctypes.data, ring.nbytes, 0)) == 0
    outs = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in frames]
    outs[4] = torch.full((H, W), 7.0)  # pageable: the kernel graph and a download
    try:
        with pkg.Sobel4(0) as s:
            pipe = pkg.Pipeline(s, H, W, "valid", "f32", slots=2)
            for k in range(len(frames)):
                slot = k % 2
                pipe.wait(slot)
                src = pinned_in[k].data_ptr() if k < 3 else ring.ctypes.data + (k - 3) * H * W
                st = pkg.sobel4_pipeline_submit_from(pipe.p, slot, src, outs[k].data_ptr())
                assert st == 0, (k, pkg.sobel4_last_cuda_error(s.handle))
            for slot in range(2):
                pipe.wait(slot)
            # back to the slot's own buffers
            pipe.inputs[0][:] = frames[0]
            pipe.submit(0)
            pipe.wait(0)
            own = pipe.outputs[0].copy()
            pipe.close()
    finally:
        cudart.cudaHostUnregister(ring.ctypes.data)
    for k, frame in enumerate(frames):
        assert same_bits(outs[k].numpy(), oracle.sobel4(frame, "valid", "f32")), k
    assert same_bits(own, oracle.sobel4(frames[0], "valid", "f32"))


def test_host_alloc_ring_through_the_pipeline():
    """A frame ring and result buffers in sobel4_host_alloc memory: every
    frame equals the oracle; the allocator rejects a zero size and frees NULL."""
    H, W, n = 96, 256, 5  # rows at the pipeline pitches (multiples of 16 bytes)
    bg = synth.video_background(H, W, 12)
    frames = [synth.video_frame(bg, k, H, W, 12) for k in range(n)]
    ring = pkg.HostBuffer((n, H, W), "uint8")
    outs = pkg.HostBuffer((n, H, W), "float32")
    try:
        ring.array[:] = np.stack(frames)
        with pkg.Sobel4(0) as s:
            pipe = pkg.Pipeline(s, H, W, "replicate", "f32", slots=3)
            for k in range(n):
                pipe.wait(k % 3)
                pipe.submit_from(k % 3, ring.address + k * H * W, outs.address + k * H * W * 4)
            for slot in range(3):
                pipe.wait(slot)
            pipe.close()
        for k in range(n):
            assert same_bits(outs.array[k], oracle.sobel4(frames[k], "replicate", "f32")), k
    finally:
        ring.close()
        outs.close()
    assert pkg.sobel4_host_alloc(0)[0] == 1
    assert pkg.sobel4_host_free(0) == 0


def test_pipeline_4k_frames():
    """3840x2160 frames, the video configuration's size, through the pipeline."""
    H, W = 2160, 3840
    bg = synth.video_background(H, W, 3)
    ks = (0, 1, 17, 220)
    frames = {k: synth.video_frame(bg, k, H, W, 3) for k in ks}
    with pkg.Sobel4(0) as s:
        pipe = pkg.Pipeline(s, H, W, "valid", "f32", slots=2)
        got = {}
        for i, k in enumerate(ks):
            slot = i % 2
            pipe.wait(slot)
            if i >= 2:
                got[ks[i - 2]] = pipe.outputs[slot].copy()
            pipe.inputs[slot][:] = frames[k]
            pipe.submit(slot)
        for i in range(len(ks) - 2, len(ks)):
            pipe.wait(i % 2)
            got[ks[i]] = pipe.outputs[i % 2].copy()
        pipe.close()
    for k in ks:
        want = oracle.sobel4(frames[k], "valid", "f32", threads=oracle.cpu_count())
        assert same_bits(got[k], want), k
