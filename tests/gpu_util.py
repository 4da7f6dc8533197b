"""Helpers for the GPU parity tests: place images at arbitrary pitches and byte
offsets in device buffers surrounded by guard bytes, run the library through
its C ABI, and read the result back."""
from __future__ import annotations

import numpy as np

import paper_2305_00515_gb300 as pkg

GUARD = 0xA5


def same_bits(a, b) -> bool:
    """Element-by-element equality of the stored bits (so -0.0 and +0.0, equal
    as numbers, differ here): the parity bar is 0 mismatched elements."""
    a, b = np.asarray(a), np.asarray(b)
    if a.shape != b.shape or a.dtype != b.dtype:
        return False
    if a.dtype.kind == "f":
        u = {2: np.uint16, 4: np.uint32, 8: np.uint64}[a.dtype.itemsize]
        return bool(np.array_equal(np.ascontiguousarray(a).view(u), np.ascontiguousarray(b).view(u)))
    return bool(np.array_equal(a, b))
ELEM = {"f32": 4, "u8": 1, "s16x4": 2, "u16": 2, "edge8": 1}
DTYPE = {"f32": np.float32, "u8": np.uint8, "s16x4": np.int16, "u16": np.uint16,
         "edge8": np.uint8}


class Placed:
    """A host array copied into a guarded device buffer at (offset, pitch)."""

    def __init__(self, torch, img: np.ndarray, pitch: int, offset: int, device="cuda:0"):
        H, W = img.shape
        self.H, self.W, self.pitch, self.offset = H, W, pitch, offset
        host = np.full(offset + H * pitch + 64, GUARD, dtype=np.uint8)
        rows = host[offset:offset + H * pitch].reshape(H, pitch)
        rows[:, :W] = img
        self.buf = torch.from_numpy(host).to(device)
        self.ptr = self.buf.data_ptr() + offset


class Output:
    """A guarded device output buffer in format `fmt` at (offset, pitch)."""

    def __init__(self, torch, H: int, W: int, fmt: str, pitch: int, offset: int, device="cuda:0"):
        self.H, self.W, self.fmt, self.pitch, self.offset = H, W, fmt, pitch, offset
        self.planes = 4 if fmt == "s16x4" else 1
        n = offset + self.planes * H * pitch + 64
        self.buf = torch.full((n,), GUARD, dtype=torch.uint8, device=device)
        self.ptr = self.buf.data_ptr() + offset

    def read(self):
        """(dense result, True if every byte outside the payload still holds the guard)."""
        host = self.buf.cpu().numpy()
        body = host[self.offset:self.offset + self.planes * self.H * self.pitch]
        body = body.reshape(self.planes * self.H, self.pitch)
        nbytes = self.W * ELEM[self.fmt]
        payload = np.ascontiguousarray(body[:, :nbytes]).view(DTYPE[self.fmt])
        payload = payload.reshape((4, self.H, self.W) if self.planes == 4 else (self.H, self.W))
        mask = np.ones(host.shape, dtype=bool)
        region = mask[self.offset:self.offset + self.planes * self.H * self.pitch]
        region.reshape(self.planes * self.H, self.pitch)[:, :nbytes] = False
        guards_ok = bool(np.all(host[mask] == GUARD))
        return payload, guards_ok


def default_pitches(W: int, fmt: str):
    return W, W * ELEM[fmt]


def run_placed(torch, h, img, border="valid", fmt="f32", src_pitch=None, src_offset=0,
               dst_pitch=None, dst_offset=0, stream=None):
    H, W = img.shape
    sp0, dp0 = default_pitches(W, fmt)
    src = Placed(torch, img, src_pitch or sp0, src_offset)
    out = Output(torch, H, W, fmt, dst_pitch or dp0, dst_offset)
    st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = pkg.sobel4_run(h, src.ptr, src.pitch, out.ptr, out.pitch, H, W, pkg.BORDERS[border],
                        pkg.FORMATS[fmt], st)
    assert rc == 0, pkg.sobel4_status_string(rc)
    torch.cuda.synchronize()
    return out.read()
