"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds none of the operator's arithmetic: it only draws images and
workloads.  Both the CUDA path and the CPU oracle receive the same arrays from
here.  The paper evaluates on natural 8-bit grayscale photographs at 512^2,
1024^2 and 2048^2 (Section 5.2); those images are not available, so these
generators stand in for them with the same size, dtype and edge structure.

Recipes
-------
rects_noise(H, W, seed)
    Background of one uniform intensity U{0..255}; 40 filled rectangles painted
    in order (20 axis-aligned, then 20 rotated by an angle U[0, pi)), centre
    uniform over the image, sides U[W/32, W/4] x U[H/32, H/4], fill U{0..255},
    painted where the pixel centre (x + 0.5, y + 0.5) lies inside; then
    additive Gaussian noise N(0, 8^2), rounded half-to-even and clamped to
    [0, 255].
uniform(H, W, seed)
    i.i.d. U{0..255} pixels (worst-case gradients).
ragged_shapes(n, seed)
    n (H, W) pairs, each side independently U{37..2048}.
video_background / video_frame
    A (H+12) x (W+16) rects_noise background; frame k is its crop at offset
    (k mod 17, 2k mod 13) plus fresh N(0, 8^2) noise keyed by (seed, k).
video_frames_torch(bg, first, count, H, W, seed, device)
    The same translation schedule with the noise drawn on a torch device
    (one seeded generator per frame: (seed, k)), for streaming thousands of
    distinct frames without a CPU noise pass; returns a (count, H, W) uint8
    tensor on `device`.
serving_trace(rate, duration, seed)
    Poisson arrival times and a resolution per request drawn from
    {640x480: 40%, 1280x720: 30%, 1920x1080: 20%, 3840x2160: 10%}.
"""
from __future__ import annotations

import math

import numpy as np

SERVING_MIX = ((480, 640, 0.4), (720, 1280, 0.3), (1080, 1920, 0.2), (2160, 3840, 0.1))


def _rng(*keys: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(k) for k in keys])))


def _paint_rect(img: np.ndarray, cx, cy, w, h, theta, value) -> None:
    H, W = img.shape
    c, s = math.cos(theta), math.sin(theta)
    ex = abs(c) * w / 2 + abs(s) * h / 2
    ey = abs(s) * w / 2 + abs(c) * h / 2
    x0, x1 = max(0, int(math.floor(cx - ex))), min(W, int(math.ceil(cx + ex)) + 1)
    y0, y1 = max(0, int(math.floor(cy - ey))), min(H, int(math.ceil(cy + ey)) + 1)
    if x0 >= x1 or y0 >= y1:
        return
    py = (np.arange(y0, y1, dtype=np.float64) + 0.5 - cy)[:, None]
    px = (np.arange(x0, x1, dtype=np.float64) + 0.5 - cx)[None, :]
    u = px * c + py * s
    v = -px * s + py * c
    inside = (np.abs(u) <= w / 2) & (np.abs(v) <= h / 2)
    img[y0:y1, x0:x1][inside] = value


def rects(H: int, W: int, seed: int, n_axis: int = 20, n_rot: int = 20) -> np.ndarray:
    """The noise-free rectangles image of rects_noise."""
    rng = _rng(seed, 1)
    img = np.full((H, W), rng.integers(0, 256), dtype=np.uint8)
    for r in range(n_axis + n_rot):
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        w = rng.uniform(W / 32, W / 4)
        h = rng.uniform(H / 32, H / 4)
        theta = 0.0 if r < n_axis else rng.uniform(0, math.pi)
        _paint_rect(img, cx, cy, w, h, theta, rng.integers(0, 256))
    return img


def add_noise(img: np.ndarray, rng: np.random.Generator, sigma: float = 8.0) -> np.ndarray:
    noise = rng.standard_normal(img.shape, dtype=np.float32)
    noise *= np.float32(sigma)
    noise += img
    np.rint(noise, out=noise)
    np.clip(noise, 0, 255, out=noise)
    return noise.astype(np.uint8)


def rects_noise(H: int, W: int, seed: int, sigma: float = 8.0) -> np.ndarray:
    return add_noise(rects(H, W, seed), _rng(seed, 2), sigma)


def uniform(H: int, W: int, seed: int) -> np.ndarray:
    return _rng(seed, 3).integers(0, 256, size=(H, W), dtype=np.uint8)


def ragged_shapes(n: int, seed: int, lo: int = 37, hi: int = 2048):
    rng = _rng(seed, 4)
    hw = rng.integers(lo, hi + 1, size=(n, 2))
    return [(int(h), int(w)) for h, w in hw]


def batch_images(n: int = 512, seed: int = 1, lo: int = 37, hi: int = 2048):
    """The ragged batch: image i is rects_noise of its own shape with sub-seed (seed, i)."""
    return [rects_noise(h, w, seed * 100003 + i) for i, (h, w) in
            enumerate(ragged_shapes(n, seed, lo, hi))]


def video_background(H: int, W: int, seed: int) -> np.ndarray:
    return rects(H + 12, W + 16, seed)


def video_offset(k: int):
    return (k % 17, (2 * k) % 13)


def video_frame(bg: np.ndarray, k: int, H: int, W: int, seed: int,
                sigma: float = 8.0) -> np.ndarray:
    dx, dy = video_offset(k)
    crop = bg[dy:dy + H, dx:dx + W]
    return add_noise(crop, _rng(seed, 5, k), sigma)


def video_frames_torch(bg: np.ndarray, first: int, count: int, H: int, W: int, seed: int,
                       device="cuda", sigma: float = 8.0):
    import torch
    bgt = torch.from_numpy(bg).to(device=device, dtype=torch.float32)
    out = torch.empty((count, H, W), dtype=torch.uint8, device=device)
    g = torch.Generator(device=device)
    for i in range(count):
        k = first + i
        dx, dy = video_offset(k)
        g.manual_seed(int(seed) * 1000003 + k)
        noise = torch.randn((H, W), generator=g, device=device, dtype=torch.float32)
        noise.mul_(sigma).add_(bgt[dy:dy + H, dx:dx + W])
        out[i] = noise.round_().clamp_(0, 255).to(torch.uint8)
    return out


def serving_trace(rate: float = 400.0, duration: float = 60.0, seed: int = 4):
    """Arrival times (s) and (H, W) per request of a Poisson stream."""
    rng = _rng(seed, 6)
    n_max = int(rate * duration * 1.5 + 100)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_max))
    t = t[t < duration]
    probs = np.array([p for (_, _, p) in SERVING_MIX])
    idx = rng.choice(len(SERVING_MIX), size=len(t), p=probs)
    shapes = [(SERVING_MIX[i][0], SERVING_MIX[i][1]) for i in idx]
    return t, shapes
