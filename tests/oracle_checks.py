"""Pins for the CPU oracle: checks against what the paper and the mathematics fix.

Each check takes an ``oracle.Oracle`` instance and raises AssertionError on a
mismatch.  ``test_oracle_pins.py`` runs them on the committed oracle;
``test_oracle_mutants.py`` runs them on copies of the oracle with a planted
mistake and requires that some check fails for every mistake.

None of these checks re-derives a value through the oracle's own tables or
loops: the references are the paper's other statements of the operator
(Eq. 5, 10, 11, 12-19), closed forms, symmetry laws, hand-enumerated fixtures,
scipy's N-D correlation, numpy's IEEE single-precision square root, and exact
rational arithmetic.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np

from factored_reference import factored_responses

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BORDERS = ("valid", "replicate", "reflect101", "constant0")


# ----------------------------------------------------------------------------
# Eq. (5) and the identities of Section 4.3.5, written from the paper.
# ----------------------------------------------------------------------------
def eq5_masks(a=1, b=2, m=6, n=4) -> np.ndarray:
    """K_x, K_y, K_d, K_dt of Eq. (5) (Section 3.2)."""
    col = np.array([1, n, m, n, 1])
    dif = np.array([-1, -b, 0, b, 1])
    Kx = a * np.outer(col, dif)
    Ky = a * np.outer(dif, col)
    Kd = a * np.array([[-m, -n, -1, -b, 0],
                       [-n, -m * b, -n * b, 0, b],
                       [-1, -n * b, 0, n * b, 1],
                       [-b, 0, n * b, m * b, n],
                       [0, b, 1, n, m]])
    Kdt = a * np.array([[0, -b, -1, -n, -m],
                        [b, 0, -n * b, -m * b, -n],
                        [1, n * b, 0, -n * b, -1],
                        [n, m * b, n * b, 0, -b],
                        [m, n, 1, b, 0]])
    return np.stack([Kx, Ky, Kd, Kdt])


def eq10_kd_plus_minus(a=1, b=2, m=6, n=4):
    """K_d+ and K_d- as printed in Eq. (10)."""
    kp = a * np.array([[-m, -n - b, -2, -n - b, -m],
                       [b - n, -m * b, -2 * n * b, -m * b, b - n],
                       [0, 0, 0, 0, 0],
                       [n - b, m * b, 2 * n * b, m * b, n - b],
                       [m, n + b, 2, n + b, m]])
    km = a * np.array([[-m, b - n, 0, n - b, m],
                       [-n - b, -m * b, 0, m * b, n + b],
                       [-2, -2 * n * b, 0, 2 * n * b, 2],
                       [-n - b, -m * b, 0, m * b, n + b],
                       [-m, b - n, 0, n - b, m]])
    return kp, km


def eq18_kd_minus(a=1, b=2, m=6, n=4):
    """K_d- rebuilt from the two outer products of Eq. (18)."""
    u1 = np.array([m, n + b, 2, n + b, m])
    v1 = np.array([-1, -b, 0, b, 1])
    u2 = np.array([m * b + b - n, n * b + b * b - m * b, 2 * b - 2 * n * b,
                   n * b + b * b - m * b, m * b - n + b])
    v2 = np.array([0, -1, 0, 1, 0])
    return a * (np.outer(u1, v1) - np.outer(u2, v2))


# ----------------------------------------------------------------------------
# Independent evaluations.
# ----------------------------------------------------------------------------
def scipy_responses(img: np.ndarray, border: str, K: np.ndarray) -> np.ndarray:
    """R_k by scipy.ndimage.correlate (the library's N-D correlation)."""
    import scipy.ndimage as ndi
    mode = {"valid": "nearest", "replicate": "nearest", "reflect101": "mirror",
            "constant0": "constant"}[border]
    I = img.astype(np.int64)
    out = np.stack([ndi.correlate(I, K[k].astype(np.int64), mode=mode, cval=0)
                    for k in range(4)])
    if border == "valid":
        H, W = img.shape
        mask = np.zeros((H, W), dtype=bool)
        if H >= 5 and W >= 5:
            mask[2:H - 2, 2:W - 2] = True
        out = np.where(mask[None], out, 0)
    return out


def exact_sqrtf_ok(g: np.float32, s: int) -> bool:
    """True iff g is sqrt(float(s)) correctly rounded to fp32 (exact rationals)."""
    x = Fraction(float(np.float32(s)))           # int -> fp32, round-to-nearest-even
    g = np.float32(g)
    if x == 0:
        return g == 0
    lo = Fraction(float(np.nextafter(g, np.float32(-np.inf), dtype=np.float32)))
    hi = Fraction(float(np.nextafter(g, np.float32(np.inf), dtype=np.float32)))
    gf = Fraction(float(g))
    m_lo = (lo + gf) / 2
    m_hi = (gf + hi) / 2
    return m_lo * m_lo <= x <= m_hi * m_hi


def rng_image(seed: int, H: int, W: int) -> np.ndarray:
    return np.random.default_rng(seed).integers(0, 256, size=(H, W), dtype=np.uint8)


def read_golden(name: str):
    rows, expect, mode = [], [], None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line in ("image", "expect"):
                mode = line
                continue
            vals = [int(v) for v in line.split()]
            (rows if mode == "image" else expect).append(vals)
    return np.array(rows, dtype=np.uint8), expect


# ----------------------------------------------------------------------------
# The checks.
# ----------------------------------------------------------------------------
def check_masks_eq3_equal_eq5(o):
    K = o.masks()
    assert np.array_equal(K, eq5_masks(1, 2, 6, 4)), "Eq. (3) tables differ from Eq. (5) at (1,2,6,4)"


def check_mask_structure(o):
    K = o.masks()
    for k in range(4):
        assert np.count_nonzero(K[k]) == 20
        assert K[k].sum() == 0
        assert K[k][K[k] > 0].sum() == 48
        assert np.array_equal(K[k][::-1, ::-1], -K[k]), "masks are point-antisymmetric"
    assert np.array_equal(K[1], K[0].T)
    assert np.array_equal(K[2], K[2].T)
    assert np.array_equal(K[3], K[2][:, ::-1])


def check_kd_plus_minus(o):
    K = o.masks()
    kp, km = eq10_kd_plus_minus()
    assert np.array_equal(K[2] + K[3], kp)
    assert np.array_equal(K[2] - K[3], km)
    assert np.array_equal(eq18_kd_minus(), km)


def check_constant_image(o):
    for v in (0, 1, 137, 255):
        img = np.full((9, 11), v, dtype=np.uint8)
        for border in BORDERS:
            R = o.responses(img, border)
            if border == "constant0":
                R = R[:, 2:-2, 2:-2]
            assert not R.any(), f"constant image gave a response ({border}, v={v})"
            G = o.sobel4(img, border, "f32")
            if border == "constant0":
                G = G[2:-2, 2:-2]
            assert not G.any()


def check_ramp_closed_form(o):
    H, W = 12, 14
    yy, xx = np.mgrid[0:H, 0:W]
    for (al, be, ga) in ((1, 0, 10), (0, 1, 30), (3, -2, 100), (-4, 5, 120), (2, 3, 0)):
        img = (al * xx + be * yy + ga).astype(np.int64)
        assert img.min() >= 0 and img.max() <= 255
        img = img.astype(np.uint8)
        want = np.array([128 * al, 128 * be, 96 * (al + be), 96 * (be - al)])
        for border in BORDERS:
            R = o.responses(img, border)[:, 2:H - 2, 2:W - 2]
            assert np.array_equal(R, np.broadcast_to(want[:, None, None], R.shape)), \
                f"ramp ({al},{be}) {border}"
        s = int((want ** 2).sum())
        assert s == 34816 * (al * al + be * be)
        G = o.sobel4(img, "valid", "f32")[2:H - 2, 2:W - 2]
        assert np.all(G == np.sqrt(np.float32(s)))
    G10 = o.sobel4(np.tile(np.arange(14, dtype=np.uint8), (9, 1)), "valid", "f32")
    assert G10[4, 6] == np.float32(np.sqrt(np.float32(34816)))


def check_impulse(o):
    img = np.zeros((9, 9), dtype=np.uint8)
    img[4, 4] = 1
    K = eq5_masks()
    R = o.responses(img, "valid")
    for k in range(4):
        assert np.array_equal(R[k, 2:7, 2:7], -K[k]), "impulse must return -K (correlation order)"
    S = (R.astype(np.int64) ** 2).sum(0)
    assert S[2, 2] == 38 and S[4, 4] == 0


def check_golden(o):
    for name in ("step_edge_7x7.txt", "diagonal_step_7x7.txt"):
        img, expect = read_golden(name)
        R = o.responses(img, "valid")
        G = o.sobel4(img, "valid", "f32")
        S16 = o.sobel4(img, "valid", "s16x4")
        for (y, x, rx, ry, rd, rdt, s) in expect:
            assert tuple(R[:, y, x]) == (rx, ry, rd, rdt), f"{name} at ({y},{x})"
            assert tuple(S16[:, y, x]) == (rx, ry, rd, rdt)
            assert G[y, x] == np.sqrt(np.float32(s))
            assert exact_sqrtf_ok(G[y, x], s)


def check_rotation_flip_transpose(o):
    for seed, (H, W) in enumerate(((9, 13), (16, 11), (7, 7))):
        I = rng_image(100 + seed, H, W)
        for border in BORDERS:
            R = o.responses(I, border).astype(np.int64)
            # 90-degree rotation: J[i][j] = I[j][W-1-i]
            Rj = o.responses(np.ascontiguousarray(np.rot90(I)), border).astype(np.int64)
            rot = lambda P: np.rot90(P)
            assert np.array_equal(Rj[0], rot(R[1]))
            assert np.array_equal(Rj[1], -rot(R[0]))
            assert np.array_equal(Rj[2], rot(R[3]))
            assert np.array_equal(Rj[3], -rot(R[2]))
            # horizontal flip
            Rf = o.responses(np.ascontiguousarray(I[:, ::-1]), border).astype(np.int64)
            fl = lambda P: P[:, ::-1]
            assert np.array_equal(Rf[0], -fl(R[0]))
            assert np.array_equal(Rf[1], fl(R[1]))
            assert np.array_equal(Rf[2], fl(R[3]))
            assert np.array_equal(Rf[3], fl(R[2]))
            # transpose
            Rt = o.responses(np.ascontiguousarray(I.T), border).astype(np.int64)
            assert np.array_equal(Rt[0], R[1].T)
            assert np.array_equal(Rt[1], R[0].T)
            assert np.array_equal(Rt[2], R[2].T)
            assert np.array_equal(Rt[3], -R[3].T)
            # magnitude is invariant under all three
            G = o.sobel4(I, border, "f32")
            assert np.array_equal(o.sobel4(np.ascontiguousarray(np.rot90(I)), border), np.rot90(G))
            assert np.array_equal(o.sobel4(np.ascontiguousarray(I[:, ::-1]), border), G[:, ::-1])


def check_inversion_linearity(o):
    I1 = rng_image(7, 10, 12) // 2
    I2 = rng_image(8, 10, 12) // 2
    for border in ("valid", "replicate", "reflect101"):
        R1 = o.responses(I1, border)
        assert np.array_equal(o.responses(255 - I1, border), -R1)
        assert np.array_equal(o.responses(I1 + I2, border), R1 + o.responses(I2, border))
    R1 = o.responses(I1, "constant0")
    assert np.array_equal(o.responses(I1 + I2, "constant0"), R1 + o.responses(I2, "constant0"))


def check_against_scipy(o):
    K = eq5_masks()
    cases = [(1, 1), (1, 7), (6, 1), (2, 2), (3, 3), (4, 6), (5, 5), (6, 4), (7, 9),
             (16, 16), (23, 37), (40, 33)]
    for idx, (H, W) in enumerate(cases):
        I = rng_image(1000 + idx, H, W)
        for border in BORDERS:
            if border == "reflect101" and (H < 3 or W < 3):
                continue
            R = o.responses(I, border).astype(np.int64)
            want = scipy_responses(I, border, K)
            assert np.array_equal(R, want), f"scipy mismatch {H}x{W} {border}"
            S = (want ** 2).sum(0)
            G = o.sobel4(I, border, "f32")
            assert np.array_equal(G, np.sqrt(S.astype(np.float32))), f"f32 {H}x{W} {border}"
            S16 = o.sobel4(I, border, "s16x4")
            assert np.array_equal(S16.astype(np.int64), want)


def check_against_factored(o):
    for idx, (H, W) in enumerate(((5, 5), (6, 9), (17, 23), (32, 40), (64, 37))):
        I = rng_image(2000 + idx, H, W)
        R = o.responses(I, "valid").astype(np.int64)[:, 2:H - 2, 2:W - 2]
        for variant in ("eq19", "eq17"):
            F = factored_responses(I, kd_minus=variant)
            assert np.array_equal(R, F), f"factored ({variant}) mismatch {H}x{W}"


def check_magnitude_rounding(o):
    rng = np.random.default_rng(5)
    specials = [0, 1, 2, 3, 4, 15, 16, 38, 34816, 65280, 65281, 2 ** 24 - 1, 2 ** 24, 2 ** 24 + 1,
                2 ** 24 + 3, 47540000, 599270400, 599270399, 452608, 255 * 255, 2 ** 26 + 5]
    values = specials + [int(v) for v in rng.integers(0, 599270401, size=3000)]
    for s in values:
        g = o.magnitude_f32(s)
        assert g == np.sqrt(np.float32(s)), f"sqrtf(float({s}))"
        assert exact_sqrtf_ok(g, s), f"not correctly rounded at {s}"


def check_u8_rule(o):
    rng = np.random.default_rng(6)
    values = list(range(0, 300)) + [65020, 65021, 65024, 65025, 65026, 65279, 65280, 65281,
                                    65282, 599270400] + \
        [int(v) for v in rng.integers(0, 70000, size=2000)] + [n * n + n for n in range(1, 256)] + \
        [n * n + n + 1 for n in range(1, 256)]
    for s in values:
        u = o.magnitude_u8(s)
        assert 0 <= u <= 255
        r = Fraction(s)
        if u < 255:
            lower = Fraction(2 * u - 1, 2) if u > 0 else Fraction(0)
            assert lower ** 2 <= r < (Fraction(2 * u + 1, 2)) ** 2, s
        else:
            assert r >= Fraction(509, 2) ** 2, s
    # u8 images agree with the rule applied to the f32 route's exact S
    I = rng_image(77, 20, 21)
    R = o.responses(I, "replicate").astype(np.int64)
    S = (R ** 2).sum(0)
    U = o.sobel4(I, "replicate", "u8")
    root = np.vectorize(math.isqrt)(S)
    want = np.minimum(255, root + (S > root * root + root))
    assert np.array_equal(U.astype(np.int64), want)


def check_pitched_rows_and_threads(o):
    I = rng_image(31, 37, 29)
    padded = np.zeros((37, 41), dtype=np.uint8)
    padded[:, :29] = I
    view = padded[:, :29]
    for border in BORDERS:
        G1 = o.sobel4(I, border, "f32")
        assert np.array_equal(o.sobel4(view, border, "f32"), G1)
        assert np.array_equal(o.sobel4(I, border, "f32", threads=4), G1)
        out = np.full((37, 35), 7.0, dtype=np.float32)
        o.run_into(I, out[:, :29], border, "f32")
        assert np.array_equal(out[:, :29], G1) and np.all(out[:, 29:] == 7.0)


def check_valid_frame(o):
    for (H, W) in ((1, 1), (4, 9), (9, 4), (5, 5), (8, 8)):
        I = rng_image(H * 100 + W, H, W)
        for fmt in ("f32", "u8", "s16x4"):
            G = o.sobel4(I, "valid", fmt)
            if fmt == "s16x4":
                G = np.abs(G).sum(0)
            if H < 5 or W < 5:
                assert not G.any()
            else:
                frame = np.ones((H, W), dtype=bool)
                frame[2:H - 2, 2:W - 2] = False
                assert not G[frame].any()


# -- grayscale input (the host preparation of Section 4.3; the rule is a reading) --
def check_rgb_gray_inputs_and_hand_values(o):
    # R = G = B = v gives v exactly: (256 v + 128) >> 8 = v
    v = np.arange(256, dtype=np.uint8)
    rgb = np.repeat(v[None, :, None], 3, axis=2)
    assert np.array_equal(o.rgb_to_gray(rgb)[0], v)
    # hand-computed pixels: Y = (77 R + 150 G + 29 B + 128) >> 8
    cases = {(255, 0, 0): 77,      # 19763 >> 8
             (0, 255, 0): 149,     # 38378 >> 8
             (0, 0, 255): 29,      # 7523 >> 8
             (10, 20, 30): 18,     # (770 + 3000 + 870 + 128) = 4768 >> 8
             (128, 64, 32): 80,    # (9856 + 9600 + 928 + 128) = 20512 >> 8
             (1, 1, 0): 1,         # 355 >> 8
             (0, 0, 1): 0,         # 157 >> 8
             (255, 255, 255): 255}  # 65408 >> 8
    px = np.array([list(k) for k in cases], dtype=np.uint8)[None]
    assert o.rgb_to_gray(px)[0].tolist() == list(cases.values())


def check_rgb_within_bt601(o):
    # every one of the 2^24 colours lies within 1 of the real-valued BT.601
    # luma 0.299 R + 0.587 G + 0.114 B (weight error <= 0.46, rounding <= 0.5)
    i = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(i >> 16) & 255, (i >> 8) & 255, i & 255], axis=1).astype(np.uint8)
    y = o.rgb_to_gray(rgb.reshape(4096, 4096, 3)).reshape(-1).astype(np.float64)
    real = 0.299 * rgb[:, 0] + 0.587 * rgb[:, 1] + 0.114 * rgb[:, 2]
    assert np.abs(y - real).max() < 1.0
    # monotone in each channel
    for c in range(3):
        lo = rgb.copy()
        lo[:, c] = np.minimum(lo[:, c], 254)
        hi = lo.copy()
        hi[:, c] += 1
        a = o.rgb_to_gray(lo[:1 << 20].reshape(1024, 1024, 3)).astype(int)
        b = o.rgb_to_gray(hi[:1 << 20].reshape(1024, 1024, 3)).astype(int)
        assert (b >= a).all()


def check_rgb_channel_steps(o):
    path = os.path.join(GOLDEN, "rgb_channel_steps_7x7.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")][1:]
    for ch, h, s in rows:
        c = "RGB".index(ch)
        rgb = np.zeros((7, 7, 3), dtype=np.uint8)
        rgb[:, 3:, c] = 255
        assert int(o.rgb_to_gray(rgb)[0, 3]) == int(h)
        G = o.sobel4_rgb(rgb, "valid", "f32")
        R = o.responses(o.rgb_to_gray(rgb), "valid")
        S = int((R[:, 3, 3].astype(np.int64) ** 2).sum())
        assert S == int(s), (ch, S)
        assert G[3, 3] == np.sqrt(np.float32(int(s)))
    # a grey RGB image gives the operator of its grey values
    img = rng_image(5, 23, 31)
    rgb = np.repeat(img[:, :, None], 3, axis=2)
    for border in ("valid", "replicate"):
        assert np.array_equal(o.sobel4_rgb(rgb, border, "f32").view(np.uint32),
                              o.sobel4(img, border, "f32").view(np.uint32))


ALL_CHECKS = [
    check_masks_eq3_equal_eq5, check_mask_structure, check_kd_plus_minus, check_constant_image,
    check_ramp_closed_form, check_impulse, check_golden, check_rotation_flip_transpose,
    check_inversion_linearity, check_against_scipy, check_against_factored,
    check_magnitude_rounding, check_u8_rule, check_pitched_rows_and_threads, check_valid_frame,
    check_rgb_gray_inputs_and_hand_values, check_rgb_within_bt601, check_rgb_channel_steps,
]
