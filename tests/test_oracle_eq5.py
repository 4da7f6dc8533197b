"""The oracle's generalised operator (Eq. 5, Section 3.2) against the paper's
other statements of it and against a library correlation.

Pins: (1, 2, 4, 6) gives the Eq. (3) tables; for general weights the sum and
difference of the diagonal masks equal the K_d+ and K_d- matrices printed in
Eq. (10), and K_d- equals the two outer products of Eq. (18) — different
printed matrices, so a wrong entry in the Eq. (5) transcription fails them;
K_y is the transpose of K_x and K_dt the left-right mirror of K_d; a linear
ramp gives the closed form a (2 + 2n + m)(4 + 2b); and runs with the
generated masks equal scipy.ndimage.correlate under every border rule.
"""
import numpy as np
import pytest

import oracle
import oracle_checks as oc

PARAMS = [(1, 2, 4, 6), (2, 0.5, 3, 4), (3, 1, 2, 5), (1, 3, 1, 1), (2, 1.5, 2, 2)]


@pytest.fixture(scope="module")
def o():
    return oracle.default()


def test_defaults_are_eq3(o):
    assert np.array_equal(o.eq5_masks(1, 2, 4, 6), o.masks())


@pytest.mark.parametrize("abnm", PARAMS)
def test_eq10_and_eq18_identities(o, abnm):
    a, b, n, m = abnm
    K = o.eq5_masks(a, b, n, m).astype(np.float64)
    kp, km = oc.eq10_kd_plus_minus(a, b, m, n)
    assert np.allclose(K[2] + K[3], kp), "K_d + K_dt must be the printed K_d+"
    assert np.allclose(K[2] - K[3], km), "K_d - K_dt must be the printed K_d-"
    assert np.allclose(K[2] - K[3], oc.eq18_kd_minus(a, b, m, n))
    assert np.array_equal(K[1], K[0].T)
    assert np.array_equal(K[3], K[2][:, ::-1])
    assert all(K[k].sum() == 0 for k in range(4))


@pytest.mark.parametrize("abnm", PARAMS)
def test_ramp_closed_form(o, abnm):
    a, b, n, m = abnm
    K = o.eq5_masks(a, b, n, m)
    H, W = 9, 12
    ramp = np.tile(np.arange(W, dtype=np.uint8) * 3, (H, 1))
    R = oc.scipy_responses(ramp, "valid", K)
    want = 3 * a * (2 + 2 * n + m) * (4 + 2 * b)
    assert (R[0][2:H - 2, 2:W - 2] == want).all()
    assert (R[1][2:H - 2, 2:W - 2] == 0).all()


@pytest.mark.parametrize("abnm", PARAMS[1:])
def test_run_with_masks_matches_scipy(o, abnm):
    K = o.eq5_masks(*abnm)
    img = oc.rng_image(7, 23, 31)
    for border in oc.BORDERS:
        R = oc.scipy_responses(img, border, K).astype(np.int64)
        S = (R ** 2).sum(axis=0)
        assert S.max() < 2 ** 31
        got = o.sobel4(img, border, "f32", masks=K)
        assert np.array_equal(got, np.sqrt(S.astype(np.float32)).astype(np.float32)), border
        s16 = o.sobel4(img, border, "s16x4", masks=K)
        if np.abs(R).max() <= 32767:
            assert np.array_equal(s16.astype(np.int64), R), border


def test_eq3_masks_through_both_entry_points(o):
    img = oc.rng_image(3, 17, 19)
    for border in oc.BORDERS:
        for fmt in ("f32", "u8", "s16x4"):
            assert np.array_equal(o.sobel4(img, border, fmt),
                                  o.sobel4(img, border, fmt, masks=o.masks()))


def test_rejects_non_integer_weights(o):
    for bad in ((1, 0.3, 4, 6), (1.5, 2, 4, 6), (0, 2, 4, 6), (1, -2, 4, 6), (1, 2, 4.5, 6)):
        with pytest.raises(ValueError):
            o.eq5_masks(*bad)


def test_u16_rule(o):
    """U16 = nearest integer to sqrt(S), unsaturated: (2r-1)^2 <= 4S < (2r+1)^2 (r > 0),
    checked on every S below 2^20, around every square and its midpoints up to
    the largest S of Eq. (3), and at the int32 end."""
    import itertools
    ss = itertools.chain(range(0, 1 << 20, 7), (k * k + d for k in range(0, 24500, 97)
                                               for d in (-k - 1, -k, -1, 0, k, k + 1) if k * k + d >= 0),
                         (599270400, (1 << 31) - 1))
    for s in ss:
        r = o.magnitude_u16(s)
        assert (r == 0 or (2 * r - 1) ** 2 <= 4 * s) and 4 * s < (2 * r + 1) ** 2, s
    img = oc.rng_image(5, 19, 23)
    R = oc.scipy_responses(img, "reflect101", o.masks()).astype(np.int64)
    S = (R ** 2).sum(axis=0)
    got = o.sobel4(img, "reflect101", "u16").astype(np.int64)
    assert (((2 * got - 1) ** 2 <= 4 * S) | (got == 0)).all() and (4 * S < (2 * got + 1) ** 2).all()


def test_two_directional_operators(o):
    """The two-directional 3x3 of Eq. (1) against scipy.ndimage.sobel (a
    library routine: [-1 0 1] along the axis, [1 2 1] across), with its
    1-pixel VALID frame; the two-directional 5x5 = the first two Eq. (3)
    masks, diagonals zero, S = R_x^2 + R_y^2 (Eq. 2)."""
    import scipy.ndimage as ndi
    m3, r3 = o.operator_masks("2dir3x3")
    m5, r5 = o.operator_masks("2dir5x5")
    assert (r3, r5) == (1, 2)
    assert np.array_equal(m5[:2], o.masks()[:2]) and not m5[2:].any() and not m3[2:].any()
    img = oc.rng_image(11, 21, 26)
    I = img.astype(np.int64)
    mode = {"replicate": "nearest", "reflect101": "mirror", "constant0": "constant"}
    for border in ("valid", "replicate", "reflect101", "constant0"):
        md = mode.get(border, "nearest")
        gx = ndi.sobel(I, axis=1, mode=md, cval=0)
        gy = ndi.sobel(I, axis=0, mode=md, cval=0)
        if border == "valid":
            keep = np.zeros(I.shape, bool)
            keep[1:-1, 1:-1] = True
            gx, gy = np.where(keep, gx, 0), np.where(keep, gy, 0)
        s16 = o.sobel4(img, border, "s16x4", masks=m3, radius=1).astype(np.int64)
        assert np.array_equal(s16[0], gx) and np.array_equal(s16[1], gy), border
        assert not s16[2:].any()
        f = o.sobel4(img, border, "f32", masks=m3, radius=1)
        assert np.array_equal(f, np.sqrt((gx * gx + gy * gy).astype(np.float32))), border
        R = oc.scipy_responses(img, border, o.masks()).astype(np.int64)
        f5 = o.sobel4(img, border, "f32", masks=m5)
        assert np.array_equal(f5, np.sqrt((R[0] ** 2 + R[1] ** 2).astype(np.float32))), border


def test_edge8_rule(o):
    """EDGE8 = 255 exactly where sqrt(S) >= T (S >= ceil(T^2)), frame 0."""
    from fractions import Fraction
    img = oc.rng_image(13, 25, 27)
    for border in oc.BORDERS:
        R = oc.scipy_responses(img, border, o.masks()).astype(np.int64)
        S = (R ** 2).sum(axis=0)
        for T in (0, 1, 100.5, 128, 1000.25, 5000):
            got = o.sobel4(img, border, "edge8", threshold=T)
            # sqrt(S) >= T  <=>  S >= T^2 (both sides non-negative), compared exactly
            want = np.array([[255 if Fraction(int(v)) >= Fraction(T) ** 2 else 0 for v in row]
                             for row in S], dtype=np.uint8)
            if border == "valid":
                frame = np.ones(S.shape, bool)
                frame[2:-2, 2:-2] = False
                want[frame] = 0
            assert np.array_equal(got, want), (border, T)
    assert oracle.edge_threshold(100.5) == 10101 and oracle.edge_threshold(128) == 16384
