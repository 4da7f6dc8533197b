"""Runtime weights (the generalised operator of Eq. 5) through the C ABI,
against the oracle's Eq. (5) masks, bit for bit.

Weights whose packed-pass coefficients sobel4_set_weights proves exact run on
the register-window kernel (every format but S16X4; all four weight sets here
do); S16X4 and DIRECT handles run the DIRECT kernel.  Batches run image by
image.  Every border, format and a batch are covered for four weight sets,
and (1, 2, 4, 6) must restore the Eq. (3) passes and results.  Tolerance:
zero mismatched elements, no write outside the payload.
"""
import numpy as np
import pytest

import oracle
import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import run_placed, same_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BORDERS = ("valid", "replicate", "reflect101", "constant0")
FORMATS = ("f32", "u8", "s16x4", "u16", "edge8")
PARAMS = [(2, 0.5, 3, 4), (3, 1, 2, 5), (1, 3, 1, 1), (2, 1.5, 2, 2)]
SHAPES = [(37, 61), (130, 256), (257, 300)]


def ceil16(v):
    return (v + 15) // 16 * 16


def assert_same(got, want, what):
    if not same_bits(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {bad[:4].tolist()}")


@pytest.fixture(scope="module")
def built():
    from paper_2305_00515_gb300 import build
    build.build()


@pytest.mark.parametrize("abnm", PARAMS, ids=lambda p: "a{}b{}n{}m{}".format(*p))
@pytest.mark.parametrize("variant", ("auto", "direct"))
def test_runtime_weights_match_oracle(built, abnm, variant):
    K = oracle.eq5_masks(*abnm)
    st, h = pkg.sobel4_create(0, pkg.VARIANTS[variant])
    assert st == 0
    try:
        assert pkg.sobel4_set_weights(h, *abnm) == 0
        # the kernel these weights run on: the register window (1) or DIRECT (3)
        kind = pkg.sobel4_tune_config(h, 512, 512, 0)[1]
        assert kind == (1 if variant == "auto" else 3), kind
        for (H, W) in SHAPES:
            img = synth.rects_noise(H, W, H * W)
            for border in BORDERS:
                for fmt in FORMATS:
                    want = oracle.sobel4(img, border, fmt, masks=K)
                    e = {"f32": 4, "u8": 1, "s16x4": 2, "u16": 2, "edge8": 1}[fmt]
                    for sp, dp in ((W, W * e), (ceil16(W), ceil16(W * e))):
                        got, guards = run_placed(torch, h, img, border, fmt, src_pitch=sp,
                                                 dst_pitch=dp)
                        assert guards, f"{abnm} {H}x{W} {border} {fmt}: outside the payload"
                        assert_same(got, want, f"{abnm} {variant} {H}x{W} {border} {fmt} sp {sp}")
        assert pkg.sobel4_device_status(h) == 0
    finally:
        pkg.sobel4_destroy(h)


def test_runtime_weights_batched_and_restore(built):
    abnm = (2, 0.5, 3, 4)
    K = oracle.eq5_masks(*abnm)
    with pkg.Sobel4(0) as s:
        s.set_weights(*abnm)
        batch = [torch.from_numpy(synth.rects_noise(H, W, 3 + H)).cuda()
                 for (H, W) in ((40, 64), (129, 300), (300, 512))]
        outs = s.run_batched(batch, border="reflect101", fmt="f32")
        big = torch.from_numpy(synth.rects_noise(1024, 2048, 5)).cuda()
        out_big = s.run(big)  # VALID F32: the register-window kernel with these coefficients
        torch.cuda.synchronize()
        for b, o in zip(batch, outs):
            assert_same(o.cpu().numpy(), oracle.sobel4(b.cpu().numpy(), "reflect101", "f32",
                                                       masks=K), "batch")
        assert_same(out_big.cpu().numpy(),
                    oracle.sobel4(big.cpu().numpy(), "valid", "f32", masks=K,
                                  threads=oracle.cpu_count()), "1024x2048")
        s.set_weights()  # (1, 2, 4, 6): Eq. (3) again
        out = s.run(big)
        torch.cuda.synchronize()
        assert_same(out.cpu().numpy(), oracle.sobel4(big.cpu().numpy(), "valid", "f32",
                                                     threads=oracle.cpu_count()), "restored")


def test_tune_with_runtime_weights(built):
    """sobel4_tune on a runtime-weight handle times the register-window kernel
    with the weights' coefficients; the chosen strip height then serves runs
    in that shape bucket, still bit-equal to the oracle.  Weights that do not
    run on the packed passes have nothing to tune (UNSUPPORTED)."""
    abnm = (2, 1.5, 2, 2)
    K = oracle.eq5_masks(*abnm)
    st, h = pkg.sobel4_create(0)
    assert st == 0
    try:
        assert pkg.sobel4_set_weights(h, *abnm) == 0
        st, us = pkg.sobel4_tune(h, 1024, 2048, 0, 0)
        assert st == 0 and us > 0
        _, kind, _, R = pkg.sobel4_tune_config(h, 1024, 2048, 0)
        assert kind == 1 and R > 0
        for (H, W) in ((1024, 2048), (1000, 1999)):
            img = synth.rects_noise(H, W, H + W)
            got, guards = run_placed(torch, h, img, "valid", "f32")
            assert guards
            assert_same(got, oracle.sobel4(img, "valid", "f32", masks=K,
                                           threads=oracle.cpu_count()), f"tuned {H}x{W}")
        assert pkg.sobel4_tune(h, 256, 256, 0, pkg.FORMATS["s16x4"])[0] == 2
        assert pkg.sobel4_set_operator(h, pkg.OPERATORS["2dir5x5"]) == 0
        assert pkg.sobel4_tune(h, 256, 256, 0, 0)[0] == 2
    finally:
        pkg.sobel4_destroy(h)
    st, h = pkg.sobel4_create(0, pkg.VARIANTS["direct"])
    try:
        assert pkg.sobel4_set_weights(h, *abnm) == 0
        assert pkg.sobel4_tune(h, 256, 256, 0, 0)[0] == 2
    finally:
        pkg.sobel4_destroy(h)


def test_runtime_weights_rejected(built):
    st, h = pkg.sobel4_create(0)
    assert st == 0
    try:
        assert pkg.sobel4_set_weights(h, 1, 0.3, 4, 6) == 1      # k_ij not integers
        assert pkg.sobel4_set_weights(h, 1.5, 2, 4, 6) == 1      # a not an integer
        assert pkg.sobel4_set_weights(h, 1, 2, 0, 6) == 1        # n not positive
        assert pkg.sobel4_set_weights(h, 8, 2, 4, 6) == 2        # S would overflow int32
        # a rejected call leaves the weights as they were (Eq. 3)
        img = synth.rects_noise(64, 64, 1)
        got, _ = run_placed(torch, h, img, "valid", "f32")
        assert_same(got, oracle.sobel4(img, "valid", "f32"), "unchanged")
    finally:
        pkg.sobel4_destroy(h)


@pytest.mark.parametrize("op", ("2dir5x5", "2dir3x3"))
@pytest.mark.parametrize("variant", ("auto", "direct"))
def test_two_directional_operators(built, op, variant):
    """The two-directional 5x5 and the 3x3 of Eq. (1)-(2) (1-pixel VALID
    frame) through the tensor-core and DIRECT kernels, against the oracle."""
    K, radius = oracle.operator_masks(op)
    st, h = pkg.sobel4_create(0, pkg.VARIANTS[variant])
    assert st == 0
    try:
        assert pkg.sobel4_set_operator(h, pkg.OPERATORS[op]) == 0
        for (H, W) in SHAPES:
            img = synth.rects_noise(H, W, H + 3 * W)
            for border in BORDERS:
                for fmt in FORMATS:
                    want = oracle.sobel4(img, border, fmt, masks=K, radius=radius)
                    e = {"f32": 4, "u8": 1, "s16x4": 2, "u16": 2, "edge8": 1}[fmt]
                    for sp, dp in ((W, W * e), (ceil16(W), ceil16(W * e))):
                        got, guards = run_placed(torch, h, img, border, fmt, src_pitch=sp,
                                                 dst_pitch=dp)
                        assert guards
                        assert_same(got, want, f"{op} {variant} {H}x{W} {border} {fmt} sp {sp}")
        assert pkg.sobel4_set_operator(h, 7) == 1
        assert pkg.sobel4_set_operator(h, pkg.OPERATORS["4dir5x5"]) == 0
        img = synth.rects_noise(64, 128, 2)
        got, _ = run_placed(torch, h, img, "valid", "f32")
        assert_same(got, oracle.sobel4(img, "valid", "f32"), "restored")
    finally:
        pkg.sobel4_destroy(h)


def test_edge8_thresholds(built):
    """EDGE8 with thresholds other than the default (T = 128), through the
    TMA-family kernels (aligned and unaligned rows) and DIRECT."""
    for variant in ("auto", "direct"):
        st, h = pkg.sobel4_create(0, pkg.VARIANTS[variant])
        assert st == 0
        try:
            for T in (0, 100.5, 777.25):
                assert pkg.sobel4_set_threshold(h, T) == 0
                for (H, W) in SHAPES:
                    img = synth.rects_noise(H, W, 7 * H + W)
                    for border in BORDERS:
                        want = oracle.sobel4(img, border, "edge8", threshold=T)
                        for sp in (W, ceil16(W)):
                            got, guards = run_placed(torch, h, img, border, "edge8", src_pitch=sp)
                            assert guards
                            assert_same(got, want, f"{variant} T={T} {H}x{W} {border} sp {sp}")
            assert pkg.sobel4_set_threshold(h, -1.0) == 1
            assert pkg.sobel4_set_threshold(h, float("nan")) == 1
        finally:
            pkg.sobel4_destroy(h)
