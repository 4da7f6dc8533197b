"""The paper's kernel ladder (Section 5.2, Table 1) as library variants —
shared-memory tile (SM), SM with prefetching (SM-P), and the plain register
window with the diagonals direct (RG), through K_d+ (RG-v1) and fully
decomposed (RG-v2) — against the CPU oracle, bit for bit: ragged shapes
around the 32-column tile, the 28-column warp strip and the 8-row tile, every
border rule and format, odd pitches and byte offsets, short RG strips, images
taller than one grid of CTAs, a batch and the host-buffer path."""
import numpy as np
import pytest

import oracle
import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import ELEM, run_placed, same_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LADDER = ("ladder_sm", "ladder_sm_p", "ladder_rg", "ladder_rg_v1", "ladder_rg_v2")
BORDERS = ("valid", "replicate", "reflect101", "constant0")
FORMATS = ("f32", "u8", "s16x4", "u16", "edge8")
SHAPES = [(1, 1), (2, 3), (3, 3), (5, 5), (7, 27), (8, 28), (9, 29), (13, 32), (16, 33),
          (17, 56), (63, 57), (64, 112), (65, 113), (70, 225), (129, 131), (200, 261)]
NCPU = oracle.cpu_count()


@pytest.fixture(scope="module")
def handles():
    from paper_2305_00515_gb300 import build
    build.build()
    hs = {}
    for v in LADDER:
        st, h = pkg.sobel4_create(0, pkg.VARIANTS[v])
        assert st == 0, pkg.sobel4_status_string(st)
        hs[v] = h
    for R in (1, 3, 7):
        for v in ("ladder_rg", "ladder_rg_v1", "ladder_rg_v2"):
            st, h = pkg.sobel4_create(0, pkg.VARIANTS[v], rows_per_strip=R)
            assert st == 0
            hs[f"{v}_r{R}"] = h
    yield hs
    for h in hs.values():
        pkg.sobel4_destroy(h)


def assert_same(got, want, what):
    if not same_bits(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {bad[:4].tolist()}")


@pytest.mark.parametrize("HW", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_ladder_every_border_and_format(handles, HW):
    H, W = HW
    img = np.random.default_rng(11 * H + W).integers(0, 256, size=(H, W), dtype=np.uint8)
    for border in BORDERS:
        if border == "reflect101" and (H < 3 or W < 3):
            continue
        for fmt in FORMATS:
            want = oracle.sobel4(img, border, fmt)
            e = ELEM[fmt]
            for v in LADDER:
                for (sp, soff, dp, doff) in ((W, 0, W * e, 0), (W + 3, 5, (W + 2) * e, e)):
                    got, guards = run_placed(torch, handles[v], img, border, fmt, src_pitch=sp,
                                             src_offset=soff, dst_pitch=dp, dst_offset=doff)
                    what = f"{v} {H}x{W} {border} {fmt} sp {sp}"
                    assert guards, f"{what}: write outside the payload"
                    assert_same(got, want, what)


def test_ladder_rg_short_strips(handles):
    """RG strips of 1, 3 and 7 rows: every strip starts and ends inside the
    image, so the 5-row window refills at each strip edge."""
    for (H, W) in ((1, 30), (4, 57), (11, 100), (50, 29), (97, 140)):
        img = synth.rects_noise(H, W, H + 7 * W)
        for border in BORDERS:
            if border == "reflect101" and (H < 3 or W < 3):
                continue
            want = oracle.sobel4(img, border, "f32")
            for R in (1, 3, 7):
                for v in ("ladder_rg", "ladder_rg_v1", "ladder_rg_v2"):
                    got, guards = run_placed(torch, handles[f"{v}_r{R}"], img, border, "f32")
                    assert guards
                    assert_same(got, want, f"{v} R={R} {H}x{W} {border}")


def test_ladder_512_rects_and_2k(handles):
    for (H, W) in ((512, 512), (1080, 1920)):
        img = synth.rects_noise(H, W, 0)
        for border in ("valid", "replicate"):
            want = oracle.sobel4(img, border, "f32", threads=NCPU)
            for v in LADDER:
                got, guards = run_placed(torch, handles[v], img, border, "f32")
                assert guards
                assert_same(got, want, f"{v} {H}x{W} {border}")


def test_taller_than_one_grid(handles):
    """More tile rows than a grid's y extent (65,535): the SM kernel walks
    8-row tiles in a loop and DIRECT takes two launches (600,000 rows), the RG
    kernels loop over 1-row strips, SM-P over 64-row strips (4.3 M rows)."""
    st, hd = pkg.sobel4_create(0, pkg.VARIANTS["direct"])
    assert st == 0
    try:
        tall = ("ladder_sm", "ladder_rg_r1", "ladder_rg_v2_r1", "direct")
        for (H, W, names) in ((600_000, 9, tall), (4_300_000, 3, ("ladder_sm_p",))):
            img = synth.uniform(H, W, 5)
            want = oracle.sobel4(img, "replicate", "u8", threads=NCPU)
            for name in names:
                h = hd if name == "direct" else handles[name]
                got, guards = run_placed(torch, h, img, "replicate", "u8")
                assert guards
                assert_same(got, want, f"{name} {H}x{W}")
    finally:
        pkg.sobel4_destroy(hd)


def test_ladder_batch_and_host_buffers():
    imgs = [synth.rects_noise(h, w, i) for i, (h, w) in enumerate(((37, 61), (130, 257), (64, 112),
                                                                   (5, 300)))]
    for v in LADDER:
        with pkg.Sobel4(0, variant=v) as s:
            outs = s.run_batched([torch.from_numpy(m).cuda() for m in imgs], border="reflect101",
                                 fmt="u16")
            torch.cuda.synchronize()
            for m, o in zip(imgs, outs):
                assert_same(o.cpu().numpy(), oracle.sobel4(m, "reflect101", "u16"), f"{v} batch")
            big = synth.rects_noise(1300, 2100, 9)
            got = s.run_host(big, border="constant0", fmt="s16x4")
            assert_same(got, oracle.sobel4(big, "constant0", "s16x4", threads=NCPU), f"{v} host")


def test_tune_config_names_the_ladder_kernels(handles):
    for k, v in enumerate(LADDER):
        st, kind, nc, R = pkg.sobel4_tune_config(handles[v], 2048, 2048, pkg.FORMATS["f32"])
        assert st == 0 and kind == 4 + k and nc == 1
        assert (R > 0) == v.startswith("ladder_rg")
    st, kind, _, R = pkg.sobel4_tune_config(handles["ladder_rg_v1_r3"], 100, 100, 0)
    assert st == 0 and kind == 7 and R == 3
    st, hd = pkg.sobel4_create(0, pkg.VARIANTS["direct"])
    assert st == 0
    try:
        assert pkg.sobel4_tune_config(hd, 512, 512, 0)[:2] == (0, 3)
    finally:
        pkg.sobel4_destroy(hd)
