"""GPU (sm_103a library through the C ABI) against the CPU oracle, bit for bit.

Tolerance: zero mismatched elements for every format.  The integer work is
exact, and the F32 output is sqrtf((float)S) on both sides (round-to-nearest
int->float conversion and the IEEE correctly rounded square root), so the
results are identical floats.
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
NCPU = oracle.cpu_count()


@pytest.fixture(scope="module")
def handles():
    from paper_2305_00515_gb300 import build
    build.build()
    hs = {}
    for v in ("rg", "direct"):
        st, h = pkg.sobel4_create(0, pkg.VARIANTS[v])
        assert st == 0, pkg.sobel4_status_string(st)
        hs[v] = h
    yield hs
    for h in hs.values():
        pkg.sobel4_destroy(h)


def assert_same(got, want, what):
    if not same_bits(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {bad[:4].tolist()}")


@pytest.mark.parametrize("variant", ["rg", "direct"])
@pytest.mark.parametrize("border", BORDERS)
@pytest.mark.parametrize("fmt", FORMATS)
def test_config0_512(handles, variant, border, fmt):
    """512x512 rects + noise (seed 0): every border rule and output format."""
    img = synth.rects_noise(512, 512, 0)
    got, guards = run_placed(torch, handles[variant], img, border, fmt)
    assert guards, "write outside the output payload"
    assert_same(got, oracle.sobel4(img, border, fmt, threads=NCPU), f"{variant} {border} {fmt}")


SMALL = [(1, 1), (1, 9), (9, 1), (2, 2), (3, 3), (4, 4), (4, 7), (5, 5), (6, 3), (7, 130),
         (5, 131), (8, 127), (9, 128), (10, 129), (11, 133), (12, 255), (13, 256), (17, 257),
         (33, 300), (64, 5), (100, 6), (70, 390), (129, 131), (3, 1000), (200, 261)]


@pytest.mark.parametrize("HW", SMALL, ids=lambda s: f"{s[0]}x{s[1]}")
def test_small_and_ragged_shapes(handles, HW):
    H, W = HW
    rng = np.random.default_rng(H * 1000 + W)
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    for border in BORDERS:
        if border == "reflect101" and (H < 3 or W < 3):
            continue
        for fmt in FORMATS:
            got, guards = run_placed(torch, handles["rg"], img, border, fmt)
            assert guards
            assert_same(got, oracle.sobel4(img, border, fmt), f"{H}x{W} {border} {fmt}")


PITCHES = [  # (src_pitch extra, src offset, dst pitch extra elements, dst offset bytes)
    (1, 1, 1, 4), (3, 2, 3, 8), (5, 3, 0, 12), (0, 1, 2, 0), (7, 0, 5, 4), (16, 3, 4, 16),
]


@pytest.mark.parametrize("case", PITCHES, ids=str)
@pytest.mark.parametrize("fmt", FORMATS)
def test_odd_pitches_and_offsets(handles, case, fmt):
    """Unaligned rows and unaligned/unpadded outputs take the general load/store paths."""
    spx, so, dpx, do = case
    elem = {"f32": 4, "u8": 1, "s16x4": 2, "u16": 2, "edge8": 1}[fmt]
    for (H, W) in ((37, 301), (64, 512), (9, 140)):
        img = synth.rects_noise(H, W, 3 + W)
        for border in BORDERS:
            got, guards = run_placed(torch, handles["rg"], img, border, fmt, src_pitch=W + spx,
                                     src_offset=so, dst_pitch=(W + dpx) * elem,
                                     dst_offset=do if fmt != "u8" else do + 1)
            assert guards
            assert_same(got, oracle.sobel4(img, border, fmt), f"{H}x{W} {case} {border} {fmt}")


@pytest.mark.parametrize("HW,kind", [((1024, 1024), "rects"), ((1024, 1024), "uniform"),
                                     ((1080, 1920), "rects"), ((1080, 1920), "uniform"),
                                     ((2160, 3840), "rects"), ((2160, 3840), "uniform"),
                                     ((4096, 4096), "rects"), ((4096, 4096), "uniform"),
                                     ((8192, 8192), "rects"), ((8192, 8192), "uniform")],
                         ids=lambda v: str(v))
def test_size_sweep_full_size(handles, HW, kind):
    """Every size of the sweep, full image, F32 with the paper's border rule (the bench launch)."""
    H, W = HW
    img = synth.rects_noise(H, W, 0) if kind == "rects" else synth.uniform(H, W, 0)
    got, guards = run_placed(torch, handles["rg"], img, "valid", "f32")
    assert guards
    assert_same(got, oracle.sobel4(img, "valid", "f32", threads=NCPU), f"{H}x{W} {kind}")


def test_pitch_variant_1080p(handles):
    """1920x1080 with src_pitch 1937 (odd) and dst_pitch 7748 (not 16-byte aligned)."""
    for seed, kind in ((0, "rects"), (1, "uniform")):
        img = synth.rects_noise(1080, 1920, seed) if kind == "rects" else synth.uniform(1080, 1920, seed)
        for border in BORDERS:
            got, guards = run_placed(torch, handles["rg"], img, border, "f32", src_pitch=1937,
                                     dst_pitch=7748)
            assert guards
            assert_same(got, oracle.sobel4(img, border, "f32", threads=NCPU), f"pitch {border}")


def test_direct_and_rg_agree_on_large(handles):
    img = synth.uniform(2048, 2100, 9)
    a, _ = run_placed(torch, handles["rg"], img, "reflect101", "s16x4")
    b, _ = run_placed(torch, handles["direct"], img, "reflect101", "s16x4")
    assert_same(a, b, "rg vs direct")
    assert_same(a, oracle.sobel4(img, "reflect101", "s16x4", threads=NCPU), "vs oracle")


def test_tensor_api_and_streams():
    with pkg.Sobel4(0) as s:
        img = synth.rects_noise(300, 500, 11)
        src = torch.from_numpy(img).cuda()
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            out = s.run(src, border="replicate", fmt="u8")
        stream.synchronize()
        assert_same(out.cpu().numpy(), oracle.sobel4(img, "replicate", "u8"), "stream u8")
        n0 = s.launches
        s.run(src)
        torch.cuda.synchronize()
        assert s.launches == n0 + 1
        # strided (column-sliced) source view
        big = torch.from_numpy(synth.rects_noise(300, 700, 12)).cuda()
        view = big[:, 100:600]
        out = s.run(view)
        torch.cuda.synchronize()
        assert_same(out.cpu().numpy(), oracle.sobel4(view.cpu().numpy(), "valid", "f32"), "view")


def test_run_host_end_to_end():
    with pkg.Sobel4(0) as s:
        for (H, W, fmt, border) in ((512, 512, "f32", "valid"), (333, 1001, "u8", "reflect101"),
                                    (100, 257, "s16x4", "constant0"), (2160, 3840, "f32", "valid")):
            img = synth.rects_noise(H, W, H + W)
            got = s.run_host(img, border=border, fmt=fmt)
            assert_same(got, oracle.sobel4(img, border, fmt, threads=NCPU), f"host {H}x{W}")
        # host source with padded rows
        padded = np.zeros((64, 100), np.uint8)
        padded[:, :77] = synth.uniform(64, 77, 2)
        got = s.run_host(padded[:, :77])
        assert_same(got, oracle.sobel4(padded[:, :77]), "host padded")


@pytest.mark.parametrize("border", ("valid", "replicate", "reflect101", "constant0"))
def test_run_host_banded(border):
    """Host-buffer runs large enough to be split into row bands (upload, kernel
    and download of neighbouring bands overlapped): every border rule, each
    format, a padded host source, and band seams at every row."""
    with pkg.Sobel4(0) as s:
        for (H, W, fmt) in ((1300, 3300, "f32"), (1100, 2000, "s16x4"), (4100, 4100, "u8")):
            img = synth.rects_noise(H, W, H ^ W)
            got = s.run_host(img, border=border, fmt=fmt)
            assert_same(got, oracle.sobel4(img, border, fmt, threads=NCPU), f"{H}x{W} {fmt}")
        padded = np.zeros((1301, 3320), np.uint8)
        padded[:, :3303] = synth.uniform(1301, 3303, 4)
        view = padded[:, :3303]
        got = s.run_host(view, border=border)
        assert_same(got, oracle.sobel4(np.ascontiguousarray(view), border, "f32", threads=NCPU),
                    "padded host source")
