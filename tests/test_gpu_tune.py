"""The autotuner: tuned configurations keep the output bit-exact, and the
tuned table survives a save / load round trip, the SOBEL4_TUNE_CACHE
variable and the creation options' cache path; the autotune option tunes
each new shape bucket on its first run."""
import numpy as np
import pytest

import oracle
import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import Output, Placed, run_placed, same_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture
def handle():
    from paper_2305_00515_gb300 import build
    build.build()
    st, h = pkg.sobel4_create(0)
    assert st == 0
    yield h
    pkg.sobel4_destroy(h)


def test_tune_single_then_run(handle, tmp_path):
    st, us = pkg.sobel4_tune(handle, 1000, 1500, 0, 0)
    assert st == 0 and us > 0
    assert pkg.sobel4_tune_entries(handle) == 1
    img = synth.rects_noise(1000, 1500, 4)
    got, guards = run_placed(torch, handle, img, "valid", "f32")
    assert guards and same_bits(got, oracle.sobel4(img, "valid", "f32", threads=8))
    path = str(tmp_path / "tune.json")
    assert pkg.sobel4_tune_save(handle, path) == 0
    st, h2 = pkg.sobel4_create(0)
    try:
        assert pkg.sobel4_tune_load(h2, path) == 0
        assert pkg.sobel4_tune_entries(h2) == 1
        got2, _ = run_placed(torch, h2, img, "valid", "f32")
        assert same_bits(got2, got)
    finally:
        pkg.sobel4_destroy(h2)


def test_autotune_option_and_cache_path(tmp_path):
    """sobel4_options.autotune: the first sobel4_run of a shape bucket tunes
    it (one entry per bucket, results exact); cache_path is rewritten after
    each automatic tune and loaded by the next handle that names it."""
    from paper_2305_00515_gb300 import build
    build.build()
    path = str(tmp_path / "auto.json")
    st, h = pkg.sobel4_create(0, autotune=1, cache_path=path)
    assert st == 0
    try:
        assert pkg.sobel4_tune_entries(h) == 0
        for (H, W, n_after) in ((1000, 1500, 1), (900, 1100, 1), (300, 200, 2)):
            img = synth.rects_noise(H, W, H + W)
            got, guards = run_placed(torch, h, img, "replicate", "f32")
            assert guards and same_bits(got, oracle.sobel4(img, "replicate", "f32", threads=8))
            assert pkg.sobel4_tune_entries(h) == n_after, (H, W)
    finally:
        pkg.sobel4_destroy(h)
    st, h2 = pkg.sobel4_create(0, cache_path=path)  # no autotune: the cache alone
    try:
        assert st == 0 and pkg.sobel4_tune_entries(h2) == 2
    finally:
        pkg.sobel4_destroy(h2)
    assert pkg.sobel4_create(0, autotune=2)[0] == 1


def test_tune_cache_rejections(handle, tmp_path, monkeypatch):
    bad = tmp_path / "bad.json"
    bad.write_text("not a tuning file\n")
    assert pkg.sobel4_tune_load(handle, str(bad)) == 1
    assert pkg.sobel4_tune_load(handle, str(tmp_path / "missing.json")) == 1
    other = tmp_path / "other.json"
    other.write_text('{"sobel4_tune": 1, "version": "0.1.0", "device": "Some Other GPU", '
                     '"sm_count": 3,\n "entries": [\n  {"kind": 0, "hb": 5, "wb": 5, "fmt": 0, '
                     '"nc": 4, "R": 8, "ctas": 4, "us": 1.000}\n ]}\n')
    assert pkg.sobel4_tune_load(handle, str(other)) == 2
    assert pkg.sobel4_tune_entries(handle) == 0
    # a table saved here loads automatically through SOBEL4_TUNE_CACHE
    assert pkg.sobel4_tune(handle, 300, 300, 1, 1)[0] == 0
    path = str(tmp_path / "cache.json")
    assert pkg.sobel4_tune_save(handle, path) == 0
    monkeypatch.setenv("SOBEL4_TUNE_CACHE", path)
    st, h2 = pkg.sobel4_create(0)
    assert st == 0
    assert pkg.sobel4_tune_entries(h2) == 1
    pkg.sobel4_destroy(h2)


def test_tune_batched_keeps_results_exact(handle):
    imgs = [synth.rects_noise(h, w, 50 + i) for i, (h, w) in
            enumerate(((37, 41), (300, 129), (131, 600), (64, 64), (500, 257)))]
    srcs = [Placed(torch, im, im.shape[1], 0) for im in imgs]
    outs = [Output(torch, im.shape[0], im.shape[1], "u8", im.shape[1], 0) for im in imgs]
    descs = [pkg.Image(s.ptr, s.pitch, o.ptr, o.pitch, *im.shape)
             for s, o, im in zip(srcs, outs, imgs)]
    torch.cuda.synchronize()
    st, us = pkg.sobel4_tune_batched(handle, descs, 2, 1)
    assert st == 0 and us > 0
    assert pkg.sobel4_tune_entries(handle) == 1
    assert pkg.sobel4_run_batched(handle, descs, 2, 1, torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    for im, o in zip(imgs, outs):
        got, guards = o.read()
        assert guards and same_bits(got, oracle.sobel4(im, "reflect101", "u8"))


def test_tune_config_reports_the_chosen_kernel(handle):
    """The configuration query follows the tuned table; every tuned strip height
    keeps the TMA-staged output exact."""
    st, kind, nc, R = pkg.sobel4_tune_config(handle, 2048, 2048, 0)
    assert st == 0 and kind == 1 and nc == 4 and R % 4 == 0 and R >= 8   # built-in rule
    assert pkg.sobel4_tune(handle, 2048, 2048, 0, 0)[0] == 0
    st, kind2, nc2, R2 = pkg.sobel4_tune_config(handle, 2048, 2048, 0)
    assert st == 0 and kind2 in (0, 1) and nc2 in (2, 4) and R2 >= 4
    img = synth.uniform(2048, 2048, 6)
    got, guards = run_placed(torch, handle, img, "valid", "f32")
    assert guards and same_bits(got, oracle.sobel4(img, "valid", "f32", threads=8))
    for R in (8, 12, 20, 44, 128):
        st, h = pkg.sobel4_create(0, pkg.VARIANTS["rg"], rows_per_strip=R)
        assert st == 0
        try:
            assert pkg.sobel4_tune_config(h, 300, 700, 0)[3] == R
            small = synth.rects_noise(300, 700, R)
            out, g = run_placed(torch, h, small, "reflect101", "u8", src_pitch=704)
            assert g and same_bits(out, oracle.sobel4(small, "reflect101", "u8")), R
        finally:
            pkg.sobel4_destroy(h)
    assert pkg.sobel4_tune_config(handle, 0, 10, 0)[0] == 1
