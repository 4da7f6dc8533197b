"""The C-ABI library on the CPU: it builds, loads, exports every declared entry
point, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

import paper_2305_00515_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sobel4.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sobel4_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_00515_gb300 import build
    build.build()
    return pkg.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), f"{name} declared in sobel4.h but not exported"
    assert sorted(pkg.EXPORTED_SYMBOLS) == names


def test_status_strings_and_version(lib):
    assert pkg.sobel4_version().count(".") == 2
    for code in range(6):
        assert pkg.sobel4_status_string(code)
    assert pkg.sobel4_status_string(99) == "unknown status"


def test_null_handle_queries(lib):
    assert pkg.sobel4_launch_count(None) == 0
    assert pkg.sobel4_last_cuda_error(None) == 0
    assert pkg.sobel4_destroy(None) == 0
    assert pkg.sobel4_set_variant(None, 0) == 1
    assert pkg.sobel4_set_weights(None, 1, 2, 4, 6) == 1
    assert pkg.sobel4_set_operator(None, 0) == 1
    assert pkg.sobel4_set_threshold(None, 10.0) == 1


def test_create_rejects_bad_options(lib):
    h = ctypes.c_void_p()
    bad = pkg.Options(10, 0, 0, 0)  # one past the last variant
    assert lib.sobel4_create(ctypes.byref(h), 0, ctypes.byref(bad)) == 1
    assert not h.value
    assert lib.sobel4_create(None, 0, None) == 1
    bad = pkg.Options(0, -1, 0, 0)
    assert lib.sobel4_create(ctypes.byref(h), 0, ctypes.byref(bad)) == 1
    bad = pkg.Options(0, 0, 0, 3)
    assert lib.sobel4_create(ctypes.byref(h), 0, ctypes.byref(bad)) == 1


# A zero-filled buffer stands in for a handle: these calls must return
# INVALID_ARG from host-side validation before the handle is ever used.
_FAKE = ctypes.create_string_buffer(1 << 16)
FAKE = ctypes.cast(_FAKE, ctypes.c_void_p)
SRC = 0x10000000
DST = 0x20000000

BAD_RUNS = [
    dict(d_src=0),
    dict(d_dst=0),
    dict(height=0),
    dict(width=0),
    dict(height=-3),
    dict(src_pitch=99),
    dict(dst_pitch=399),
    dict(dst_pitch=402),                     # F32 pitch not a multiple of 4
    dict(d_dst=DST + 2),                     # F32 destination not 4-byte aligned
    dict(border=4),
    dict(border=-1),
    dict(fmt=5),
    dict(border=2, height=2),                # REFLECT101 needs >= 3
    dict(border=2, width=2, src_pitch=100, dst_pitch=400),
    dict(d_dst=SRC + 50),                    # output overlaps input
    dict(src_pitch=1 << 31),
    dict(fmt=2, dst_pitch=201),              # S16X4 pitch must be even
]


@pytest.mark.parametrize("bad", BAD_RUNS, ids=lambda d: ",".join(f"{k}={v}" for k, v in d.items()))
def test_run_validation(lib, bad):
    args = dict(h=FAKE, d_src=SRC, src_pitch=100, d_dst=DST, dst_pitch=400, height=50, width=100,
                border=0, fmt=0, stream=None)
    args.update(bad)
    assert pkg.sobel4_run(*args.values()) == 1


def test_run_null_handle(lib):
    assert pkg.sobel4_run(None, SRC, 100, DST, 400, 50, 100, 0, 0, None) == 1


def test_batched_validation(lib):
    ok = pkg.Image(SRC, 100, DST, 400, 50, 100)
    assert pkg.sobel4_run_batched(FAKE, [], 0, 0, None) == 1
    assert lib.sobel4_run_batched(FAKE, None, 1, 0, 0, None) == 1
    assert pkg.sobel4_run_batched(FAKE, [ok], 9, 0, None) == 1
    # two outputs overlapping each other
    twin = pkg.Image(SRC + 10000, 100, DST + 400, 400, 50, 100)
    assert pkg.sobel4_run_batched(FAKE, [ok, twin], 0, 0, None) == 1
    # an output overlapping another image's input
    cross = pkg.Image(SRC + 20000, 100, SRC + 60, 400, 50, 100)
    assert pkg.sobel4_run_batched(FAKE, [ok, cross], 0, 0, None) == 1
    # one bad descriptor anywhere rejects the batch
    bad = pkg.Image(SRC + 30000, 10, DST + 40000, 400, 50, 100)
    assert pkg.sobel4_run_batched(FAKE, [ok, bad], 0, 0, None) == 1


def test_run_host_validation(lib):
    buf = ctypes.create_string_buffer(100)
    assert pkg.sobel4_run_host(FAKE, 0, 10, ctypes.addressof(buf), 40, 2, 10, 0, 0) == 1
    assert pkg.sobel4_run_host(FAKE, ctypes.addressof(buf), 9, ctypes.addressof(buf), 40, 2, 10,
                               0, 0) == 1


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "library_path", lambda: "/nonexistent/libsobel4.so")
    with pytest.raises(ImportError):
        pkg.load()


def header_enum(prefix):
    """{name: value} of the `prefix`* enumerators declared in sobel4.h."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1).lower(): int(m.group(2))
            for m in re.finditer(rf"\b{prefix}([A-Z0-9_]+)\s*=\s*(\d+)", text)}


def test_binding_enums_match_the_header():
    assert header_enum("SOBEL4_VARIANT_") == pkg.VARIANTS
    assert header_enum("SOBEL4_BORDER_") == pkg.BORDERS
    assert header_enum("SOBEL4_OUT_") == pkg.FORMATS
    assert {k.replace("_", ""): v for k, v in header_enum("SOBEL4_OP_").items()} == pkg.OPERATORS
