"""Every plausible mistake planted in a copy of the oracle must fail some pin.

Each mutant is the committed oracle source with one textual change (a wrong
sign, a transposed index, convolution instead of correlation, a dropped term,
a wrong border rule, ...), compiled into a temporary library.  The pins of
``oracle_checks.py`` are then run on it; at least one must fail.  This shows
the pins are strong enough to catch the mistakes they are meant to catch.
"""
import os
import subprocess
import sys

import pytest

import oracle

TESTS = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(TESTS)

# Runs every pin on one mutant library and reports each failed pin on its own
# line.  A mutant may read or write outside its buffers (a wrong plane stride,
# an index past the last row), so it runs in a child process: its damage
# cannot reach the test process.
CHILD = """
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle, oracle_checks as oc
o = oracle.Oracle(sys.argv[1])
for check in oc.ALL_CHECKS:
    try:
        check(o)
    except (AssertionError, ValueError):
        print("FAILED", check.__name__, flush=True)
print("DONE", flush=True)
"""

SRC = os.path.join(os.path.dirname(oracle.__file__), "sobel4_oracle.c")

MUTANTS = {
    "gd_sign_flip": ("{-2, 0, 8, 12, 4},", "{-2, 0, 8, 12, -4},"),
    "gx_swapped_taps": ("{-4, -8, 0, 8, 4},\n     {-6", "{-8, -4, 0, 8, 4},\n     {-6"),
    "gdt_row_swap": ("{2, 0, -8, -12, -4},", "{0, 2, -8, -12, -4},"),
    "transposed_mask": ("r[k] += masks[k][i][j] * v", "r[k] += masks[k][j][i] * v"),
    "convolution_order": ("read_pixel(src, sp, H, W, y + i - 2, x + j - 2, border)",
                          "read_pixel(src, sp, H, W, y - i + 2, x - j + 2, border)"),
    "row_offset": ("sp, H, W, y + i - 2, x + j - 2, border);", "sp, H, W, y + i - 1, x + j - 2, border);"),
    "dropped_dt_term": ("+ r[3] * r[3];", ";"),
    "reflect_not_101": ("if (i < 0) return -i;", "if (i < 0) return -i - 1;"),
    "replicate_edge": ("return i < 0 ? 0 : n - 1;", "return i < 0 ? 0 : n - 2;"),
    "constant_reads_edge": ("case OR_CONSTANT0:\n      return -1;", "case OR_CONSTANT0:\n      return i < 0 ? 0 : n - 1;"),
    "valid_frame_off_by_one": ("y <= H - 1 - radius && x >= radius", "y <= H - radius && x >= radius"),
    "sqrt_in_double": ("((float *)row)[x] = sqrtf((float)s);",
                       "((float *)row)[x] = (float)sqrt((double)s);"),
    "u8_truncates": ("if ((uint32_t)s > n * n + n) n += 1;", "if ((uint32_t)s > n * n) n += 0;"),
    "u8_no_saturation": ("return (uint8_t)(n > 255u ? 255u : n);", "return (uint8_t)n;"),
    "s16_plane_stride": ("(size_t)k * (size_t)jb->H * jb->dp", "(size_t)k * (size_t)jb->W * jb->dp"),
    "rgb_bgr_order": ("const uint32_t r = in[3 * x], g = in[3 * x + 1], b = in[3 * x + 2];",
                      "const uint32_t r = in[3 * x + 2], g = in[3 * x + 1], b = in[3 * x];"),
    "rgb_truncates": ("29u * b + 128u) >> 8", "29u * b) >> 8"),
    "rgb_weight_sum_255": ("(77u * r + 150u * g", "(76u * r + 150u * g"),
    "band_split_gap": ("(int)((int64_t)H * (t + 1) / nthreads)}", "(int)((int64_t)H * (t + 1) / nthreads) - (t + 1 < nthreads)}"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    before, after = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(before) == 1, f"mutation site for {name} not found exactly once"
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(before, after))
    lib = oracle.build(str(src), str(tmp_path / "libmutant.so"), force=True)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, tests=TESTS), lib],
                       capture_output=True, text=True, timeout=600)
    failed = [ln.split()[1] for ln in r.stdout.splitlines() if ln.startswith("FAILED ")]
    # A pin must fail by assertion; a mutant that only crashes is not caught.
    assert failed, (f"no pin caught mutant {name} (exit {r.returncode}):\n"
                    f"{r.stdout[-2000:]}{r.stderr[-2000:]}")
