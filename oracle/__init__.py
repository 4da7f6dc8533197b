"""Plain CPU oracle for the four-directional 5x5 Sobel operator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2305_00515_gb300``) never imports it, and it
imports nothing from there: the two share no code, tables or helpers.

The arithmetic lives in ``sobel4_oracle.c`` (a direct 25-tap correlation per
mask, Eq. (3) and Eq. (4) of Section 3.1, written out with no factoring; the
generalised masks of Eq. (5) written out entry by entry); this
module only compiles it with gcc and marshals numpy arrays through ctypes.
Every function here is pinned by ``tests/test_oracle_pins.py`` against the
paper's other statements of the operator (Eq. (5), (10), (18)), closed forms,
invariants, and an independent library correlation (scipy.ndimage).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sobel4_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libsobel4_oracle.so")

BORDERS = {"valid": 0, "replicate": 1, "reflect101": 2, "constant0": 3}
FORMATS = {"f32": 0, "u8": 1, "s16x4": 2, "u16": 3, "edge8": 4}
_OUT_DTYPE = {"f32": np.float32, "u8": np.uint8, "s16x4": np.int16, "u16": np.uint16,
              "edge8": np.uint8}
DEFAULT_THRESHOLD = 128

_lock = threading.Lock()
_default = None


def build(src: str = _SRC, out: str = _LIB_PATH, force: bool = False) -> str:
    """Compile the oracle C source into a shared library (gcc, no fast-math)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-pthread",
           "-fno-fast-math", "-ffp-contract=off", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class Oracle:
    """ctypes view of one compiled oracle library."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.sobel4_oracle_run.argtypes = [u8p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.c_size_t, ctypes.c_int32]
        lib.sobel4_oracle_run.restype = ctypes.c_int
        lib.sobel4_oracle_responses.argtypes = [u8p, ctypes.c_size_t, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_int32)]
        lib.sobel4_oracle_responses.restype = ctypes.c_int
        lib.sobel4_oracle_masks.argtypes = [ctypes.POINTER(ctypes.c_int32)]
        lib.sobel4_oracle_masks.restype = ctypes.c_int
        lib.sobel4_oracle_eq5_masks.argtypes = [ctypes.c_double] * 4 + [
            ctypes.POINTER(ctypes.c_int32)]
        lib.sobel4_oracle_eq5_masks.restype = ctypes.c_int
        lib.sobel4_oracle_run_masks.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                                ctypes.c_int64, u8p, ctypes.c_size_t,
                                                ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32]
        lib.sobel4_oracle_operator_masks.argtypes = [ctypes.c_int32,
                                                     ctypes.POINTER(ctypes.c_int32),
                                                     ctypes.POINTER(ctypes.c_int32)]
        lib.sobel4_oracle_operator_masks.restype = ctypes.c_int
        lib.sobel4_oracle_run_masks.restype = ctypes.c_int
        lib.sobel4_oracle_rgb_to_gray.argtypes = [u8p, ctypes.c_size_t, ctypes.c_int32,
                                                  ctypes.c_int32, u8p, ctypes.c_size_t]
        lib.sobel4_oracle_rgb_to_gray.restype = ctypes.c_int
        lib.sobel4_oracle_magnitude_f32.argtypes = [ctypes.c_int32]
        lib.sobel4_oracle_magnitude_f32.restype = ctypes.c_float
        lib.sobel4_oracle_magnitude_u8.argtypes = [ctypes.c_int32]
        lib.sobel4_oracle_magnitude_u8.restype = ctypes.c_int32
        lib.sobel4_oracle_magnitude_u16.argtypes = [ctypes.c_int32]
        lib.sobel4_oracle_magnitude_u16.restype = ctypes.c_int32
        self.lib = lib
        self.path = lib_path

    # -- Eq. (3) tables -------------------------------------------------------
    def masks(self) -> np.ndarray:
        """The four 5x5 masks G_x, G_y, G_d, G_dt of Eq. (3), shape (4, 5, 5)."""
        out = np.zeros((4, 5, 5), dtype=np.int32)
        rc = self.lib.sobel4_oracle_masks(out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        assert rc == 0
        return out

    # -- Eq. (3)/(4) per pixel ----------------------------------------------------
    @staticmethod
    def _src(img: np.ndarray):
        if img.dtype != np.uint8 or img.ndim != 2:
            raise ValueError("image must be a 2-D uint8 array")
        if img.strides[1] != 1:
            img = np.ascontiguousarray(img)
        return img, img.strides[0]

    def responses(self, img: np.ndarray, border: str = "valid") -> np.ndarray:
        """R_x, R_y, R_d, R_dt of Eq. (3) as int32 planes, shape (4, H, W)."""
        img, sp = self._src(img)
        H, W = img.shape
        out = np.zeros((4, H, W), dtype=np.int32)
        rc = self.lib.sobel4_oracle_responses(
            img.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), sp, H, W, BORDERS[border],
            out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if rc != 0:
            raise ValueError(f"oracle rejected arguments (H={H}, W={W}, border={border})")
        return out

    def run_into(self, img: np.ndarray, out: np.ndarray, border: str = "valid",
                 fmt: str = "f32", threads: int = 1, masks=None, radius: int = 2,
                 threshold=None) -> None:
        """Gradient output of Eq. (4) written into a caller array (rows may be padded);
        `masks` (4, 5, 5) integers replace the Eq. (3) masks when given."""
        img, sp = self._src(img)
        H, W = img.shape
        u8 = img.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        if masks is None and fmt == "edge8":
            masks = self.masks()
        if masks is None:
            rc = self.lib.sobel4_oracle_run(u8, sp, H, W, BORDERS[border], FORMATS[fmt],
                                            out.ctypes.data, out.strides[-2], int(threads))
        else:
            m = np.ascontiguousarray(masks, dtype=np.int32).reshape(100)
            rc = self.lib.sobel4_oracle_run_masks(
                m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(radius),
                edge_threshold(DEFAULT_THRESHOLD if threshold is None else threshold), u8, sp,
                H, W, BORDERS[border], FORMATS[fmt], out.ctypes.data, out.strides[-2],
                int(threads))
        if rc != 0:
            raise ValueError(f"oracle rejected arguments (H={H}, W={W}, border={border})")

    def sobel4(self, img: np.ndarray, border: str = "valid", fmt: str = "f32",
               threads: int = 1, masks=None, radius: int = 2, threshold=None) -> np.ndarray:
        """Gradient output of Eq. (4): (H, W) f32/u8/u16, or (4, H, W) int16 for s16x4."""
        H, W = img.shape
        shape = (4, H, W) if fmt == "s16x4" else (H, W)
        out = np.zeros(shape, dtype=_OUT_DTYPE[fmt])
        self.run_into(img, out, border, fmt, threads, masks, radius, threshold)
        return out

    def operator_masks(self, op: str):
        """(masks (4, 5, 5), radius) of the 2dir5x5 or 2dir3x3 operator."""
        out = np.zeros(100, dtype=np.int32)
        r = ctypes.c_int32(0)
        rc = self.lib.sobel4_oracle_operator_masks(
            {"2dir5x5": 1, "2dir3x3": 2}[op], out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            ctypes.byref(r))
        if rc != 0:
            raise ValueError(op)
        return out.reshape(4, 5, 5), r.value

    def eq5_masks(self, a: float, b: float, n: float, m: float) -> np.ndarray:
        """The generalised masks of Eq. (5) as (4, 5, 5) int32 (x, y, d, dt)."""
        out = np.zeros(100, dtype=np.int32)
        rc = self.lib.sobel4_oracle_eq5_masks(float(a), float(b), float(n), float(m),
                                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if rc != 0:
            raise ValueError(f"Eq. (5) weights are not integers for {(a, b, n, m)}")
        return out.reshape(4, 5, 5)

    # -- grayscale input (the host preparation of Section 4.3) ------------------
    def rgb_to_gray(self, rgb: np.ndarray) -> np.ndarray:
        """Y = (77 R + 150 G + 29 B + 128) >> 8 per pixel of an (H, W, 3) uint8 RGB
        image (rows may be padded: row stride >= 3 W), as an (H, W) uint8 image."""
        if rgb.dtype != np.uint8 or rgb.ndim != 3 or rgb.shape[2] != 3:
            raise ValueError("image must be an (H, W, 3) uint8 array")
        if rgb.strides[1:] != (3, 1):
            rgb = np.ascontiguousarray(rgb)
        H, W, _ = rgb.shape
        sp = rgb.strides[0] if H > 1 else 3 * W  # a single row may carry stride 0
        out = np.empty((H, W), dtype=np.uint8)
        u8 = ctypes.POINTER(ctypes.c_uint8)
        rc = self.lib.sobel4_oracle_rgb_to_gray(rgb.ctypes.data_as(u8), sp, H, W,
                                                out.ctypes.data_as(u8), W)
        if rc != 0:
            raise ValueError("oracle rejected arguments")
        return out

    def sobel4_rgb(self, rgb: np.ndarray, border: str = "valid", fmt: str = "f32",
                   threads: int = 1) -> np.ndarray:
        """The operator on the grayscale of an RGB image: convert, then Eq. (3)-(4)."""
        return self.sobel4(self.rgb_to_gray(rgb), border, fmt, threads)

    def magnitude_f32(self, s: int) -> np.float32:
        return np.float32(self.lib.sobel4_oracle_magnitude_f32(int(s)))

    def magnitude_u8(self, s: int) -> int:
        return int(self.lib.sobel4_oracle_magnitude_u8(int(s)))

    def magnitude_u16(self, s: int) -> int:
        return int(self.lib.sobel4_oracle_magnitude_u16(int(s)))


def default() -> Oracle:
    """The oracle built from the committed source (compiled on first use)."""
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
        return _default


def masks() -> np.ndarray:
    return default().masks()


def responses(img: np.ndarray, border: str = "valid") -> np.ndarray:
    return default().responses(img, border)


def sobel4(img: np.ndarray, border: str = "valid", fmt: str = "f32", threads: int = 1,
           masks=None, radius: int = 2, threshold=None):
    return default().sobel4(img, border, fmt, threads, masks, radius, threshold)


def edge_threshold(t) -> int:
    """ceil(t^2) for the EDGE8 rule sqrt(S) >= t, in exact rational arithmetic."""
    from fractions import Fraction
    import math
    q = Fraction(t) ** 2
    return math.ceil(q)


def rgb_to_gray(rgb: np.ndarray) -> np.ndarray:
    return default().rgb_to_gray(rgb)


def sobel4_rgb(rgb: np.ndarray, border: str = "valid", fmt: str = "f32", threads: int = 1):
    return default().sobel4_rgb(rgb, border, fmt, threads)


def operator_masks(op: str):
    return default().operator_masks(op)


def eq5_masks(a: float, b: float, n: float, m: float) -> np.ndarray:
    return default().eq5_masks(a, b, n, m)


def cpu_count() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
