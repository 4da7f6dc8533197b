"""Python binding of the GB300 four-directional 5x5 Sobel library (``include/sobel4.h``).

Argument marshalling only: every step of the operator runs in the sm_103a
kernels of ``_build/libsobel4.so``.  The functions named ``sobel4_*`` mirror
the C ABI one to one and take raw pointers; :class:`Sobel4` wraps them for
PyTorch CUDA tensors (PyTorch provides device memory and streams, nothing
else) and numpy host arrays.

The library must have been built (``python -m paper_2305_00515_gb300.build``
or ``__graft_entry__.build()``); loading fails loudly otherwise.  There is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "BORDERS", "FORMATS", "VARIANTS", "Sobel4", "Sobel4Error", "Image", "Options",
    "library_path", "load", "sobel4_create", "sobel4_destroy", "sobel4_run", "sobel4_run_rgb",
    "sobel4_run_batched", "sobel4_run_host", "sobel4_status_string", "sobel4_last_cuda_error",
    "sobel4_device_status", "sobel4_inject_stage_loss", "sobel4_set_weights", "sobel4_set_operator", "sobel4_set_threshold", "OPERATORS", "sobel4_launch_count", "sobel4_set_variant", "sobel4_version", "sobel4_check_magnitude",
    "sobel4_run_batched_static", "sobel4_tune", "sobel4_tune_batched", "sobel4_tune_entries",
    "sobel4_tune_config", "sobel4_tune_save", "sobel4_tune_load", "sobel4_pipeline_create",
    "sobel4_pipeline_buffers", "sobel4_pipeline_submit", "sobel4_pipeline_submit_from",
    "sobel4_pipeline_wait", "sobel4_pipeline_destroy", "Pipeline", "sobel4_host_alloc",
    "sobel4_host_free", "HostBuffer",
    "sobel4_server_create", "sobel4_server_submit", "sobel4_server_wait", "sobel4_server_stats",
    "sobel4_server_destroy", "ServerOptions", "ServerStats", "EXPORTED_SYMBOLS",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
BORDERS = {"valid": 0, "replicate": 1, "reflect101": 2, "constant0": 3}
FORMATS = {"f32": 0, "u8": 1, "s16x4": 2, "u16": 3, "edge8": 4}
VARIANTS = {"auto": 0, "direct": 1, "rg": 2, "rg_lanecopy": 3, "tc": 4, "ladder_sm": 5,
            "ladder_sm_p": 6, "ladder_rg": 7, "ladder_rg_v1": 8, "ladder_rg_v2": 9}
OPERATORS = {"4dir5x5": 0, "2dir5x5": 1, "2dir3x3": 2}
ELEM_SIZE = {"f32": 4, "u8": 1, "s16x4": 2, "u16": 2, "edge8": 1}
STATUS = {0: "SOBEL4_OK", 1: "SOBEL4_ERR_INVALID_ARG", 2: "SOBEL4_ERR_UNSUPPORTED",
          3: "SOBEL4_ERR_OOM", 4: "SOBEL4_ERR_CUDA", 5: "SOBEL4_ERR_TIMEOUT"}

EXPORTED_SYMBOLS = (
    "sobel4_create", "sobel4_destroy", "sobel4_run", "sobel4_run_rgb", "sobel4_run_batched",
    "sobel4_run_host",
    "sobel4_status_string", "sobel4_last_cuda_error", "sobel4_device_status",
    "sobel4_inject_stage_loss", "sobel4_set_weights", "sobel4_set_operator",
    "sobel4_set_threshold", "sobel4_launch_count", "sobel4_set_variant", "sobel4_version", "sobel4_check_magnitude",
    "sobel4_run_batched_static", "sobel4_tune", "sobel4_tune_batched", "sobel4_tune_entries",
    "sobel4_tune_config", "sobel4_tune_save", "sobel4_tune_load", "sobel4_pipeline_create",
    "sobel4_pipeline_buffers", "sobel4_pipeline_submit", "sobel4_pipeline_submit_from",
    "sobel4_pipeline_wait", "sobel4_pipeline_destroy", "sobel4_host_alloc", "sobel4_host_free",
    "sobel4_server_create", "sobel4_server_submit", "sobel4_server_wait", "sobel4_server_stats",
    "sobel4_server_destroy",
)


class Sobel4Error(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class Image(ctypes.Structure):
    """``sobel4_image``: one image of a batch (device pointers)."""
    _fields_ = [("src", ctypes.c_void_p), ("src_pitch", ctypes.c_size_t),
                ("dst", ctypes.c_void_p), ("dst_pitch", ctypes.c_size_t),
                ("height", ctypes.c_int32), ("width", ctypes.c_int32)]


class ServerOptions(ctypes.Structure):
    """``sobel4_server_options``."""
    _fields_ = [("memory_budget", ctypes.c_int64), ("max_batch", ctypes.c_int32),
                ("border", ctypes.c_int32), ("format", ctypes.c_int32), ("plain", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    """``sobel4_server_counters``."""
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("max_batch_seen", ctypes.c_uint64),
                ("device_bytes_in_use", ctypes.c_int64), ("device_bytes_peak", ctypes.c_int64)]


class Options(ctypes.Structure):
    """``sobel4_options``."""
    _fields_ = [("variant", ctypes.c_int32), ("rows_per_strip", ctypes.c_int32),
                ("persistent_ctas_per_sm", ctypes.c_int32), ("columns_per_lane", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("cache_path", ctypes.c_char_p)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return os.path.join(_PKG, "_build", "libsobel4.so")


def load() -> ctypes.CDLL:
    """Load the built library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "`python -m paper_2305_00515_gb300.build`")
        lib = ctypes.CDLL(path)
        vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32
        lib.sobel4_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(Options)]
        lib.sobel4_destroy.argtypes = [vp]
        lib.sobel4_run.argtypes = [vp, vp, sz, vp, sz, i32, i32, i32, i32, vp]
        lib.sobel4_run_rgb.argtypes = [vp, vp, sz, vp, sz, i32, i32, i32, i32, vp]
        lib.sobel4_run_batched.argtypes = [vp, ctypes.POINTER(Image), i32, i32, i32, vp]
        lib.sobel4_run_host.argtypes = [vp, vp, sz, vp, sz, i32, i32, i32, i32]
        lib.sobel4_status_string.argtypes = [ctypes.c_int]
        lib.sobel4_status_string.restype = ctypes.c_char_p
        lib.sobel4_last_cuda_error.argtypes = [vp]
        lib.sobel4_last_cuda_error.restype = i32
        lib.sobel4_device_status.argtypes = [vp]
        lib.sobel4_inject_stage_loss.argtypes = [vp, i32]
        lib.sobel4_set_weights.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double]
        lib.sobel4_set_operator.argtypes = [vp, i32]
        lib.sobel4_set_threshold.argtypes = [vp, ctypes.c_double]
        lib.sobel4_launch_count.argtypes = [vp]
        lib.sobel4_launch_count.restype = ctypes.c_uint64
        lib.sobel4_set_variant.argtypes = [vp, i32]
        lib.sobel4_version.restype = ctypes.c_char_p
        lib.sobel4_check_magnitude.argtypes = [vp, i32, i32, ctypes.POINTER(ctypes.c_uint64)]
        lib.sobel4_run_batched_static.argtypes = [ctypes.POINTER(Image), i32, i32, i32, vp]
        fp = ctypes.POINTER(ctypes.c_float)
        lib.sobel4_tune.argtypes = [vp, i32, i32, i32, i32, fp]
        lib.sobel4_tune_batched.argtypes = [vp, ctypes.POINTER(Image), i32, i32, i32, fp]
        lib.sobel4_tune_entries.argtypes = [vp]
        lib.sobel4_tune_entries.restype = i32
        ip = ctypes.POINTER(i32)
        lib.sobel4_tune_config.argtypes = [vp, i32, i32, i32, ip, ip, ip]
        lib.sobel4_tune_save.argtypes = [vp, ctypes.c_char_p]
        lib.sobel4_tune_load.argtypes = [vp, ctypes.c_char_p]
        lib.sobel4_pipeline_create.argtypes = [vp, i32, i32, i32, i32, i32, ctypes.POINTER(vp)]
        lib.sobel4_pipeline_buffers.argtypes = [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                ctypes.POINTER(sz), ctypes.POINTER(sz)]
        lib.sobel4_pipeline_submit.argtypes = [vp, i32]
        lib.sobel4_pipeline_submit_from.argtypes = [vp, i32, vp, vp]
        lib.sobel4_pipeline_wait.argtypes = [vp, i32]
        lib.sobel4_pipeline_destroy.argtypes = [vp]
        lib.sobel4_host_alloc.argtypes = [sz, ctypes.POINTER(vp)]
        lib.sobel4_host_free.argtypes = [vp]
        lib.sobel4_server_create.argtypes = [vp, ctypes.POINTER(ServerOptions), ctypes.POINTER(vp)]
        lib.sobel4_server_submit.argtypes = [vp, vp, sz, vp, sz, i32, i32,
                                             ctypes.POINTER(ctypes.c_uint64)]
        lib.sobel4_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_double)]
        lib.sobel4_server_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        lib.sobel4_server_destroy.argtypes = [vp]
        for name in ("sobel4_create", "sobel4_destroy", "sobel4_run", "sobel4_run_rgb",
                     "sobel4_run_batched",
                     "sobel4_run_host", "sobel4_set_variant", "sobel4_check_magnitude",
                     "sobel4_device_status", "sobel4_inject_stage_loss", "sobel4_tune_config",
                     "sobel4_set_weights", "sobel4_set_operator", "sobel4_set_threshold",
                     "sobel4_run_batched_static", "sobel4_tune", "sobel4_tune_batched",
                     "sobel4_tune_save", "sobel4_tune_load", "sobel4_pipeline_create",
                     "sobel4_pipeline_buffers", "sobel4_pipeline_submit",
                     "sobel4_pipeline_submit_from", "sobel4_pipeline_wait",
                     "sobel4_pipeline_destroy", "sobel4_server_create", "sobel4_server_submit",
                     "sobel4_server_wait", "sobel4_server_stats", "sobel4_server_destroy"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


# -- one-to-one C ABI wrappers (raw pointers; return the status code) ----------
def sobel4_create(device: int = 0, variant: int = 0, rows_per_strip: int = 0,
                  persistent_ctas_per_sm: int = 0, columns_per_lane: int = 0, autotune: int = 0,
                  cache_path: str = None):
    h = ctypes.c_void_p()
    opt = Options(variant, rows_per_strip, persistent_ctas_per_sm, columns_per_lane, autotune,
                  cache_path.encode() if cache_path else None)
    st = load().sobel4_create(ctypes.byref(h), device, ctypes.byref(opt))
    return st, h


def sobel4_destroy(h) -> int:
    return load().sobel4_destroy(h)


def sobel4_run(h, d_src: int, src_pitch: int, d_dst: int, dst_pitch: int, height: int,
               width: int, border: int, fmt: int, stream: int) -> int:
    return load().sobel4_run(h, d_src, src_pitch, d_dst, dst_pitch, height, width, border, fmt,
                             stream)


def sobel4_run_rgb(h, d_src: int, src_pitch: int, d_dst: int, dst_pitch: int, height: int,
                   width: int, border: int, fmt: int, stream: int) -> int:
    """The operator on the gray of an interleaved RGB image (device pointers)."""
    return load().sobel4_run_rgb(h, d_src, src_pitch, d_dst, dst_pitch, height, width, border,
                                 fmt, stream)


def sobel4_run_batched(h, images, border: int, fmt: int, stream: int) -> int:
    arr = images if isinstance(images, ctypes.Array) else (Image * len(images))(*images)
    return load().sobel4_run_batched(h, arr, len(arr), border, fmt, stream)


def sobel4_run_batched_static(images, border: int, fmt: int, stream: int) -> int:
    """Allocation-free batched run on the current device (no handle)."""
    arr = images if isinstance(images, ctypes.Array) else (Image * len(images))(*images)
    return load().sobel4_run_batched_static(arr, len(arr), border, fmt, stream)


def sobel4_run_host(h, h_src: int, src_pitch: int, h_dst: int, dst_pitch: int, height: int,
                    width: int, border: int, fmt: int) -> int:
    return load().sobel4_run_host(h, h_src, src_pitch, h_dst, dst_pitch, height, width, border,
                                  fmt)


def sobel4_status_string(status: int) -> str:
    return load().sobel4_status_string(status).decode()


def sobel4_last_cuda_error(h) -> int:
    return load().sobel4_last_cuda_error(h)


def sobel4_device_status(h) -> int:
    return load().sobel4_device_status(h)


def sobel4_set_threshold(h, t: float) -> int:
    """EDGE8 threshold T for the handle's later runs (255 where sqrt(S) >= T)."""
    return load().sobel4_set_threshold(h, t)


def sobel4_set_operator(h, op: int) -> int:
    """Operator for the handle's later runs (OPERATORS)."""
    return load().sobel4_set_operator(h, op)


def sobel4_set_weights(h, a: float, b: float, n: float, m: float) -> int:
    """Eq. (5) weights for the handle's later runs (1, 2, 4, 6 = Eq. 3)."""
    return load().sobel4_set_weights(h, a, b, n, m)


def sobel4_inject_stage_loss(h, stage: int) -> int:
    return load().sobel4_inject_stage_loss(h, stage)


def sobel4_launch_count(h) -> int:
    return load().sobel4_launch_count(h)


def sobel4_set_variant(h, variant: int) -> int:
    return load().sobel4_set_variant(h, variant)


def sobel4_check_magnitude(h, s_begin: int, s_end: int):
    """(status, mismatches) of the on-device magnitude self-check over [s_begin, s_end)."""
    n = ctypes.c_uint64()
    st = load().sobel4_check_magnitude(h, s_begin, s_end, ctypes.byref(n))
    return st, n.value


def sobel4_tune(h, height: int, width: int, border: int, fmt: int):
    """(status, best_us) of the per-shape autotuner."""
    us = ctypes.c_float()
    st = load().sobel4_tune(h, height, width, border, fmt, ctypes.byref(us))
    return st, us.value


def sobel4_tune_batched(h, images, border: int, fmt: int):
    """(status, best_us) of the batch autotuner (runs the batch repeatedly)."""
    arr = images if isinstance(images, ctypes.Array) else (Image * len(images))(*images)
    us = ctypes.c_float()
    st = load().sobel4_tune_batched(h, arr, len(arr), border, fmt, ctypes.byref(us))
    return st, us.value


def sobel4_tune_entries(h) -> int:
    return load().sobel4_tune_entries(h)


def sobel4_tune_config(h, height: int, width: int, fmt: int):
    """(status, kernel, columns_per_lane, rows_per_strip) used for aligned images of the shape."""
    k, nc, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    st = load().sobel4_tune_config(h, height, width, fmt, ctypes.byref(k), ctypes.byref(nc),
                                   ctypes.byref(r))
    return st, k.value, nc.value, r.value


def sobel4_tune_save(h, path: str) -> int:
    return load().sobel4_tune_save(h, path.encode())


def sobel4_tune_load(h, path: str) -> int:
    return load().sobel4_tune_load(h, path.encode())


def sobel4_pipeline_create(h, height: int, width: int, border: int, fmt: int, slots: int):
    p = ctypes.c_void_p()
    st = load().sobel4_pipeline_create(h, height, width, border, fmt, slots, ctypes.byref(p))
    return st, p


def sobel4_pipeline_buffers(p, slot: int):
    """(status, h_in, h_out, in_pitch, out_pitch) of one slot."""
    a, b = ctypes.c_void_p(), ctypes.c_void_p()
    ip, op = ctypes.c_size_t(), ctypes.c_size_t()
    st = load().sobel4_pipeline_buffers(p, slot, ctypes.byref(a), ctypes.byref(b),
                                        ctypes.byref(ip), ctypes.byref(op))
    return st, a.value, b.value, ip.value, op.value


def sobel4_pipeline_submit(p, slot: int) -> int:
    return load().sobel4_pipeline_submit(p, slot)


def sobel4_pipeline_submit_from(p, slot: int, h_in: int, h_out: int) -> int:
    """Launch the slot on caller host buffers (0 keeps the slot's own buffer)."""
    return load().sobel4_pipeline_submit_from(p, slot, h_in or None, h_out or None)


def sobel4_pipeline_wait(p, slot: int) -> int:
    return load().sobel4_pipeline_wait(p, slot)


def sobel4_pipeline_destroy(p) -> int:
    return load().sobel4_pipeline_destroy(p)


def sobel4_host_alloc(nbytes: int):
    """(status, address) of `nbytes` of page-locked host memory."""
    p = ctypes.c_void_p()
    st = load().sobel4_host_alloc(nbytes, ctypes.byref(p))
    return st, p.value or 0


def sobel4_host_free(address: int) -> int:
    return load().sobel4_host_free(address or None)


class HostBuffer:
    """Page-locked host memory from sobel4_host_alloc with a numpy view
    (``.array``, `dtype` x `shape`); freed by close() or garbage collection."""

    def __init__(self, shape, dtype="uint8"):
        import numpy as np
        self.shape = tuple(shape) if hasattr(shape, "__len__") else (int(shape),)
        self.dtype = np.dtype(dtype)
        nbytes = int(np.prod(self.shape)) * self.dtype.itemsize
        st, self.address = sobel4_host_alloc(nbytes)
        _check(st, "sobel4_host_alloc")
        raw = (ctypes.c_uint8 * nbytes).from_address(self.address)
        self.array = np.frombuffer(raw, dtype=self.dtype).reshape(self.shape)

    def close(self):
        if self.address:
            self.array = None
            _check(sobel4_host_free(self.address), "sobel4_host_free")
            self.address = 0

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Pipeline:
    """numpy views over a graph-captured video pipeline's pinned slot buffers."""

    def __init__(self, sobel: "Sobel4", height: int, width: int, border: str = "valid",
                 fmt: str = "f32", slots: int = 2):
        import numpy as np
        st, p = sobel4_pipeline_create(sobel.handle, height, width, BORDERS[border],
                                       FORMATS[fmt], slots)
        _check(st, "sobel4_pipeline_create")
        self.p, self.slots, self.H, self.W, self.fmt = p, slots, height, width, fmt
        dtype = {"f32": np.float32, "u8": np.uint8, "s16x4": np.int16, "u16": np.uint16, "edge8": np.uint8}[fmt]
        planes = 4 if fmt == "s16x4" else 1
        self.inputs, self.outputs = [], []
        for k in range(slots):
            st, a, b, ip, op = sobel4_pipeline_buffers(p, k)
            _check(st, "sobel4_pipeline_buffers")
            raw_in = (ctypes.c_uint8 * (ip * height)).from_address(a)
            raw_out = (ctypes.c_uint8 * (op * height * planes)).from_address(b)
            vin = np.frombuffer(raw_in, dtype=np.uint8).reshape(height, ip)[:, :width]
            vout = np.frombuffer(raw_out, dtype=np.uint8).reshape(planes * height, op)
            vout = vout[:, :width * ELEM_SIZE[fmt]].view(dtype)
            self.inputs.append(vin)
            self.outputs.append(vout.reshape(4, height, width) if planes == 4 else vout)

    def submit(self, slot: int):
        _check(sobel4_pipeline_submit(self.p, slot), "sobel4_pipeline_submit")

    def submit_from(self, slot: int, h_in: int, h_out: int = 0):
        """Launch the slot on a caller frame (pinned host address of height rows at
        the input pitch); the result goes to h_out, or to the slot's output if 0."""
        _check(sobel4_pipeline_submit_from(self.p, slot, h_in, h_out),
               "sobel4_pipeline_submit_from")

    def wait(self, slot: int):
        _check(sobel4_pipeline_wait(self.p, slot), "sobel4_pipeline_wait")

    def close(self):
        if getattr(self, "p", None):
            sobel4_pipeline_destroy(self.p)
            self.p = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def sobel4_server_create(h, memory_budget: int = 0, max_batch: int = 0, border: int = 0,
                         fmt: int = 0, plain: int = 0):
    srv = ctypes.c_void_p()
    opt = ServerOptions(memory_budget, max_batch, border, fmt, plain)
    st = load().sobel4_server_create(h, ctypes.byref(opt), ctypes.byref(srv))
    return st, srv


def sobel4_server_submit(srv, h_src: int, src_pitch: int, h_dst: int, dst_pitch: int,
                         height: int, width: int):
    """(status, ticket)."""
    t = ctypes.c_uint64()
    st = load().sobel4_server_submit(srv, h_src, src_pitch, h_dst, dst_pitch, height, width,
                                     ctypes.byref(t))
    return st, t.value


def sobel4_server_wait(srv, ticket: int, timeout_us: int = -1):
    """(status, latency_us)."""
    lat = ctypes.c_double()
    st = load().sobel4_server_wait(srv, ticket, timeout_us, ctypes.byref(lat))
    return st, lat.value


def sobel4_server_stats(srv):
    out = ServerStats()
    st = load().sobel4_server_stats(srv, ctypes.byref(out))
    return st, {f: getattr(out, f) for f, _ in ServerStats._fields_}


def sobel4_server_destroy(srv) -> int:
    return load().sobel4_server_destroy(srv)


def sobel4_version() -> str:
    return load().sobel4_version().decode()


# -- tensor-level convenience --------------------------------------------------
def _check(st: int, what: str):
    if st != 0:
        raise Sobel4Error(st, what)


class Sobel4:
    """A library handle bound to one CUDA device."""

    def __init__(self, device: int = 0, variant: str = "auto", rows_per_strip: int = 0,
                 persistent_ctas_per_sm: int = 0, columns_per_lane: int = 0,
                 autotune: bool = False, cache_path: str = None):
        st, h = sobel4_create(device, VARIANTS[variant], rows_per_strip, persistent_ctas_per_sm,
                              columns_per_lane, int(autotune), cache_path)
        _check(st, "sobel4_create")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            sobel4_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def launches(self) -> int:
        return sobel4_launch_count(self.handle)

    def set_variant(self, variant: str):
        _check(sobel4_set_variant(self.handle, VARIANTS[variant]), "sobel4_set_variant")

    def set_threshold(self, t: float = 128.0):
        """EDGE8 threshold (255 where sqrt(S) >= t)."""
        _check(sobel4_set_threshold(self.handle, t), "sobel4_set_threshold")

    def set_operator(self, name: str = "4dir5x5"):
        """4dir5x5 (Eq. 3), 2dir5x5 or 2dir3x3 (Eq. 1-2)."""
        _check(sobel4_set_operator(self.handle, OPERATORS[name]), "sobel4_set_operator")

    def set_weights(self, a: float = 1, b: float = 2, n: float = 4, m: float = 6):
        """The generalised operator of Eq. (5); the defaults restore Eq. (3)."""
        _check(sobel4_set_weights(self.handle, a, b, n, m), "sobel4_set_weights")

    @staticmethod
    def _stream(stream) -> int:
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)

    @staticmethod
    def empty_output(src, fmt: str = "f32"):
        import torch
        H, W = src.shape
        dtype = {"f32": torch.float32, "u8": torch.uint8, "s16x4": torch.int16, "u16": torch.uint16, "edge8": torch.uint8}[fmt]
        shape = (4, H, W) if fmt == "s16x4" else (H, W)
        return torch.empty(shape, dtype=dtype, device=src.device)

    @staticmethod
    def _pitches(src, out, fmt):
        import torch
        if src.dtype != torch.uint8 or src.dim() != 2 or not src.is_cuda or src.stride(1) != 1:
            raise ValueError("src must be a 2-D uint8 CUDA tensor with unit column stride")
        if out.stride(-1) != 1:
            raise ValueError("out must have unit column stride")
        if fmt == "s16x4":
            if out.dim() != 3 or out.shape[0] != 4 or out.stride(0) != out.shape[1] * out.stride(1):
                raise ValueError("s16x4 output must be 4 stacked planes")
        return src.stride(0), out.stride(-2) * ELEM_SIZE[fmt]

    def run(self, src, out=None, border: str = "valid", fmt: str = "f32", stream=None):
        """Gradient output of a uint8 CUDA tensor [H, W]; asynchronous on `stream`."""
        if out is None:
            out = self.empty_output(src, fmt)
        sp, dp = self._pitches(src, out, fmt)
        H, W = src.shape
        _check(sobel4_run(self.handle, src.data_ptr(), sp, out.data_ptr(), dp, H, W,
                          BORDERS[border], FORMATS[fmt], self._stream(stream)), "sobel4_run")
        return out

    def run_rgb(self, src, out=None, border: str = "valid", fmt: str = "f32", stream=None):
        """Gradient output of the gray of a uint8 CUDA tensor [H, W, 3] (interleaved
        RGB, rows may be strided); asynchronous on `stream`."""
        H, W, C = src.shape
        if C != 3 or src.stride(2) != 1 or src.stride(1) != 3:
            raise ValueError("src must be a uint8 [H, W, 3] tensor with interleaved pixels")
        if out is None:
            out = self.empty_output(src[:, :, 0], fmt)
        dp = out.stride(-2) * ELEM_SIZE[fmt]
        _check(sobel4_run_rgb(self.handle, src.data_ptr(), src.stride(0), out.data_ptr(), dp, H,
                              W, BORDERS[border], FORMATS[fmt], self._stream(stream)),
               "sobel4_run_rgb")
        return out

    def run_batched(self, srcs, outs=None, border: str = "valid", fmt: str = "f32",
                    stream=None):
        """Many images in one persistent launch; returns the outputs."""
        if outs is None:
            outs = [self.empty_output(s, fmt) for s in srcs]
        imgs = (Image * len(srcs))()
        for i, (s, o) in enumerate(zip(srcs, outs)):
            sp, dp = self._pitches(s, o, fmt)
            imgs[i] = Image(s.data_ptr(), sp, o.data_ptr(), dp, s.shape[0], s.shape[1])
        _check(sobel4_run_batched(self.handle, imgs, BORDERS[border], FORMATS[fmt],
                                  self._stream(stream)), "sobel4_run_batched")
        return outs

    def run_host(self, src, out=None, border: str = "valid", fmt: str = "f32"):
        """End to end from a host numpy array (synchronous)."""
        import numpy as np
        if src.dtype != np.uint8 or src.ndim != 2 or src.strides[1] != 1:
            raise ValueError("src must be a 2-D uint8 array with unit column stride")
        H, W = src.shape
        if out is None:
            dtype = {"f32": np.float32, "u8": np.uint8, "s16x4": np.int16, "u16": np.uint16, "edge8": np.uint8}[fmt]
            out = np.empty((4, H, W) if fmt == "s16x4" else (H, W), dtype=dtype)
        _check(sobel4_run_host(self.handle, src.ctypes.data, src.strides[0], out.ctypes.data,
                               out.strides[-2], H, W, BORDERS[border], FORMATS[fmt]),
               "sobel4_run_host")
        return out
