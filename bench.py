#!/usr/bin/env python
"""Benchmark of the four-directional 5x5 Sobel operator on GB300.

One step = one pass of the whole operator (all four masks, Eq. 3; the
magnitude, Eq. 4) over one 8192x8192 uint8 image into float32 with the
paper's border rule -- the largest image of the single-image size sweep, the
one the headline Gpixel/s and HBM roofline are quoted on.

Default (our arm): prints one JSON line with
  value          Gpixel/s, device-timed, inputs resident in HBM; consecutive
                 steps rotate over buffer sets whose combined footprint
                 exceeds the 129 MB L2, so no step reads another's cached data;
  roofline       the RG kernel's algorithmic bytes (1 B in + 4 B out per pixel)
                 over its mean CUDA-event duration, against the measured HBM peak;
  e2e            the same metric through sobel4_run_host (pinned host buffers,
                 host->device copy, kernel, device->host copy every step);
  cpu_baseline   the CPU oracle on all of this host's cores over a bounded sample
                 (and on one core: "one_core");
  clocks         nvidia-smi SM clocks and throttle reasons sampled during the run.
Under torchrun (N > 1) each rank processes its own image (weak scaling, no
collective on the data path); the time is the max over ranks.

--impl reference runs the CPU oracle as the reference arm (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4-dir 5x5 Sobel Gpixel/s and % of HBM peak; batched/served p50/p99 latency"
H, W = 8192, 8192
BYTES_PER_PX = 5  # 1 B read + 4 B written (F32)
WORKLOAD = "single 8192x8192 uint8 rects+noise image -> float32 gradient magnitude, paper border rule (VALID)"
L2_BYTES = 129 * 2 ** 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows-per-strip", type=int, default=0)
    ap.add_argument("--variant", choices=["auto", "rg", "tc"], default="auto",
                    help="kernel variant of the timed handle (auto: the tuner's choice)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (built-in strip-height rule)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, video and serving measurements")
    ap.add_argument("--video-frames", type=int, default=2000)
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the Poisson serving run per mode (the configuration's 60 s)")
    ap.add_argument("--profile-batch", type=int, default=0, metavar="N",
                    help="run the first N images of the 512-image ragged batch (seed 1) through "
                         "sobel4_run_batched twice and exit (a capture target for ncu)")
    ap.add_argument("--profile-single", choices=["rgb", "weights", "pitch"], default=None,
                    help="launch one image twice, then exit (for ncu): 8192x8192 through the "
                         "colour input or the runtime-weight path, or the size sweep's "
                         "1920x1080 pitch-1937/7748 case")
    ap.add_argument("--profile-variants", action="store_true",
                    help="run every kernel variant twice on the workload image and exit "
                         "(a capture target for ncu; prints no JSON line)")
    return ap.parse_args()


# ----------------------------------------------------------------------------
def dist_setup(gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def max_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time (every rank calls this)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(px_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job Gpixel/s: every rank's pixels over the slowest rank's time."""
    return world * px_per_rank * steps / (max_ms * 1e-3) / 1e9


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling in the background."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        util = [num(r[4]) for r in self.rows]
        loaded = [num(r[1]) for r in self.rows if num(r[4]) is not None and num(r[4]) >= 50
                  and num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(loaded or sm) if (loaded or sm) else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows), "samples_under_load": len(loaded),
                "power_w_max": max((num(r[3]) for r in self.rows if num(r[3]) is not None),
                                   default=None)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Sources of each timed kernel family: its own files plus the shared device
# headers (arithmetic, PTX wrappers, descriptors, launch declarations).
KERNEL_SOURCES = {"tma": "sobel4_tma", "lanecopy": "sobel4_rg", "tc": "sobel4_tc"}
SHARED_SOURCES = ("sobel4_arith.cuh", "sobel4_device.cuh", "sobel4_ptx.cuh", "sobel4_launch.h")


def code_only(text: str) -> str:
    """C++ source without its comments and blank lines (what the compiler sees)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_source_hash(stem: str = "tma") -> str:
    """SHA-256 (first 16 hex digits) of the code, comments stripped, of the
    sources the `stem` kernel family is compiled from; a committed ncu summary
    carries the value it was taken on."""
    csrc = os.path.join(ROOT, "paper_2305_00515_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if name in SHARED_SOURCES or (name.startswith(KERNEL_SOURCES.get(stem, "\0")) and
                                      name.endswith((".cu", ".cuh", ".h"))):
            with open(os.path.join(csrc, name), encoding="utf-8") as f:
                h.update(name.encode() + code_only(f.read()).encode())
    return h.hexdigest()[:16]


KERNELS = {0: ("lanecopy", "rg_single_kernel<F32>"), 1: ("tma", "tma_single_kernel<F32>"),
           2: ("tc", "tc_single_kernel<F32>")}


def recorded_traffic(stem: str):
    """DRAM bytes per launch of the timed kernel from its committed ncu summary
    (profiles/<stem>_f32_8192_full.md, lines "kernel_source_hash: ..." and
    "dram_bytes_per_launch: ..."), only when that capture was taken on the
    current kernel source; otherwise None."""
    path = os.path.join(ROOT, "profiles", f"{stem}_f32_8192_full.md")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as f:
        for line in f:
            line = line.strip().lstrip("-* ").replace("`", "")
            if ":" in line:
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
    if fields.get("kernel_source_hash") != kernel_source_hash(stem):
        return None
    try:
        return int(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ----------------------------------------------------------------------------
def _events(torch, n):
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(n)]


def bench_batched(torch, pkg, synth, reps: int = 5):
    """512 ragged images (sides U{37..2048}, seed 1) as ONE persistent launch
    versus 512 single-image launches on one stream; F32, paper border rule."""
    import numpy as np
    imgs = synth.batch_images(512, 1)
    px = sum(i.size for i in imgs)
    srcs = [torch.from_numpy(i).cuda() for i in imgs]
    outs_b = [torch.empty(i.shape, dtype=torch.float32, device="cuda") for i in imgs]
    outs_s = [torch.empty(i.shape, dtype=torch.float32, device="cuda") for i in imgs]
    st, h = pkg.sobel4_create(0)
    assert st == 0
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    descs = (pkg.Image * len(imgs))(*[pkg.Image(s.data_ptr(), s.stride(0), o.data_ptr(),
                                                 o.stride(0) * 4, *s.shape)
                                      for s, o in zip(srcs, outs_b)])
    tuned = pkg.sobel4_tune_batched(h, descs, 0, 0)[1]
    sha = hashlib.sha256()
    for i in imgs:
        sha.update(np.array(i.shape, dtype=np.int64).tobytes() + i.tobytes())

    def batched():
        assert pkg.sobel4_run_batched(h, descs, 0, 0, sh) == 0

    def singles():
        for s_, o in zip(srcs, outs_s):
            assert pkg.sobel4_run(h, s_.data_ptr(), s_.stride(0), o.data_ptr(), o.stride(0) * 4,
                                  s_.shape[0], s_.shape[1], 0, 0, sh) == 0

    res = {}
    n0 = pkg.sobel4_launch_count(h)
    batched()
    per_call = pkg.sobel4_launch_count(h) - n0
    for name, fn in (("one_persistent_launch", batched), ("separate_launches", singles)):
        for _ in range(2):
            fn()
        ev = _events(torch, reps)
        with torch.cuda.stream(stream):
            for a, b in ev:
                a.record(stream)
                fn()
                b.record(stream)
        stream.synchronize()
        ms = sorted(a.elapsed_time(b) for a, b in ev)
        res[name] = {"ms_median": ms[len(ms) // 2], "gpix_s": px / (ms[len(ms) // 2] * 1e-3) / 1e9,
                     "frac_of_hbm_peak": px * BYTES_PER_PX / (ms[len(ms) // 2] * 1e-3) / 1e9 /
                     measured_peaks()[0]}
    torch.cuda.synchronize()
    same = all(torch.equal(a, b) for a, b in zip(outs_b, outs_s))
    import oracle
    for k in (0, 100, 511):
        assert np.array_equal(outs_b[k].cpu().numpy().view(np.uint32),
                              oracle.default().sobel4(imgs[k], "valid", "f32",
                                                      threads=8).view(np.uint32))
    pkg.sobel4_destroy(h)
    return {"workload": "512 ragged uint8 images, sides U{37..2048} (seed 1), F32, VALID",
            "pixels": px, "inputs_sha256": sha.hexdigest(),
            "launches_per_call": {"total": int(per_call), "batched_kernels": 1,
                                  "descriptor_uploads": int(per_call) - 1},
            **res, "speedup": res["separate_launches"]["ms_median"] /
            res["one_persistent_launch"]["ms_median"], "tuned_us": tuned,
            "batch_equals_single_runs": bool(same)}


SWEEP_SHAPES = ((1024, 1024), (1080, 1920), (2160, 3840), (4096, 4096), (8192, 8192))


def bench_sweep(torch, pkg, synth, peak: float, reps: int = 20):
    """The single-image size sweep: 1024^2, 1920x1080, 3840x2160, 4096^2 and
    8192^2, each as rects+noise and as i.i.d. uniform noise, tight pitches,
    plus 1920x1080 rects+noise at source pitch 1937 / destination pitch 7748
    bytes (odd and unaligned rows).  Each shape is autotuned once (untimed);
    each case is timed over `reps` back-to-back launches rotating over buffer
    sets that together exceed twice the L2, after 3 warm-up launches.  Four
    rows of the last output are checked bit for bit against the CPU oracle."""
    import numpy as np

    import oracle
    cases = [(H, W, c, W, 4 * W) for (H, W) in SWEEP_SHAPES for c in ("rects", "uniform")]
    cases.append((1080, 1920, "rects", 1937, 7748))
    st, h = pkg.sobel4_create(0)
    assert st == 0
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    tuned, out = set(), []
    for (H, W, content, sp, dp) in cases:
        img = synth.rects_noise(H, W, 11) if content == "rects" else synth.uniform(H, W, 11)
        if (H, W) not in tuned:
            st, _ = pkg.sobel4_tune(h, H, W, 0, 0)
            assert st == 0, pkg.sobel4_status_string(st)
            tuned.add((H, W))
        per_set = H * (sp + dp)
        nsets = max(2, -(-2 * L2_BYTES // per_set) + 1)
        host = torch.from_numpy(img)
        srcs, outs = [], []
        for _ in range(nsets):
            t = torch.empty((H, sp), dtype=torch.uint8, device="cuda")
            t[:, :W].copy_(host)
            srcs.append(t)
            outs.append(torch.empty((H, dp // 4), dtype=torch.float32, device="cuda"))

        def launch(i):
            rc = pkg.sobel4_run(h, srcs[i % nsets].data_ptr(), sp, outs[i % nsets].data_ptr(), dp,
                                H, W, 0, 0, sh)
            assert rc == 0, pkg.sobel4_status_string(rc)

        for i in range(3):
            launch(i)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            for i in range(reps):
                launch(3 + i)
            b.record(stream)
        stream.synchronize()
        us = a.elapsed_time(b) * 1e3 / reps
        y0 = H // 2
        got = outs[(2 + reps) % nsets][y0:y0 + 4, :W].cpu().numpy()
        want = oracle.default().sobel4(img[y0 - 2:y0 + 6], "valid", "f32")[2:6]
        out.append({"height": H, "width": W, "content": content, "src_pitch": sp, "dst_pitch": dp,
                    "us": round(us, 2), "gpix_s": round(H * W / (us * 1e-6) / 1e9, 1),
                    "frac": round(H * W * BYTES_PER_PX / (us * 1e-6) / 1e9 / peak, 4),
                    "rows_match_oracle": bool(np.array_equal(got.view(np.uint32),
                                                             want.view(np.uint32))),
                    "input_sha256": hashlib.sha256(img.tobytes()).hexdigest()})
        del srcs, outs
    pkg.sobel4_destroy(h)
    torch.cuda.empty_cache()
    return {"workload": "single images, F32 VALID, rects+noise and uniform, tight pitches plus "
                        "the 1920x1080 pitch-1937/7748 variant; frac of measured HBM peak at "
                        f"{BYTES_PER_PX} B/px; back-to-back launches over buffer sets > 2x L2",
            "cases": out}


def bench_rgb(torch, pkg, synth, peak: float, reps: int = 20):
    """The fused colour input: an 8192x8192 interleaved RGB image (three
    differently seeded rects+noise channels) -> gray (Y = (77R + 150G + 29B +
    128) >> 8, inside the kernel) -> F32 VALID.  Algorithmic bytes 3 read + 4
    written per pixel.  Back-to-back launches over two buffer sets (each 470 MB,
    > 2x L2) after 3 warm-up launches; four rows checked against the oracle."""
    import numpy as np

    import oracle
    H = W = 8192
    rgb = np.stack([synth.rects_noise(H, W, 50 + c) for c in range(3)], axis=2)
    srcs = [torch.from_numpy(rgb).cuda() for _ in range(2)]
    outs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in range(2)]
    stream = torch.cuda.Stream()
    st, h = pkg.sobel4_create(0)
    assert st == 0

    def launch(i):
        rc = pkg.sobel4_run_rgb(h, srcs[i % 2].data_ptr(), 3 * W, outs[i % 2].data_ptr(), 4 * W,
                                H, W, 0, 0, stream.cuda_stream)
        assert rc == 0, pkg.sobel4_status_string(rc)

    for i in range(3):
        launch(i)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        for i in range(reps):
            launch(3 + i)
        b.record(stream)
    stream.synchronize()
    us = a.elapsed_time(b) * 1e3 / reps
    y0 = 4000
    got = outs[(2 + reps) % 2][y0:y0 + 4].cpu().numpy()
    want = oracle.default().sobel4_rgb(rgb[y0 - 2:y0 + 6], "valid", "f32")[2:6]
    assert pkg.sobel4_device_status(h) == 0
    pkg.sobel4_destroy(h)
    del srcs, outs
    torch.cuda.empty_cache()
    return {"workload": "8192x8192 interleaved RGB -> gray in the kernel -> F32 VALID",
            "us": us, "gpix_s": H * W / (us * 1e-6) / 1e9, "bytes_per_px": 7,
            "frac": H * W * 7 / (us * 1e-6) / 1e9 / peak,
            "rows_match_oracle": bool(np.array_equal(got.view(np.uint32), want.view(np.uint32))),
            "input_sha256": hashlib.sha256(rgb.tobytes()).hexdigest()}


def bench_runtime_weights(torch, pkg, synth, peak: float, eq3_us: float, reps: int = 20):
    """Runtime weights of Eq. (5), (a, b, n, m) = (2, 1.5, 2, 2), on the
    8192x8192 headline image (F32 VALID) through the register-window kernel
    with the weights' coefficients (strip height autotuned like the headline
    leg's); compared with the Eq. (3) kernel's time from the headline leg.  Back-to-back launches over two buffer sets (> 2x
    L2); four rows checked against the oracle's Eq. (5) masks."""
    import numpy as np

    import oracle
    H = W = 8192
    abnm = (2, 1.5, 2, 2)
    img = synth.rects_noise(H, W, 0)
    srcs = [torch.from_numpy(img).cuda() for _ in range(2)]
    outs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in range(2)]
    stream = torch.cuda.Stream()
    st, h = pkg.sobel4_create(0)
    assert st == 0 and pkg.sobel4_set_weights(h, *abnm) == 0
    st, _ = pkg.sobel4_tune(h, H, W, 0, 0)  # strip height for these coefficients
    assert st == 0, pkg.sobel4_status_string(st)
    _, kind, _, rows = pkg.sobel4_tune_config(h, H, W, 0)

    def launch(i):
        rc = pkg.sobel4_run(h, srcs[i % 2].data_ptr(), W, outs[i % 2].data_ptr(), 4 * W, H, W,
                            0, 0, stream.cuda_stream)
        assert rc == 0, pkg.sobel4_status_string(rc)

    for i in range(3):
        launch(i)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        for i in range(reps):
            launch(3 + i)
        b.record(stream)
    stream.synchronize()
    us = a.elapsed_time(b) * 1e3 / reps
    y0 = 4000
    got = outs[(2 + reps) % 2][y0:y0 + 4].cpu().numpy()
    want = oracle.default().sobel4(img[y0 - 2:y0 + 6], "valid", "f32",
                                   masks=oracle.eq5_masks(*abnm))[2:6]
    pkg.sobel4_destroy(h)
    del srcs, outs
    torch.cuda.empty_cache()
    return {"workload": "8192x8192 rects+noise, F32 VALID, Eq. (5) weights (a, b, n, m) = "
                        "(2, 1.5, 2, 2)",
            "kernel": {1: "register window (packed passes, runtime coefficients)",
                       2: "tensor core", 3: "direct"}.get(kind, str(kind)),
            "autotuned_rows_per_strip": rows,
            "us": us, "gpix_s": H * W / (us * 1e-6) / 1e9,
            "frac": H * W * BYTES_PER_PX / (us * 1e-6) / 1e9 / peak,
            "vs_eq3_time": us / eq3_us,
            "rows_match_oracle": bool(np.array_equal(got.view(np.uint32), want.view(np.uint32)))}


def bench_ablation(torch, pkg, synth):
    """The paper's kernel ladder (Table 1, 5x5 four-directional) re-measured
    here: GM = the direct 25-tap kernel; SM, SM-P, RG, RG-v1, RG-v2 = the
    ladder variants in the paper's plain form (shared-memory tile, with
    prefetching, register window with the diagonals direct / through K_d+ /
    fully decomposed); then the GB300 kernels: the packed register window
    with per-lane copies and with TMA staging, and the tensor-core variant.
    F32 VALID, mean CUDA-event time per launch (images up to 2048^2 stay in
    L2 between launches, as in the paper's repeated runs)."""
    variants = (("GM_direct", "direct"), ("SM", "ladder_sm"), ("SM_P", "ladder_sm_p"),
                ("RG", "ladder_rg"), ("RG_v1", "ladder_rg_v1"), ("RG_v2", "ladder_rg_v2"),
                ("RG_lanecopy", "rg_lanecopy"), ("RG_tma", "rg"), ("TC_tensor_core", "tc"))
    res = {}
    stream = torch.cuda.Stream()
    for side in (512, 1024, 2048, 8192):
        img = synth.rects_noise(side, side, side)
        src = torch.from_numpy(img).cuda()
        out = torch.empty((side, side), dtype=torch.float32, device="cuda")
        row = {}
        for name, variant in variants:
            st, h = pkg.sobel4_create(0, pkg.VARIANTS[variant])
            assert st == 0

            def launch():
                assert pkg.sobel4_run(h, src.data_ptr(), side, out.data_ptr(), 4 * side, side, side,
                                      0, 0, stream.cuda_stream) == 0
            for _ in range(5):
                launch()
            n = 50 if side <= 2048 else 20
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                a.record(stream)
                for _ in range(n):
                    launch()
                b.record(stream)
            stream.synchronize()
            row[name] = round(a.elapsed_time(b) * 1e3 / n, 2)
            pkg.sobel4_destroy(h)
        res[f"{side}x{side}"] = row
    return {"workload": "one rects+noise image per size, F32 VALID; microseconds per launch",
            **res}


def host_link_probe(torch, in_bytes: int, out_bytes: int, reps: int = 20):
    """Plain cudaMemcpyAsync between pinned host memory and the device, in the
    sizes of one frame's copies: host->device alone, device->host alone, and
    both directions at once on two streams.  The last is the ceiling of any
    pipeline that moves those bytes per frame."""
    hi = torch.empty(in_bytes, dtype=torch.uint8, pin_memory=True)
    ho = torch.empty(out_bytes, dtype=torch.uint8, pin_memory=True)
    di = torch.empty(in_bytes, dtype=torch.uint8, device="cuda")
    do = torch.empty(out_bytes, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def run(h2d: bool, d2h: bool) -> float:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            if h2d:
                with torch.cuda.stream(s1):
                    di.copy_(hi, non_blocking=True)
            if d2h:
                with torch.cuda.stream(s2):
                    ho.copy_(do, non_blocking=True)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    run(True, True)  # warm up
    t_in, t_out, t_both = run(True, False), run(False, True), run(True, True)
    return {"h2d_gb_s": reps * in_bytes / t_in / 1e9, "d2h_gb_s": reps * out_bytes / t_out / 1e9,
            "both_directions_gb_s": reps * (in_bytes + out_bytes) / t_both / 1e9,
            "ceiling_frames_per_s": reps / t_both}


def bench_video(torch, pkg, synth, frames: int, slots: int = 4):
    """Frames of 3840x2160 through the graph-captured pipeline (H2D + kernel +
    D2H per frame, `slots` frame slots).  All `frames` frames are distinct --
    frame k is the background translated by (k mod 17, 2k mod 13) with fresh
    noise keyed by k -- and are generated, untimed, into a page-locked host
    ring (sobel4_host_alloc) before the timed loop; each submit hands the
    slot its frame (upload, the slot's kernel graph, download).  Reported against a plain-copy ceiling of the host link; then an
    untimed pass checks every frame's output against a single-image launch on
    the same frame (bit for bit, on the device) and three frames against the
    CPU oracle."""
    import numpy as np

    import oracle
    H, W = 2160, 3840
    fb = H * W
    bg = synth.video_background(H, W, 3)
    ring_buf = pkg.HostBuffer((frames, H, W), "uint8")  # page-locked (sobel4_host_alloc)
    ring = ring_buf.array
    try:
        t0 = time.perf_counter()
        for k0 in range(0, frames, 64):
            chunk = synth.video_frames_torch(bg, k0, min(64, frames - k0), H, W, 3)
            torch.from_numpy(ring[k0:k0 + chunk.shape[0]]).copy_(chunk)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        sha = hashlib.sha256()
        for k in range(0, frames, max(1, frames // 16)):
            sha.update(ring[k].tobytes())
        link = host_link_probe(torch, fb, fb * 4)
        base = ring.ctypes.data
        with pkg.Sobel4(0) as s:
            pipe = pkg.Pipeline(s, H, W, "valid", "f32", slots=slots)
            for k in range(slots):  # warm up
                pipe.submit_from(k, base + k * fb)
            for k in range(slots):
                pipe.wait(k)
            t0 = time.perf_counter()
            for k in range(frames):
                slot = k % slots
                pipe.wait(slot)
                pipe.submit_from(slot, base + k * fb)
            for k in range(slots):
                pipe.wait(k)
            dt = time.perf_counter() - t0
            # untimed checks: every frame against a single-image launch on the device
            d_in = torch.empty((H, W), dtype=torch.uint8, device="cuda")
            d_ref = torch.empty((H, W), dtype=torch.float32, device="cuda")
            d_got = torch.empty((H, W), dtype=torch.float32, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            mismatched = []
            oracle_checked = {}
            for k in range(frames):
                pipe.submit_from(0, base + k * fb)
                d_in.copy_(torch.from_numpy(ring[k]))
                rc = pkg.sobel4_run(s.handle, d_in.data_ptr(), W, d_ref.data_ptr(), W * 4, H, W,
                                    0, 0, stream)
                assert rc == 0
                pipe.wait(0)
                d_got.copy_(torch.from_numpy(pipe.outputs[0]))
                if not torch.equal(d_got.view(torch.int32), d_ref.view(torch.int32)):
                    mismatched.append(k)
                if k in (0, frames // 2, frames - 1):
                    want = oracle.default().sobel4(ring[k], "valid", "f32",
                                                   threads=oracle.cpu_count())
                    oracle_checked[k] = bool(np.array_equal(
                        np.ascontiguousarray(pipe.outputs[0]).view(np.uint32), want.view(np.uint32)))
            pipe.close()
    finally:
        ring = None
        ring_buf.close()
    fps = frames / dt
    return {"workload": f"{frames} distinct frames of 3840x2160 u8 -> f32 through {slots} graph "
                        "slots, from a page-locked host ring generated beforehand (untimed)",
            "frames_per_s": fps, "ms_per_frame": 1e3 / fps, "gpix_s": fps * fb / 1e9,
            "host_link_gb_s": fps * fb * 5 / 1e9, "link_probe": link,
            "link_ceiling_gb_s": link["both_directions_gb_s"],
            "frac_of_link_ceiling": fps / link["ceiling_frames_per_s"],
            "all_frames_match": not mismatched, "mismatched_frames": mismatched[:10],
            "oracle_frames_match": oracle_checked, "frames_generated_s": gen_s,
            "inputs_sha256_every_16th_part": sha.hexdigest()}


SERVING_MODES = (("plain_one_stream", 2), ("batched", 0))


def bench_serving(torch, pkg, synth, seconds: float):
    """Poisson arrivals (400 req/s for `seconds`) of the serving resolution mix
    through the continuous-batching server (batched), against one sobel4_run
    per request in arrival order on one stream (plain_one_stream: the same
    server with plain = 2, so both share the host machinery).  Results land
    in the client's pinned buffers, written there by the kernels.  Each mode's
    server first serves the trace's first 5 s untimed (steady state), then
    one measured round over the whole trace, the modes in turn; latency runs from each
    request's arrival time to its result in host memory (the client's own
    delay before submitting, if any, plus the server's submit-to-completion
    time); p50/p99 over every request of the round.  Then a saturation burst
    per mode: 2000 requests that all arrive at t = 0 (latency from t = 0,
    including the wait for a free client buffer), and shorter rounds at 1600
    and 6400 req/s."""
    import numpy as np
    import threading
    t_arr, shapes = synth.serving_trace(400.0, seconds, 4)
    pool = {}
    sha = hashlib.sha256()
    for (H, W, _) in synth.SERVING_MIX:
        srcs = []
        for k in range(4):
            img = synth.rects_noise(H, W, 70 + k)
            sha.update(img.tobytes())
            t = torch.empty((H, W), dtype=torch.uint8, pin_memory=True)
            t.copy_(torch.from_numpy(img))
            srcs.append(t)
        outs = [torch.empty((H, W), dtype=torch.float32, pin_memory=True) for _ in range(48)]
        pool[(H, W)] = (srcs, outs)

    def run(plain: int, arrivals, shapes_, warm_s: float = 0.0):
        with pkg.Sobel4(0) as s:
            st, srv = pkg.sobel4_server_create(s.handle, 8 << 30, 0, 0, 0, plain)
            assert st == 0
            if warm_s:
                # steady state: the first seconds of the trace through this
                # server, untimed, before the measured round (a fresh server
                # runs slower for its first seconds)
                warm = [(t, hw) for t, hw in zip(arrivals, shapes_) if t < warm_s]
                t0 = time.perf_counter()
                pending = []
                for i, (ta, (H, W)) in enumerate(warm):
                    now = time.perf_counter() - t0
                    if ta > now:
                        time.sleep(ta - now)
                    srcs, outs = pool[(H, W)]
                    rc, t = pkg.sobel4_server_submit(srv, srcs[i % len(srcs)].data_ptr(), W,
                                                     outs[i % len(outs)].data_ptr(), W * 4, H, W)
                    assert rc == 0
                    pending.append(t)
                    if len(pending) >= 32:
                        assert pkg.sobel4_server_wait(srv, pending.pop(0), -1)[0] == 0
                for t in pending:
                    assert pkg.sobel4_server_wait(srv, t, -1)[0] == 0
            tickets = []
            counters = {k: 0 for k in pool}
            free = {k: threading.Semaphore(len(v[1])) for k, v in pool.items()}
            lat = np.empty(len(arrivals))
            srv_lat = np.empty(len(arrivals))
            done = threading.Event()

            def collector():
                for i in range(len(arrivals)):
                    while i >= len(tickets):
                        time.sleep(0.0002)
                    t, key, delay = tickets[i]
                    rc, l = pkg.sobel4_server_wait(srv, t, -1)
                    assert rc == 0
                    lat[i] = delay + l * 1e-6
                    srv_lat[i] = l * 1e-6
                    free[key].release()
                done.set()

            th = threading.Thread(target=collector, daemon=True)
            th.start()
            t0 = time.perf_counter()
            for ta, (H, W) in zip(arrivals, shapes_):
                now = time.perf_counter() - t0
                if ta > now:
                    time.sleep(ta - now)
                key = (H, W)
                free[key].acquire()
                srcs, outs = pool[key]
                c = counters[key]
                counters[key] += 1
                src, out = srcs[c % len(srcs)], outs[c % len(outs)]
                delay = time.perf_counter() - t0 - ta  # arrival -> submit
                rc, t = pkg.sobel4_server_submit(srv, src.data_ptr(), W, out.data_ptr(), W * 4,
                                                 H, W)
                assert rc == 0
                tickets.append((t, key, max(0.0, delay)))
            done.wait()
            span = time.perf_counter() - t0
            stats = pkg.sobel4_server_stats(srv)[1]
            pkg.sobel4_server_destroy(srv)
        px = sum(h * w for h, w in shapes_)
        return {"p50_ms": float(np.percentile(lat, 50)) * 1e3,
                "p99_ms": float(np.percentile(lat, 99)) * 1e3,
                "mean_ms": float(lat.mean()) * 1e3, "max_ms": float(lat.max()) * 1e3,
                "server_p50_ms": float(np.percentile(srv_lat, 50)) * 1e3,
                "server_p99_ms": float(np.percentile(srv_lat, 99)) * 1e3,
                "gpix_s": px / span / 1e9, "requests": len(arrivals),
                "batches": stats["batches"], "max_batch": stats["max_batch_seen"],
                "span_s": span}

    # The client's two Python threads hand the interpreter lock over every
    # 5 ms by default; a late submit would count as server latency.
    switch = sys.getswitchinterval()
    sys.setswitchinterval(1e-4)
    n_burst = min(len(t_arr), 2000)
    burst = np.zeros(n_burst)
    for _, plain in SERVING_MODES:  # warm up: kernel loading, first use of the pinned pools
        run(plain, burst[:200], shapes[:200])
    res = {}
    for name, plain in SERVING_MODES:
        res[name] = run(plain, t_arr, shapes, warm_s=min(5.0, seconds / 4))
    for name, plain in SERVING_MODES:
        res["burst_" + name] = run(plain, burst, shapes[:n_burst])
    # higher request rates (10 s each, after 2 s of warm-up traffic)
    res["rates"] = {}
    for rate in (1600.0, 6400.0):
        ta, sh = synth.serving_trace(rate, 12.0, 5)
        row = {}
        for name, plain in SERVING_MODES:
            r = run(plain, ta, sh, warm_s=2.0)
            row[name] = {k: r[k] for k in ("p50_ms", "p99_ms", "gpix_s", "max_batch")}
        res["rates"][f"{rate:.0f}_req_s"] = row
    sys.setswitchinterval(switch)
    b, p = res["batched"], res["plain_one_stream"]
    return {"workload": f"Poisson 400 req/s for {seconds:.0f} s ({len(t_arr)} requests), "
                        "640x480 40% / 1280x720 30% / 1920x1080 20% / 3840x2160 10%, F32 VALID, "
                        "8 GiB admission budget; results written by the kernels into the client's "
                        "pinned buffers; per mode 5 s of warm-up traffic, then one measured round; "
                        "latency from arrival (server_*: from submit); "
                        f"burst = {n_burst} requests arriving at t = 0; rates: 12 s Poisson traces "
                        "at 1600 and 6400 req/s, their first 2 s served untimed as warm-up, then the "
                        "whole trace measured",
            "inputs_sha256": sha.hexdigest(), **res,
            "batched_beats_plain": {"p99": b["p99_ms"] < p["p99_ms"],
                                    "p50": b["p50_ms"] < p["p50_ms"],
                                    "gpix_s": b["gpix_s"] >= p["gpix_s"]}}


# ----------------------------------------------------------------------------
def cpu_baseline(img, seconds: float):
    """The oracle over bands of the image on all host threads for `seconds`,
    then on one thread for a third of that (both reported)."""
    import numpy as np

    import oracle
    o = oracle.default()
    cores = oracle.cpu_count()
    out = np.empty(img.shape, np.float32)

    def rate(threads: int, budget: float):
        # rows of the same image, whole bands at a time, until `budget` has passed
        rows_done, y, band = 0, 0, 1024 if threads > 1 else 128
        t0 = time.perf_counter()
        while True:
            y1 = min(img.shape[0], y + band)
            o.run_into(img[max(0, y - 2):min(img.shape[0], y1 + 2)],
                       out[max(0, y - 2):min(img.shape[0], y1 + 2)], "valid", "f32",
                       threads=threads)
            rows_done += y1 - y
            y = 0 if y1 >= img.shape[0] else y1
            if time.perf_counter() - t0 >= budget:
                break
        return rows_done, time.perf_counter() - t0

    rows_1, dt_1 = rate(1, seconds / 3)
    rows_done, dt = rate(cores, seconds)
    px = rows_done * img.shape[1]
    return {"value": px / dt / 1e9, "unit": "Gpixel/s", "cores": cores, "kind": "oracle",
            "sample": f"{rows_done} rows of the 8192-wide image (1024-row bands + 2-row halos), "
                      f"{dt:.1f} s on {cores} host threads",
            "one_core": {"value": rows_1 * img.shape[1] / dt_1 / 1e9, "unit": "Gpixel/s",
                         "sample": f"{rows_1} rows (128-row bands), {dt_1:.1f} s on 1 thread"}}


def workload_config(world: int) -> dict:
    """The `config` both arms print (the same dict, so the two lines compare)."""
    return {"workload": WORKLOAD, "height": H, "width": W, "format": "f32", "border": "valid",
            "per_rank_images": 1, "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2: the GPU arm rotates over buffer sets of "
                  "336 MB each (> 2x the 129 MB L2) instead of a flush; the CPU arm "
                  "streams row bands of the image"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    import synth
    img = synth.rects_noise(H, W, 0)
    o = oracle.default()
    cores = oracle.cpu_count()
    import numpy as np
    # size each step's sample so the whole run takes about a minute
    probe = img[:256]
    outp = np.empty(probe.shape, np.float32)
    t0 = time.perf_counter()
    o.run_into(probe, outp, "valid", "f32", threads=cores)
    rate = probe.size / max(time.perf_counter() - t0, 1e-6)
    budget = 60.0
    rows = int(max(8, min(H, budget * rate / max(1, args.steps + args.warmup) / W)))
    out = np.empty((rows, W), np.float32)
    for i in range(args.warmup):
        o.run_into(img[:rows], out, "valid", "f32", threads=cores)
    t0 = time.perf_counter()
    for i in range(args.steps):
        y0 = (i * rows) % max(1, H - rows)
        o.run_into(img[y0:y0 + rows], out, "valid", "f32", threads=cores)
    dt = time.perf_counter() - t0
    px = rows * W * args.steps
    value = px / dt / 1e9
    line = {
        "impl": "reference", "input_sha256": hashlib.sha256(img.tobytes()).hexdigest(),
        "metric": METRIC, "value": value, "unit": "Gpixel/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic",
        "config": workload_config(world),
        "cpu_baseline": {"value": value, "unit": "Gpixel/s", "cores": cores, "kind": "oracle",
                         "sample": f"{rows}x{W} rows of the 8192x8192 image per step"},
        "e2e": {"value": value, "unit": "Gpixel/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2305_00515_gb300 as pkg
    import synth
    from paper_2305_00515_gb300 import build
    build.build()
    dev = local
    torch.cuda.set_device(dev)
    img = synth.rects_noise(H, W, rank)
    px = H * W
    per_set = px * BYTES_PER_PX
    nsets = max(2, -(-2 * L2_BYTES // per_set) + 1)
    srcs = [torch.from_numpy(img).to(f"cuda:{dev}") for _ in range(nsets)]
    outs = [torch.empty((H, W), dtype=torch.float32, device=f"cuda:{dev}") for _ in range(nsets)]
    st, h = pkg.sobel4_create(dev, pkg.VARIANTS[args.variant], args.rows_per_strip)
    assert st == 0, pkg.sobel4_status_string(st)
    # The library's autotuner (untimed) picks the kernel and strip height for
    # this shape, as a serving deployment would once per shape.
    tuned = None
    _, kind0, _, _ = pkg.sobel4_tune_config(h, H, W, 0)
    stem, kernel_name = KERNELS[kind0]
    if not args.no_tune:
        st, _ = pkg.sobel4_tune(h, H, W, 0, 0)
        assert st == 0, pkg.sobel4_status_string(st)
        _, kind, ncl, rps = pkg.sobel4_tune_config(h, H, W, 0)
        stem, kernel_name = KERNELS[kind]
        tuned = {"kernel": KERNELS[kind][0], "columns_per_lane": ncl, "rows_per_strip": rps}
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream

    def launch(i):
        s, o = srcs[i % nsets], outs[i % nsets]
        rc = pkg.sobel4_run(h, s.data_ptr(), W, o.data_ptr(), W * 4, H, W, 0, 0, sh)
        if rc:
            raise RuntimeError(pkg.sobel4_status_string(rc))

    for i in range(args.warmup):
        launch(i)
    stream.synchronize()
    # correctness spot check of the timed configuration: a few rows against the oracle
    if rank == 0:
        import oracle
        got = outs[(args.warmup - 1) % nsets][4000:4016].cpu().numpy() if args.warmup else None
        if got is not None:
            want = oracle.default().sobel4(img[3998:4018], "valid", "f32")[2:18]
            assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), \
                "bench output differs from the oracle"

    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    n0 = pkg.sobel4_launch_count(h)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize(dev)
    # The timed region: K back-to-back launches (each launch's prologue may
    # overlap the end of the one before: programmatic dependent launch).
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for i in range(args.steps):
            launch(args.warmup + i)
        t_end.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    launches = pkg.sobel4_launch_count(h) - n0
    clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    # Untimed for `value`: the same launches with an event pair around each
    # (the events keep the launches from overlapping), for the per-launch spread.
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            ev[i][0].record(stream)
            launch(args.warmup + args.steps + i)
            ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(total_ms, world)
    value = weak_scaling_value(px, args.steps, world, total_ms)
    # the kernel's average launch duration over the timed region
    mean_kernel_s = total_ms * 1e-3 / args.steps
    peak, peak_kind = measured_peaks()
    achieved = px * BYTES_PER_PX / mean_kernel_s / 1e9
    traffic = recorded_traffic(stem)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        h_src = torch.from_numpy(img).pin_memory()
        h_dst = torch.empty((H, W), dtype=torch.float32).pin_memory()
        for _ in range(2):
            pkg.sobel4_run_host(h, h_src.data_ptr(), W, h_dst.data_ptr(), W * 4, H, W, 0, 0)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            rc = pkg.sobel4_run_host(h, h_src.data_ptr(), W, h_dst.data_ptr(), W * 4, H, W, 0, 0)
            assert rc == 0
        dt = max_over_ranks(time.perf_counter() - t0, world)
        barrier(world)
        e2e = {"value": world * px * args.e2e_steps / dt / 1e9, "unit": "Gpixel/s",
               "h2d_bytes_per_step": px, "d2h_bytes_per_step": px * 4,
               "ms_per_step": dt * 1e3 / args.e2e_steps, "steps": args.e2e_steps}
    pkg.sobel4_destroy(h)

    extras = {}
    if world == 1 and not args.no_extras:
        del srcs, outs
        torch.cuda.empty_cache()
        # The host-link legs first: they allocate their page-locked rings and
        # pools as a streaming application does at start-up.  Run after the
        # legs that allocate and free gigabytes, the same video loop measured
        # 4035-4071 instead of 5100 frames/s (the pinned buffers then reach the
        # GPU less efficiently).
        extras["video"] = bench_video(torch, pkg, synth, args.video_frames)
        extras["serving"] = bench_serving(torch, pkg, synth, args.serve_seconds)
        torch.cuda.empty_cache()
        extras["sweep"] = bench_sweep(torch, pkg, synth, peak)
        extras["rgb"] = bench_rgb(torch, pkg, synth, peak)
        extras["runtime_weights"] = bench_runtime_weights(torch, pkg, synth, peak,
                                                          mean_kernel_s * 1e6)
        extras["batched"] = bench_batched(torch, pkg, synth)
        extras["ablation_us"] = bench_ablation(torch, pkg, synth)

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(img, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": "Gpixel/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8->int32->f32", "data": "synthetic",
        "config": workload_config(world),
        "input_sha256": hashlib.sha256(img.tobytes()).hexdigest(),
        "autotuned": tuned,
        "l2_buffer_sets": nsets,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kernel_name, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": px * BYTES_PER_PX,
                     "mean_kernel_us": mean_kernel_s * 1e6,
                     "timing": "timed region / launches (back-to-back launches)",
                     "event_per_launch_us": {"mean": statistics.fmean(kern_ms) * 1e3,
                                             "p50": statistics.median(kern_ms) * 1e3}},
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clocks.summary(),
        "gpu_launches": int(launches),
        **extras,
    }
    print(json.dumps(line), flush=True)


PROFILE_VARIANTS = ("direct", "ladder_sm", "ladder_sm_p", "ladder_rg", "ladder_rg_v1",
                    "ladder_rg_v2", "rg_lanecopy", "rg", "tc")


def profile_variants():
    """Each kernel variant (GM, the paper's ladder, the GB300 kernels) launched
    twice on the 8192x8192 rects+noise image, F32 VALID, default options."""
    import torch

    import paper_2305_00515_gb300 as pkg
    import synth
    img = synth.rects_noise(H, W, 0)
    src = torch.from_numpy(img).cuda()
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    for v in PROFILE_VARIANTS:
        st, h = pkg.sobel4_create(0, pkg.VARIANTS[v])
        assert st == 0, pkg.sobel4_status_string(st)
        for _ in range(2):
            rc = pkg.sobel4_run(h, src.data_ptr(), W, out.data_ptr(), 4 * W, H, W, 0, 0,
                                stream.cuda_stream)
            assert rc == 0, pkg.sobel4_status_string(rc)
        stream.synchronize()
        assert pkg.sobel4_device_status(h) == 0
        pkg.sobel4_destroy(h)
        print(f"{v}: ok", flush=True)


def profile_batch(n: int):
    """The first n images of the 512-image ragged batch (sides U{37..2048},
    seed 1, tight pitches), F32 VALID, through sobel4_run_batched twice with
    the handle's default configuration."""
    import torch

    import paper_2305_00515_gb300 as pkg
    import synth
    imgs = synth.batch_images(512, 1)[:n]
    srcs = [torch.from_numpy(i).cuda() for i in imgs]
    outs = [torch.empty(i.shape, dtype=torch.float32, device="cuda") for i in imgs]
    descs = (pkg.Image * len(imgs))(*[pkg.Image(s.data_ptr(), s.stride(0), o.data_ptr(),
                                                 o.stride(0) * 4, *s.shape)
                                      for s, o in zip(srcs, outs)])
    st, h = pkg.sobel4_create(0)
    assert st == 0, pkg.sobel4_status_string(st)
    stream = torch.cuda.Stream()
    for _ in range(2):
        rc = pkg.sobel4_run_batched(h, descs, 0, 0, stream.cuda_stream)
        assert rc == 0, pkg.sobel4_status_string(rc)
    stream.synchronize()
    assert pkg.sobel4_device_status(h) == 0
    pkg.sobel4_destroy(h)
    print(f"batch of {n}: ok ({sum(i.size for i in imgs)} pixels)", flush=True)


def profile_single(kind: str):
    """One image launched twice: 8192x8192 through the fused colour input
    ("rgb": interleaved RGB rects+noise, F32 VALID) or the runtime-weight path
    ("weights": Eq. (5) weights (a, b, n, m) = (2, 1.5, 2, 2), F32 VALID), or
    the size sweep's 1920x1080 rects+noise image at source pitch 1937 and
    output pitch 7748 ("pitch", F32 VALID)."""
    import numpy as np
    import torch

    import paper_2305_00515_gb300 as pkg
    import synth
    st, h = pkg.sobel4_create(0)
    assert st == 0, pkg.sobel4_status_string(st)
    stream = torch.cuda.Stream()
    if kind == "pitch":
        # the size sweep's pitch variant: 1920x1080, source pitch 1937, output pitch 7748
        h1, w1, sp, dp = 1080, 1920, 1937, 7748
        src = torch.zeros(h1 * sp, dtype=torch.uint8, device="cuda")
        src.view(h1, sp)[:, :w1] = torch.from_numpy(synth.rects_noise(h1, w1, 0)).cuda()
        out = torch.empty(h1 * dp, dtype=torch.uint8, device="cuda")
        for _ in range(2):
            rc = pkg.sobel4_run(h, src.data_ptr(), sp, out.data_ptr(), dp, h1, w1, 0, 0,
                                stream.cuda_stream)
            assert rc == 0, pkg.sobel4_status_string(rc)
        stream.synchronize()
        assert pkg.sobel4_device_status(h) == 0
        pkg.sobel4_destroy(h)
        print(f"{kind}: ok", flush=True)
        return
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    if kind == "rgb":
        src = torch.from_numpy(np.stack([synth.rects_noise(H, W, 50 + c) for c in range(3)],
                                        axis=2)).cuda()
        run, pitch = pkg.sobel4_run_rgb, 3 * W
    else:
        assert pkg.sobel4_set_weights(h, 2, 1.5, 2, 2) == 0
        src = torch.from_numpy(synth.rects_noise(H, W, 0)).cuda()
        run, pitch = pkg.sobel4_run, W
    for _ in range(2):
        rc = run(h, src.data_ptr(), pitch, out.data_ptr(), 4 * W, H, W, 0, 0, stream.cuda_stream)
        assert rc == 0, pkg.sobel4_status_string(rc)
    stream.synchronize()
    assert pkg.sobel4_device_status(h) == 0
    pkg.sobel4_destroy(h)
    print(f"{kind}: ok", flush=True)


def main():
    args = parse_args()
    if args.profile_variants:
        profile_variants()
        return
    if args.profile_single:
        profile_single(args.profile_single)
        return
    if args.profile_batch:
        profile_batch(args.profile_batch)
        return
    if args.impl == "reference":
        # the CPU oracle runs on rank 0 alone; other ranks exit without work
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_setup(args.gpus)
    run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
