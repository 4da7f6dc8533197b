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
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the Poisson serving run (the full configuration is 60)")
    ap.add_argument("--profile-batch", type=int, default=0, metavar="N",
                    help="run the first N images of the 512-image ragged batch (seed 1) through "
                         "sobel4_run_batched twice and exit (a capture target for ncu)")
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

    def batched():
        assert pkg.sobel4_run_batched(h, descs, 0, 0, sh) == 0

    def singles():
        for s_, o in zip(srcs, outs_s):
            assert pkg.sobel4_run(h, s_.data_ptr(), s_.stride(0), o.data_ptr(), o.stride(0) * 4,
                                  s_.shape[0], s_.shape[1], 0, 0, sh) == 0

    res = {}
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
        res[name] = {"ms_median": ms[len(ms) // 2], "gpix_s": px / (ms[len(ms) // 2] * 1e-3) / 1e9}
    torch.cuda.synchronize()
    same = all(torch.equal(a, b) for a, b in zip(outs_b, outs_s))
    import oracle
    for k in (0, 100, 511):
        assert np.array_equal(outs_b[k].cpu().numpy().view(np.uint32),
                              oracle.default().sobel4(imgs[k], "valid", "f32",
                                                      threads=8).view(np.uint32))
    pkg.sobel4_destroy(h)
    return {"workload": "512 ragged uint8 images, sides U{37..2048} (seed 1), F32, VALID",
            "pixels": px, **res, "speedup": res["separate_launches"]["ms_median"] /
            res["one_persistent_launch"]["ms_median"], "tuned_us": tuned,
            "batch_equals_single_runs": bool(same)}


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


def bench_video(torch, pkg, synth, frames: int, slots: int = 4):
    """3840x2160 frames through the graph-captured pipeline (H2D + kernel + D2H
    per frame, `slots` frame slots); the slot buffers hold pre-generated frames
    (frame k uses the frame of slot k mod slots)."""
    import numpy as np
    H, W = 2160, 3840
    bg = synth.video_background(H, W, 3)
    with pkg.Sobel4(0) as s:
        pipe = pkg.Pipeline(s, H, W, "valid", "f32", slots=slots)
        ring = [synth.video_frame(bg, k, H, W, 3) for k in range(slots)]
        for k in range(slots):
            pipe.inputs[k][:] = ring[k]
        for k in range(slots):  # warm up
            pipe.submit(k)
        for k in range(slots):
            pipe.wait(k)
        t0 = time.perf_counter()
        for k in range(frames):
            slot = k % slots
            pipe.wait(slot)
            pipe.submit(slot)
        for k in range(slots):
            pipe.wait(k)
        dt = time.perf_counter() - t0
        import oracle
        last = (frames - 1) % slots
        ok = np.array_equal(np.ascontiguousarray(pipe.outputs[last]).view(np.uint32),
                            oracle.default().sobel4(ring[last], "valid", "f32",
                                                    threads=8).view(np.uint32))
        pipe.close()
    fps = frames / dt
    bytes_per_frame = H * W * 5
    return {"workload": f"{frames} frames of 3840x2160 u8 -> f32 through {slots} graph slots",
            "frames_per_s": fps, "ms_per_frame": 1e3 / fps, "gpix_s": fps * H * W / 1e9,
            "host_link_gb_s": fps * bytes_per_frame / 1e9, "last_frame_matches_oracle": bool(ok)}


def bench_serving(torch, pkg, synth, seconds: float):
    """Poisson arrivals (400 req/s) of the serving resolution mix through the
    continuous-batching server, batched and plain (one launch per request);
    p50/p99 latency from submit to result in host memory; then a saturation
    burst (every request submitted at once) for throughput."""
    import numpy as np
    import threading
    t_arr, shapes = synth.serving_trace(400.0, seconds, 4)
    pool = {}
    for (H, W, _) in synth.SERVING_MIX:
        srcs = []
        for k in range(4):
            t = torch.empty((H, W), dtype=torch.uint8, pin_memory=True)
            t.copy_(torch.from_numpy(synth.rects_noise(H, W, 70 + k)))
            srcs.append(t)
        outs = [torch.empty((H, W), dtype=torch.float32, pin_memory=True) for _ in range(48)]
        pool[(H, W)] = (srcs, outs)

    def run(plain: int, arrivals):
        with pkg.Sobel4(0) as s:
            st, srv = pkg.sobel4_server_create(s.handle, 8 << 30, 0, 0, 0, plain)
            assert st == 0
            tickets = []
            counters = {k: 0 for k in pool}
            free = {k: threading.Semaphore(len(v[1])) for k, v in pool.items()}
            lat = []
            done = threading.Event()

            def collector():
                i = 0
                while i < len(arrivals):
                    while i >= len(tickets):
                        time.sleep(0.0002)
                    t, key = tickets[i]
                    rc, l = pkg.sobel4_server_wait(srv, t, -1)
                    assert rc == 0
                    lat.append(l)
                    free[key].release()
                    i += 1
                done.set()

            th = threading.Thread(target=collector, daemon=True)
            th.start()
            t0 = time.perf_counter()
            for ta, (H, W) in zip(arrivals, shapes):
                now = time.perf_counter() - t0
                if ta > now:
                    time.sleep(ta - now)
                key = (H, W)
                free[key].acquire()
                srcs, outs = pool[key]
                c = counters[key]
                counters[key] += 1
                src, out = srcs[c % len(srcs)], outs[c % len(outs)]
                rc, t = pkg.sobel4_server_submit(srv, src.data_ptr(), W, out.data_ptr(), W * 4,
                                                 H, W)
                assert rc == 0
                tickets.append((t, key))
            done.wait()
            span = time.perf_counter() - t0
            stats = pkg.sobel4_server_stats(srv)[1]
            pkg.sobel4_server_destroy(srv)
        px = sum(h * w for h, w in shapes[:len(arrivals)])
        lat = np.array(lat)
        return {"p50_ms": float(np.percentile(lat, 50)) / 1e3,
                "p99_ms": float(np.percentile(lat, 99)) / 1e3,
                "mean_ms": float(lat.mean()) / 1e3, "gpix_s": px / span / 1e9,
                "requests": len(arrivals), "batches": stats["batches"],
                "max_batch": stats["max_batch_seen"], "span_s": span}

    res = {}
    # One short unrecorded burst per mode first (kernel loading, first use of
    # the pinned pools).  Then the Poisson trace twice per mode, alternating
    # the modes; each mode reports its round with the lower p99 (on one box
    # the same mode's p99 moved by 3x between rounds: the 3840x2160 frames'
    # host-link copies dominate the tail and their speed drifts).
    burst = np.zeros(min(len(t_arr), 2000))
    for plain in (1, 0):
        run(plain, burst[:200])
    poisson = {"batched": [], "plain_launch_per_request": []}
    for _ in range(2):
        for name, plain in (("plain_launch_per_request", 1), ("batched", 0)):
            poisson[name].append(run(plain, t_arr))
    for name, rs in poisson.items():
        res[name] = min(rs, key=lambda r: r["p99_ms"])
        res[name]["p99_rounds_ms"] = [r["p99_ms"] for r in rs]
    # Saturation bursts: two rounds alternating the modes; each mode reports
    # its faster round (a single burst's span moved by up to 2x with what ran
    # before it in the process).
    rounds = {"burst_batched": [], "burst_plain": []}
    for _ in range(2):
        for name, plain in (("burst_plain", 1), ("burst_batched", 0)):
            rounds[name].append(run(plain, burst))
    for name, rs in rounds.items():
        res[name] = min(rs, key=lambda r: r["span_s"])
        res[name]["spans_s"] = [r["span_s"] for r in rs]
    return {"workload": f"Poisson 400 req/s for {seconds:.0f} s ({len(t_arr)} requests), "
                        "640x480 40% / 1280x720 30% / 1920x1080 20% / 3840x2160 10%, F32, "
                        "8 GiB admission budget, after a warm-up burst; each mode's round "
                        "with the lower p99 of two alternating rounds; burst = 2000 "
                        "requests at t=0 (faster of two alternating rounds)", **res}


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
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gpixel/s",
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
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            launch(args.warmup + i)
            ev[i][1].record(stream)
        t_end.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    launches = pkg.sobel4_launch_count(h) - n0
    clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(total_ms, world)
    value = weak_scaling_value(px, args.steps, world, total_ms)
    mean_kernel_s = statistics.fmean(kern_ms) * 1e-3
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
        extras["batched"] = bench_batched(torch, pkg, synth)
        extras["ablation_us"] = bench_ablation(torch, pkg, synth)
        torch.cuda.empty_cache()
        extras["video"] = bench_video(torch, pkg, synth, args.video_frames)
        extras["serving"] = bench_serving(torch, pkg, synth, args.serve_seconds)

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
        "autotuned": tuned,
        "l2_buffer_sets": nsets,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kernel_name, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": px * BYTES_PER_PX,
                     "mean_kernel_us": mean_kernel_s * 1e6,
                     "p50_kernel_us": statistics.median(kern_ms) * 1e3},
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


def main():
    args = parse_args()
    if args.profile_variants:
        profile_variants()
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
