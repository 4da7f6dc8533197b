"""The continuous-batching server: every request's result equals the oracle
and its own standalone sobel4_run, whether it ran in a batch with others, as
its own launch, or in the one-stream plain mode, and whether the kernel wrote
it into pinned host memory or it was staged and downloaded; admission respects the
device-memory budget; the batched mode really packs concurrent requests into
shared launches (a large first request keeps the GPU busy while the others
arrive, so they meet in the next batch)."""
import threading

import numpy as np
import pytest

import oracle
import paper_2305_00515_gb300 as pkg
import synth
from gpu_util import same_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def pinned(shape, dtype):
    t = torch.empty(int(np.prod(shape)) * np.dtype(dtype).itemsize, dtype=torch.uint8,
                    pin_memory=True)
    return t, t.numpy().view(dtype).reshape(shape)


def make_requests(n, seed, fmt, first=None):
    """Pinned inputs; every third result buffer is pageable (numpy) memory,
    which the server stages in its arena and downloads, the others pinned,
    which the kernel writes itself."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        H, W = (int(v) for v in rng.integers(5, 400, size=2))
        if i == 0 and first:
            H, W = first
        _, src = pinned((H, W), np.uint8)
        src[:] = synth.rects_noise(H, W, seed * 100 + i)
        dt = {"f32": np.float32, "u8": np.uint8, "s16x4": np.int16}[fmt]
        shape = (4, H, W) if fmt == "s16x4" else (H, W)
        if i % 3 == 2:
            keep, dst = None, np.full(shape, 7, dt)
        else:
            keep, dst = pinned(shape, dt)
        reqs.append((src, dst, keep))
    return reqs


def run_server(reqs, fmt, border, plain, budget=0, threads=1):
    with pkg.Sobel4(0) as s:
        st, srv = pkg.sobel4_server_create(s.handle, budget, 0, pkg.BORDERS[border],
                                           pkg.FORMATS[fmt], plain)
        assert st == 0
        tickets = [None] * len(reqs)

        def submit(idx):
            for i in idx:
                src, dst, _ = reqs[i]
                rc, t = pkg.sobel4_server_submit(srv, src.ctypes.data, src.strides[0],
                                                 dst.ctypes.data, dst.strides[-2], *src.shape)
                assert rc == 0
                tickets[i] = t

        parts = [list(range(k, len(reqs), threads)) for k in range(threads)]
        ths = [threading.Thread(target=submit, args=(p,)) for p in parts]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        lats = []
        for t in tickets:
            rc, lat = pkg.sobel4_server_wait(srv, t, -1)
            assert rc == 0
            lats.append(lat)
        rc, stats = pkg.sobel4_server_stats(srv)
        assert rc == 0
        assert pkg.sobel4_server_destroy(srv) == 0
        stats["launches"] = s.launches
    return lats, stats


def run_alone(img, border, fmt):
    """The request's image through its own sobel4_run (no server, no batch)."""
    with pkg.Sobel4(0) as s:
        out = s.run(torch.from_numpy(np.ascontiguousarray(img)).cuda(), border=border, fmt=fmt)
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("plain", [0, 1, 2])
@pytest.mark.parametrize("fmt,border", [("f32", "valid"), ("u8", "reflect101"),
                                        ("s16x4", "constant0")])
def test_server_results_match_oracle_alone_and_in_the_mix(plain, fmt, border):
    # request 0 is a 3840x2160 frame: while it is on the GPU the others arrive
    reqs = make_requests(24, 3 + plain, fmt, first=(2160, 3840))
    lats, stats = run_server(reqs, fmt, border, plain, threads=1)
    assert stats["submitted"] == stats["completed"] == len(reqs)
    assert all(l > 0 for l in lats)
    assert 1 <= stats["batches"] <= len(reqs)
    if plain == 0:
        # batches of four or more take one batched launch (plus its descriptor upload)
        assert stats["max_batch_seen"] >= 4, "no four requests ever met in a batch"
        assert stats["launches"] < len(reqs), "no two requests ever shared a launch"
    else:
        assert stats["launches"] >= len(reqs)  # a sobel4_run (one or more kernels) per request
        if plain == 2:
            assert stats["max_batch_seen"] == 1  # one request per step on the one stream
    assert stats["device_bytes_in_use"] == 0
    for src, dst, _ in reqs:
        assert same_bits(dst, oracle.sobel4(src, border, fmt))
        assert same_bits(dst, run_alone(src, border, fmt))


def test_server_admission_under_small_budget():
    reqs = make_requests(16, 9, "f32")
    budget = 1 << 20  # ~1 MiB: only a few requests fit at once
    lats, stats = run_server(reqs, "f32", "replicate", 0, budget=budget)
    assert stats["completed"] == len(reqs)
    assert stats["device_bytes_peak"] <= budget
    for src, dst, _ in reqs:
        assert same_bits(dst, oracle.sobel4(src, "replicate", "f32"))


def test_server_rejects_and_times_out():
    with pkg.Sobel4(0) as s:
        st, srv = pkg.sobel4_server_create(s.handle, 1 << 16, 0, 0, 0, 0)
        assert st == 0
        _, big = pinned((1000, 1000), np.uint8)
        _, out = pinned((1000, 1000), np.float32)
        rc, _ = pkg.sobel4_server_submit(srv, big.ctypes.data, 1000, out.ctypes.data, 4000,
                                         1000, 1000)
        assert rc == 2  # can never fit the budget
        assert pkg.sobel4_server_wait(srv, 12345, 0)[0] == 1  # unknown ticket
        _, small = pinned((60, 70), np.uint8)
        small[:] = synth.uniform(60, 70, 1)
        _, o2 = pinned((60, 70), np.float32)
        rc, t = pkg.sobel4_server_submit(srv, small.ctypes.data, 70, o2.ctypes.data, 280, 60, 70)
        assert rc == 0
        rc, _ = pkg.sobel4_server_wait(srv, t, 0)
        if rc == 5:  # still pending: the ticket stays valid
            rc, _ = pkg.sobel4_server_wait(srv, t, -1)
        assert rc == 0
        assert same_bits(o2, oracle.sobel4(small))
        assert pkg.sobel4_server_destroy(srv) == 0


def test_allocation_failures_surface_as_oom():
    """Failure injection on the host: allocations no GPU can satisfy."""
    with pkg.Sobel4(0) as s:
        st, srv = pkg.sobel4_server_create(s.handle, 1 << 52, 0, 0, 0, 0)
        assert st == 3 and not srv.value
        st, _ = pkg.sobel4_tune(s.handle, 1 << 26, 1 << 26, 0, 0)
        assert st == 3
        assert s.launches == 0
        # the handle still works afterwards
        img = synth.uniform(40, 50, 3)
        out = s.run(torch.from_numpy(img).cuda())
        torch.cuda.synchronize()
        assert same_bits(out.cpu().numpy(), oracle.sobel4(img))
