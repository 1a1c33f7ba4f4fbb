"""Benchmark: GLCM throughput (Gpairs/s) and HBM-read roofline on GB300.

Default workload (the contention sweep): 12 distinct 4096 x 4096 uint8
images -- iid, smooth (sigma 8 px) and constant-128, each at N = 8, 16, 32
and 256 levels -- with the 4 offsets at d = 1 (0/45/90/135 degrees).  One
step is one pass of the whole path over the batch: quantize, partner
lookup and vote of every pair, merge, symmetrize + normalize, and the 14
Haralick features, replayed from one CUDA graph (the N = 256 images vote
first and their epilogue overlaps the other images' votes).  The batch
(201 MB) is larger than the 129 MB L2, so no flush is needed between steps.
Before timing, the vote configuration of each (levels, offsets) class is
autotuned on this batch (cached per GPU under the package's _build/).

Printed (one JSON line, rank 0): value = pairs per second over all ranks
with inputs resident in HBM; e2e = the same through the C ABI with pinned
host buffers (host->device image copies and device->host results inside the
timed region); plain = one image at a time with a sync per image; roofline
of the vote kernels from CUDA events on their stream; ceilings = measured
shared-reduction and HBM-read rates (glcm_measure_ceilings); classes = each
kind and N of the sweep as one image per launch (the vote kernel's own
roofline line per class); serving = the served stream (continuous batching
vs a one-at-a-time loop, p50/p99 latency); parity = the timed batch's own
counts, normalized GLCMs and features against the CPU oracle (a mismatch
makes the run fail); cpu_baseline = the CPU oracle on a bounded sample.
``--impl reference`` times the oracle alone.
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

METRIC = "GLCM Gpairs/s & HBM-roofline %, batched vs plain launch (bit-exact); p99 latency"
UNIT = "Gpairs/s"
WORKLOAD = ("contention sweep: 12 x 4096^2 uint8 images (iid, smooth sigma=8, constant 128) x N in "
            "{8,16,32,256}, offsets d=1 at 0/45/90/135 deg, plain uint32 counts + symmetric normalized GLCMs "
            "+ 14 Haralick features, one batched graph launch per step")


def workload_config():
    """The workload both arms measure (the same dict in both JSON lines)."""
    return {"workload": WORKLOAD, "images": 12, "side": 4096, "levels": [8, 16, 32, 256],
            "kinds": ["iid", "smooth", "constant"], "offsets": [[1, 0], [1, -1], [0, -1], [-1, -1]],
            "pairs_per_step": 12 * 67084290, "image_bytes_per_step": 12 * 4096 * 4096,
            "l2": "inputs 201 MB > 129 MB L2 per step, no flush"}


def rank_helpers(dist):
    """(barrier, max_over_ranks) for the ranks of a gloo process group (host
    tensors only: no data-path collective), or no-ops when dist is None."""
    import torch

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    return barrier, max_over_ranks


def whole_job_value(world: int, pairs_per_rank_step: float, steps: int, seconds: float) -> float:
    """Gpairs/s of all ranks together: every rank processes the same batch
    (weak scaling) and the slowest rank's time counts."""
    return world * pairs_per_rank_step * steps / seconds / 1e9


def pairs_of(w, h, offsets):
    return sum(max(0, w - abs(dx)) * max(0, h - abs(dy)) for dx, dy in offsets)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# The vote kernels' sources (the column walk and the general kernel).
VOTE_SOURCES = ("vote.cu", "vote_fast.cuh", "vote_fast.cu", "vote_fast_unaligned.cu")


def vote_code_sha256() -> str:
    """code_sha256 of the vote kernels' sources, concatenated in VOTE_SOURCES order."""
    csrc = os.path.join(ROOT, "paper_1710_06189_gb300", "csrc")
    return code_sha256("\n".join(open(os.path.join(csrc, f)).read() for f in VOTE_SOURCES))


def profiled_traffic(name: str):
    """DRAM bytes of a step's vote launches from the committed ncu summary,
    valid only while the vote kernels' code is unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_step:\s*([0-9.eE+]+)", text)
    s = re.search(r"vote_code_sha256:\s*([0-9a-f]{64})", text)
    if not m or not s:
        return None
    return float(m.group(1)) if vote_code_sha256() == s.group(1) else None


def code_sha256(text: str) -> str:
    """SHA-256 of a source file's code: each line without its // comment and
    surrounding blanks, empty lines dropped (a comment edit keeps the hash)."""
    lines = []
    for ln in text.splitlines():
        i = ln.find("//")
        ln = (ln[:i] if i >= 0 else ln).strip()
        if ln:
            lines.append(ln)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


class ClockSampler:
    """nvidia-smi clock / throttle sampling (every 50 ms) over a loaded window.

    The window is the timed region plus LOAD_SECONDS of the same step before and
    after it, so that a timed region shorter than the sampling period still has
    samples taken under its load; `mark` brackets the timed region itself and
    `samples_timed` counts the samples that arrived inside it."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t_start = self.t_end = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, start: bool):
        if start:
            self.t_start = time.perf_counter()
        else:
            self.t_end = time.perf_counter()

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons, timed = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            if self.t_start is not None and self.t_end is not None and self.t_start <= t <= self.t_end:
                timed += 1
            for k, nm in enumerate(names):
                if parts[3 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "samples_timed": timed,
                "window": f"timed region plus {LOAD_SECONDS:g} s of the same step before and after"}


LOAD_SECONDS = 0.5


def keep_loaded(step, seconds: float):
    """Run `step` untimed for about `seconds` of wall time, synchronizing every
    32 steps so the host never runs far ahead of the device."""
    import torch

    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        step()
        n += 1
        if n % 32 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()


def oracle_sample(jobs, seconds: float):
    """Time the CPU oracle (counts + symmetric normalize + features) on whole
    images of the workload until `seconds` of work; returns (Gpairs/s, desc)."""
    import oracle
    oracle.build()
    done_pairs, t0, k = 0, time.perf_counter(), 0
    while True:
        j = jobs[k % len(jobs)]
        img = j["image"]
        P = oracle.glcm(img, j["levels"], j["offsets"])
        oracle.haralick_batch(P, True)
        done_pairs += pairs_of(img.shape[1], img.shape[0], j["offsets"])
        k += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return done_pairs / el / 1e9, f"{k} whole 4096^2 images of the sweep (counts + features), {el:.1f} s, 1 thread"


def oracle_sample_all_cores(jobs, seconds: float):
    """The same oracle on every host core: one thread per core, each taking whole
    images of the workload in turn until `seconds` have passed (the oracle's C
    counting loop runs outside the GIL); returns (Gpairs/s, threads, desc)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    oracle.build()
    threads = max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))
    t0 = time.perf_counter()
    stop = t0 + seconds

    def worker(w):
        done, n, k = 0, 0, w
        while time.perf_counter() < stop:
            j = jobs[k % len(jobs)]
            img = j["image"]
            P = oracle.glcm(img, j["levels"], j["offsets"])
            oracle.haralick_batch(P, True)
            done += pairs_of(img.shape[1], img.shape[0], j["offsets"])
            n += 1
            k += threads
        return done, n

    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(worker, range(threads)))
    el = time.perf_counter() - t0
    pairs = sum(r[0] for r in res)
    images = sum(r[1] for r in res)
    return pairs / el / 1e9, threads, f"{images} whole 4096^2 images of the sweep on {threads} threads, {el:.1f} s"


def run_reference(args):
    import numpy as np  # noqa: F401

    import glcm_synth as S
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    jobs = S.contention_jobs(4096)
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(jobs, min(per_step, 5.0))
    vals = []
    t0 = time.perf_counter()
    descs = []
    for _ in range(args.steps):
        v, d = oracle_sample(jobs, per_step)
        vals.append(v)
        descs.append(d)
    el = time.perf_counter() - t0
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "each step: whole images of the sweep for ~%.0f s; last: %s" % (per_step, descs[-1])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


SERVE_REQUESTS = 256
SERVE_LOADS = (0.5, 0.9, 1.5)


def _pace(target: float):
    """Sleep, then spin, until perf_counter() reaches target."""
    while True:
        d = target - time.perf_counter()
        if d <= 0:
            return
        if d > 0.0005:
            time.sleep(d - 0.0003)


def serving_leg(G, S, torch, local: int, n_req: int = SERVE_REQUESTS):
    """Served stream: Poisson requests (seeded) of uint8 images, sides
    log-uniform 256..8192, N in {8,16,32,64}, 1..12 offsets, iid/smooth 50/50,
    from pinned host memory; counts + symmetric features back to pinned host
    buffers.  The plain loop runs one request at a time through the public API
    (copy in, launch, copy out, sync); the server batches continuously.  Both
    see the same arrival times at loads of 0.5, 0.9 and 1.5 x the plain loop's
    capacity, plus an all-at-once burst for saturation throughput.  Latency is
    from a request's scheduled arrival to its results being in host memory."""
    import numpy as np

    reqs = S.request_stream(n_req, 1.0, lo=256, hi=8192)
    crops = S.request_crops(reqs)
    bases = {k: torch.from_numpy(S.image(k, S.serve_base_seed(k), S.SERVE_BASE_SIDE, S.SERVE_BASE_SIDE,
                                         np.uint8, 8.0)).pin_memory() for k in ("iid", "smooth")}
    views = [bases[r.kind][y0:y0 + r.side, x0:x0 + r.side] for r, (y0, x0) in zip(reqs, crops)]
    outs = [(torch.empty((len(r.offsets), r.levels, r.levels), dtype=torch.int32).pin_memory(),
             torch.empty((len(r.offsets), 14), dtype=torch.float32).pin_memory()) for r in reqs]
    pairs = [pairs_of(r.side, r.side, r.offsets) for r in reqs]
    total_pairs = float(sum(pairs))
    unit_arrivals = [r.arrival_s for r in reqs]  # a rate-1 Poisson process
    sym = G.GLCM_SYMMETRIC

    ctx = G.Context(local, hbm_budget_bytes=2 << 30)

    def plain_one(i):
        r = reqs[i]
        ctx.batch([dict(image=views[i], levels=r.levels, offsets=r.offsets, flags=sym, counts=outs[i][0],
                        features=outs[i][1])])

    for i in range(4):
        plain_one(i)
    t0 = time.perf_counter()
    for i in range(n_req):
        plain_one(i)
    plain_s = time.perf_counter() - t0
    capacity = n_req / plain_s

    def plain_run(arr):
        lat = []
        t0 = time.perf_counter()
        for i in range(n_req):
            _pace(t0 + arr[i])
            plain_one(i)
            lat.append(time.perf_counter() - t0 - arr[i])
        return lat, time.perf_counter() - t0

    srv = G.Server(local, hbm_budget_bytes=8 << 30, lanes=2)

    def served_run(arr):
        tickets = [None] * n_req
        lag = [0.0] * n_req
        ready = threading.Semaphore(0)

        def producer():
            t0 = start[0]
            for i in range(n_req):
                r = reqs[i]
                _pace(t0 + arr[i])
                tickets[i] = srv.submit(views[i], r.levels, r.offsets, sym, counts=outs[i][0], features=outs[i][1])
                lag[i] = time.perf_counter() - t0 - arr[i]
                ready.release()

        start = [time.perf_counter()]
        th = threading.Thread(target=producer)
        th.start()
        lat = []
        for i in range(n_req):
            ready.acquire()
            st, ms, _ = srv.wait(tickets[i])
            if st != G.GLCM_OK:
                raise RuntimeError(f"served request {i} failed ({st}): {srv.last_error()}")
            lat.append(lag[i] + ms * 1e-3)
        th.join()
        return lat, time.perf_counter() - start[0]

    served_run([0.0] * n_req)  # warm-up burst

    def pct(v, q):
        return float(np.percentile(np.asarray(v) * 1e3, q))

    out = {"requests": n_req, "mean_image_bytes": float(np.mean([r.side * r.side for r in reqs])),
           "pairs": total_pairs, "plain_capacity_rps": capacity,
           "plain_gpairs_s": total_pairs / plain_s / 1e9, "loads": []}
    # Saturation: the median of three all-at-once bursts (one burst is ~25 ms of
    # wall clock, so a single one is noisy).
    bursts = sorted(served_run([0.0] * n_req)[1] for _ in range(3))
    el = bursts[1]
    out["served_burst_gpairs_s"] = total_pairs / el / 1e9
    out["served_burst_runs_gpairs_s"] = [total_pairs / b / 1e9 for b in bursts]
    out["served_over_plain"] = out["served_burst_gpairs_s"] / out["plain_gpairs_s"]
    for load in SERVE_LOADS:
        arr = [a / (load * capacity) for a in unit_arrivals]
        lp, elp = plain_run(arr)
        ls, els = served_run(arr)
        out["loads"].append({"load_x_plain_capacity": load, "rate_rps": load * capacity,
                             "served": {"gpairs_s": total_pairs / els / 1e9, "p50_ms": pct(ls, 50),
                                        "p99_ms": pct(ls, 99)},
                             "plain": {"gpairs_s": total_pairs / elp / 1e9, "p50_ms": pct(lp, 50),
                                       "p99_ms": pct(lp, 99)}})
    st = srv.stats()
    out["server_stats"] = {k: st[k] for k in ("batches", "max_batch", "kernel_launches", "arena_peak",
                                             "completed", "failed")}
    srv.close()
    ctx.close()
    return out


def _timed(stream, fn, warm=2, reps=5):
    """Milliseconds per call of fn() on `stream` (CUDA events, after warm-up)."""
    import torch
    for _ in range(warm):
        fn()
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


EXTRA_LEGS = ("plain_512", "multispectral", "windows", "histogram", "uneven")


def other_workloads(G, S, torch, local: int, only=None):
    """Device-resident throughput of the other workload shapes (each through
    the same public calls a user makes, inputs already in HBM):
    plain 512^2 N=8 levels-mode single offset; 8 bands of 8192^2 uint16 x 12
    offsets with symmetric normalized GLCMs and features in one batch; the
    2048^2 sliding-window texture maps (259,081 windows x 4 offsets), also
    without counts; the gray-level histogram of a 16384^2 uint8 image; 1000
    uneven uint8 images (64..2048) in one batch, and with the windows in one
    graph.  only: a set of EXTRA_LEGS names to run (None: all)."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor

    def want(name):
        return only is None or name in only

    out = {}
    stream = torch.cuda.Stream(device=local)
    ctx = G.Context(local, hbm_budget_bytes=8 << 30, stream=stream)
    with torch.cuda.stream(stream):
        # Plain method: one small image per call.
        if want("plain_512"):
            img, n, offs = S.plain_512()
            d = torch.from_numpy(img).cuda(local)
            c = torch.empty((1, n, n), dtype=torch.int32, device=f"cuda:{local}")
            ms = _timed(stream, lambda: ctx.compute(d, n, offs, G.GLCM_INPUT_LEVELS, out=c), warm=3, reps=50)
            out["plain_512"] = {"us_per_image": ms * 1e3, "gpairs_s": pairs_of(512, 512, offs) / (ms * 1e-3) / 1e9}
        # Multispectral bands.
        if want("multispectral"):
            with ThreadPoolExecutor(8) as ex:
                bands = list(ex.map(S.multispectral_band, range(8)))
            offs = S.MULTISPECTRAL_OFFSETS
            spec = [dict(image=torch.from_numpy(b).cuda(local), levels=32, offsets=offs, flags=G.GLCM_SYMMETRIC,
                         normalized=True, features=True) for b in bands]
            prepared = ctx.prepare(spec)
            ms = _timed(stream, lambda: ctx.run(prepared))
            pairs = 8 * pairs_of(8192, 8192, offs)
            out["multispectral_8x8192_u16"] = {"ms_per_batch": ms, "gpairs_s": pairs / (ms * 1e-3) / 1e9,
                                               "hbm_read_gbs": 8 * 8192 * 8192 * 2 / (ms * 1e-3) / 1e9}
            del spec, prepared, bands
        # Sliding-window texture maps.
        wimg = torch.from_numpy(S.window_image()).cuda(local)
        offs = S.CONTENTION_OFFSETS
        nw = ((2048 - 15) // 4 + 1) ** 2
        cw = torch.empty((509, 509, 4, 16, 16), dtype=torch.int32, device=f"cuda:{local}")
        mw = torch.empty((4, 4, 509, 509), dtype=torch.float32, device=f"cuda:{local}")
        src, w, h, pitch, dt = G.image_args(wimg)
        wp = nw * sum((15 - abs(dx)) * (15 - abs(dy)) for dx, dy in offs)
        if want("windows"):
            ms = _timed(stream, lambda: G.glcm_windows(ctx.ctx, src, w, h, pitch, dt, 16, 15, 4, offs,
                                                        G.GLCM_SYMMETRIC, cw, mw))
            out["windows_2048_15x15_s4"] = {"ms": ms, "windows_per_s": nw / (ms * 1e-3),
                                            "gpairs_s": wp / (ms * 1e-3) / 1e9}
        # Gray-level histogram of a 16384^2 uint8 image (268 MB, above L2), N = 256.
        if want("histogram"):
            himg = torch.from_numpy(S.iid(S.BASE_SEED + 900, 16384, 16384, np.uint8)).cuda(local)
            hh = torch.empty(256, dtype=torch.int32, device=f"cuda:{local}")
            hsrc, hw, hhgt, hpitch, hdt = G.image_args(himg)
            ms = _timed(stream, lambda: G.glcm_histogram(ctx.ctx, hsrc, hw, hhgt, hpitch, hdt, 256, 0, hh))
            hpeak, hkind = load_peaks()
            gbs = 16384 * 16384 / (ms * 1e-3) / 1e9
            out["histogram_16384_u8_n256"] = {"ms": ms, "gpixels_s": gbs, "hbm_read_gbs": gbs,
                                              "frac_of_hbm": gbs / hpeak, "peak_kind": f"{hkind} hbm_gbs (copy)"}
            del himg, hh
        # The same maps without the per-window counts (1.06 GB not written).
        if want("windows"):
            ms = _timed(stream, lambda: G.glcm_windows(ctx.ctx, src, w, h, pitch, dt, 16, 15, 4, offs,
                                                        G.GLCM_SYMMETRIC, None, mw))
            out["windows_2048_15x15_s4_maps_only"] = {"ms": ms, "windows_per_s": nw / (ms * 1e-3),
                                                      "gpairs_s": wp / (ms * 1e-3) / 1e9}
        del cw, mw
        if not want("uneven"):
            stream.synchronize()
            ctx.close()
            return out
        # 1000 uneven images.
        recipe = S.uneven_batch()
        with ThreadPoolExecutor(8) as ex:
            imgs = list(ex.map(lambda r: S.image(r["kind"], r["seed"], r["side"], r["side"], np.uint8, 4.0), recipe))
        spec = [dict(image=torch.from_numpy(im).cuda(local), levels=r["levels"], offsets=r["offsets"],
                     flags=G.GLCM_SYMMETRIC, normalized=False, features=True) for im, r in zip(imgs, recipe)]
        # Descriptors built once (prepare), so the timed calls measure the GPU, not
        # Python building 1000 descriptors per call.
        prepared = ctx.prepare(spec)
        ms = _timed(stream, lambda: ctx.run(prepared))
        pairs = sum(pairs_of(r["side"], r["side"], r["offsets"]) for r in recipe)
        out["uneven_1000"] = {"ms_per_batch": ms, "gpairs_s": pairs / (ms * 1e-3) / 1e9}
        del prepared
        # The whole of config 4 in one CUDA-graph launch: the 2048^2 window
        # counts and maps, then the 1000 images (glcm_compute_batch_windows).
        wjobs = [dict(image=wimg, levels=16, win=15, stride=4, offsets=S.CONTENTION_OFFSETS,
                      flags=G.GLCM_SYMMETRIC, counts=True, maps=True)]
        pw = ctx.prepare_batch_windows(spec, wjobs)
        ms = _timed(stream, lambda: ctx.run_batch_windows(pw))
        out["config4_one_graph"] = {"ms_per_launch": ms, "gpairs_s": (pairs + wp) / (ms * 1e-3) / 1e9,
                                    "windows": nw, "images": len(recipe), "graph_launches_per_call": 1}
        del pw
    stream.synchronize()
    ctx.close()
    return out


def ceilings_leg(G, local: int):
    """Measured ceilings of the vote kernels on this GPU (glcm_measure_ceilings):
    shared-memory reductions per second for interleaved copies, one word per
    warp and random words of one copy, and a streaming HBM read rate."""
    c = G.binding.glcm_measure_ceilings(local)
    c["kind"] = "measured by microbenchmark kernels in csrc/ceilings.cu (glcm_measure_ceilings)"
    return c


CLASS_POOL = 8  # distinct 4096^2 images per class (134 MB, above the 129 MB L2)


def class_lines(G, torch, ctx, imgs, jobs, local: int, peak: float, ceil_red: float | None, stream, reps: int = 5):
    """Per-class vote-kernel lines: each 4096^2 uint8 image timed alone (one
    glcm_compute per image, the context's CUDA events around its vote launch),
    for every kind and N of the sweep.  A class rotates over 8 distinct images:
    the sweep's four images of that kind and four circular shifts of them
    (the smooth generator is circular, so shifts keep its statistics).  Runs
    on the benchmark's context, so each class has the vote configuration the
    batch was timed with."""
    out = {}
    offs = jobs[0]["offsets"]
    pairs = pairs_of(4096, 4096, offs)
    by_kind = {}
    for im, j in zip(imgs, jobs):
        by_kind.setdefault(j["kind"], []).append(im)
    G.glcm_get_timing(ctx.ctx, reset=True)
    for kind, base in by_kind.items():
        with torch.cuda.stream(stream):
            pool = list(base) + [torch.roll(b, shifts=977 * (k + 1), dims=1) for k, b in enumerate(base)]
            pool = pool[:CLASS_POOL]
        for n in sorted({j["levels"] for j in jobs}):
            res = torch.empty((len(offs), n, n), dtype=torch.int32, device=f"cuda:{local}")
            with torch.cuda.stream(stream):
                for im in pool:
                    ctx.compute(im, n, offs, out=res)
                stream.synchronize()
                G.glcm_get_timing(ctx.ctx, reset=True)
                for _ in range(reps):
                    for im in pool:
                        ctx.compute(im, n, offs, out=res)
                ms, nl, _ = G.glcm_get_timing(ctx.ctx, reset=True)
            us = ms * 1e3 / (reps * len(pool))
            gbs = 4096 * 4096 / (us * 1e-6) / 1e9
            line = {"us_per_image": us, "hbm_read_gbs": gbs, "frac_of_hbm": gbs / peak,
                    "tvotes_s": pairs / (us * 1e-6) / 1e12, "vote_launches_per_image": nl / (reps * len(pool))}
            if ceil_red:
                line["frac_of_red_ceiling"] = pairs / (us * 1e-6) / ceil_red
            out[f"{kind}_N{n}"] = line
        del pool
    return out


def parity_leg(outs, jobs):
    """The timed batch's own results against the CPU oracle: counts bit for bit
    for every GLCM, symmetric normalized GLCMs within 4e-7 relative, features
    within 1e-5 scaled error (floor 1 for correlation and the three
    correlation measures, 1/N^2 for the rest).  Part of the CPU-baseline leg."""
    import numpy as np

    import oracle
    oracle.build()
    worst, worst_norm, bad = 0.0, 0.0, []
    for (c, nm, ft), j in zip(outs, jobs):
        P = oracle.glcm(j["image"], j["levels"], j["offsets"])
        got = c.cpu().numpy().view(np.uint32)
        if not np.array_equal(got, P):
            bad.append(f"{j['kind']} N={j['levels']}: counts differ at {int((got != P).sum())} bins")
            continue
        S_ = oracle.symmetrize(P)
        pw = oracle.normalize(S_)
        g = nm.cpu().numpy().astype(np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            rn = np.where(pw > 0, np.abs(g - pw) / pw, np.abs(g - pw))
        worst_norm = max(worst_norm, float(rn.max()))
        fw = oracle.haralick_batch(P, True)
        floor = np.full(14, 1.0 / (j["levels"] ** 2))
        floor[[2, 11, 12, 13]] = 1.0
        err = np.abs(ft.cpu().numpy().astype(np.float64) - fw) / np.maximum(np.abs(fw), floor)
        worst = max(worst, float(err.max()))
    ok = not bad and worst <= 1e-5 and worst_norm <= 4e-7
    return {"counts": "bit_exact" if not bad else "MISMATCH", "glcms": sum(len(j["offsets"]) for j in jobs),
            "max_scaled_feature_error": worst, "max_normalized_rel_error": worst_norm, "ok": ok,
            "failures": bad}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-all-seconds", type=float, default=6.0,
                    help="seconds of the all-core oracle run beside the 1-thread one (0: skip)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workload shapes")
    ap.add_argument("--extra", default="", help="comma-separated subset of the other workload shapes to run: "
                    + ", ".join(EXTRA_LEGS) + " (default: all)")
    ap.add_argument("--no-tune", action="store_true", help="use the planner's default vote configurations")
    ap.add_argument("--no-classes", action="store_true", help="skip the per-class single-image lines")
    ap.add_argument("--no-ceilings", action="store_true", help="skip the shared-reduction / HBM ceilings")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import glcm_synth as S
    import paper_1710_06189_gb300 as G

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    G.binding.load()

    ceilings = None if args.no_ceilings else ceilings_leg(G, local)
    jobs = S.contention_jobs(4096)
    pairs_step = sum(pairs_of(4096, 4096, j["offsets"]) for j in jobs)
    bytes_step = sum(j["image"].nbytes for j in jobs)
    stream = torch.cuda.Stream(device=local)
    ctx = G.Context(local, hbm_budget_bytes=16 << 30, stream=stream)
    G.glcm_set_timing(ctx.ctx, True)
    with torch.cuda.stream(stream):
        imgs = [torch.from_numpy(j["image"]).cuda(local) for j in jobs]
    stream.synchronize()
    spec = [dict(image=im, levels=j["levels"], offsets=j["offsets"], flags=G.GLCM_SYMMETRIC,
                 normalized=True, features=True) for im, j in zip(imgs, jobs)]
    # Vote configuration per (levels, offsets) class, tuned on this batch
    # itself before anything is measured (the planner's defaults are the
    # incumbents; cached per GPU).
    from paper_1710_06189_gb300 import autotune
    tuned = {}
    if not args.no_tune:
        cache = autotune.TuneCache(os.path.join(ROOT, "paper_1710_06189_gb300", "_build", "vote_tune.json"))
        with torch.cuda.stream(stream):
            tuned = autotune.tune_batch(ctx, spec, cache=cache, gpu=torch.cuda.get_device_name(local))
    G.glcm_get_timing(ctx.ctx, reset=True)
    with torch.cuda.stream(stream):
        step_batch = ctx.prepare(spec)  # descriptors and output buffers, built once
        ctx.run(step_batch)  # plan + capture
        for _ in range(max(3, args.warmup)):
            ctx.run(step_batch)
    stream.synchronize()

    barrier, max_over_ranks = rank_helpers(dist)

    # --- device-resident, batched (the headline value) ---
    # Timed on the graph without the vote-timing event nodes (the host
    # re-points those before every replay); the vote kernels' own time for
    # the roofline comes from a second pass of the same step with them.
    G.glcm_set_timing(ctx.ctx, False)
    with torch.cuda.stream(stream):
        ctx.run(step_batch)  # capture the uninstrumented graph
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        keep_loaded(lambda: ctx.run(step_batch), LOAD_SECONDS)
        G.glcm_get_timing(ctx.ctx, reset=True)
        barrier()
        torch.cuda.synchronize()
        clk.mark(True)
        e0.record(stream)
        for _ in range(args.steps):
            ctx.run(step_batch)
        e1.record(stream)
        torch.cuda.synchronize()
        clk.mark(False)
        _, _, launches = G.glcm_get_timing(ctx.ctx, reset=True)
        keep_loaded(lambda: ctx.run(step_batch), LOAD_SECONDS)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    value = whole_job_value(world, pairs_step, args.steps, ms * 1e-3)
    # Vote-kernel time per step (CUDA events around the step's vote launches).
    G.glcm_set_timing(ctx.ctx, True)
    vote_steps = max(20, min(args.steps, 200))
    with torch.cuda.stream(stream):
        ctx.run(step_batch)  # the instrumented graph
        stream.synchronize()
        G.glcm_get_timing(ctx.ctx, reset=True)
        for _ in range(vote_steps):
            ctx.run(step_batch)
    vote_ms, vote_n, _ = G.glcm_get_timing(ctx.ctx, reset=True)

    # --- plain: one image at a time, sync per image ---
    plain_steps = max(3, args.steps // 5)
    plain_outs = [(torch.empty((4, j["levels"], j["levels"]), dtype=torch.int32, device=f"cuda:{local}"),
                   torch.empty((4, j["levels"], j["levels"]), dtype=torch.float32, device=f"cuda:{local}"),
                   torch.empty((4, 14), dtype=torch.float32, device=f"cuda:{local}")) for j in jobs]

    def plain_step():
        for im, j, (c, nm, ft) in zip(imgs, jobs, plain_outs):
            ctx.compute(im, j["levels"], j["offsets"], G.GLCM_SYMMETRIC, normalized=True, out=c, norm_out=nm)
            ctx.features(c, j["levels"], symmetric=True, out=ft)
            stream.synchronize()

    plain_step()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(plain_steps):
        plain_step()
    torch.cuda.synchronize()
    plain_s = max_over_ranks(time.perf_counter() - t0)
    plain_value = world * pairs_step * plain_steps / plain_s / 1e9
    G.glcm_get_timing(ctx.ctx, reset=True)

    # --- end to end through the C ABI with pinned host buffers ---
    hosts = [torch.from_numpy(j["image"]).pin_memory() for j in jobs]
    h_outs = [(torch.empty((4, j["levels"], j["levels"]), dtype=torch.int32).pin_memory(),
               torch.empty((4, j["levels"], j["levels"]), dtype=torch.float32).pin_memory(),
               torch.empty((4, 14), dtype=torch.float32).pin_memory()) for j in jobs]
    h_spec = [dict(image=h, levels=j["levels"], offsets=j["offsets"], flags=G.GLCM_SYMMETRIC, counts=o[0],
                   normalized=o[1], features=o[2]) for h, j, o in zip(hosts, jobs, h_outs)]
    h_batch = ctx.prepare(h_spec)  # descriptors built once, as a serving caller would
    ctx.run(h_batch)
    e2e_steps = max(10, args.steps // 2)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.run(h_batch)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = world * pairs_step * e2e_steps / e2e_s / 1e9
    d2h = sum(o[0].numel() * 4 + o[1].numel() * 4 + o[2].numel() * 4 for o in h_outs)

    peak, peak_kind = load_peaks()
    classes = None
    if not args.no_classes:
        classes = class_lines(G, torch, ctx, imgs, jobs, local, peak,
                              ceilings["red_interleaved_per_s"] if ceilings else None, stream)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # One CUDA-event pair brackets all vote launches of a step (one launch, or
    # two when the batch is split so that expensive epilogues overlap votes).
    avg_vote_ms = vote_ms / max(1, vote_steps)
    achieved = bytes_step / (avg_vote_ms * 1e-3) / 1e9 if (vote_n and avg_vote_ms > 0) else None
    traffic = profiled_traffic("vote_contention_4096.md")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(),
        "vote_configs": tuned or "planner defaults",
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": "vote kernels (k_glcm_vote_d1 column walk, k_glcm_vote general)",
                     "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                     "vote_ms_per_step": avg_vote_ms, "vote_launches_per_step": vote_n / max(1, vote_steps), "vote_steps_timed": vote_steps,
                     "algorithmic_bytes_per_step": bytes_step},
        "plain": {"value": plain_value, "unit": UNIT, "batched_over_plain": value / plain_value},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bytes_step, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if ceilings:
        line["ceilings"] = ceilings
        line["roofline"]["red_ceiling_per_s"] = ceilings["red_interleaved_per_s"]
        line["roofline"]["tvotes_s"] = pairs_step / (avg_vote_ms * 1e-3) / 1e12 if avg_vote_ms > 0 else None
    if classes:
        line["classes"] = {"workload": "one 4096^2 uint8 image per launch, 4 offsets at d = 1, vote kernel only "
                                       "(CUDA events), 8 distinct images per class (134 MB > L2)",
                           "peak_kind": f"{peak_kind} hbm_gbs (copy)", "lines": classes}
    if not args.no_serving:
        line["serving"] = serving_leg(G, S, torch, local)
    if not args.no_extra:
        only = {x for x in args.extra.split(",") if x} or None
        bad = sorted(only - set(EXTRA_LEGS)) if only else []
        if bad:
            raise SystemExit(f"unknown --extra leg(s): {bad}")
        line["other_workloads"] = other_workloads(G, S, torch, local, only)
    parity = None
    if not args.no_cpu_baseline and world == 1:
        # The oracle, first on the timed batch's own results (untimed), then timed.
        parity = parity_leg(step_batch.outs, jobs)
        line["parity"] = parity
        v, desc = oracle_sample(jobs, args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
        if args.cpu_all_seconds > 0:
            va, nt, da = oracle_sample_all_cores(jobs, args.cpu_all_seconds)
            line["cpu_baseline"]["all_cores"] = {"value": va, "unit": UNIT, "cores": nt, "sample": da}
    else:
        line["parity"] = "not checked (no CPU-baseline leg)"
    print(json.dumps(line))
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    if parity is not None and not parity["ok"]:
        print(f"parity check failed: {parity}", file=sys.stderr)
        return 1
    return 0


if __name__ == "__main__":
    sys.exit(main())
