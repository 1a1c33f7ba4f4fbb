"""Autotuner for the vote kernel.

For one (levels, offsets, pixel type) class it times every feasible vote
configuration -- threads per CTA, log2 of the private histogram copies and
the shared-memory layout, including the column-walk kernel (layout 4; see
glcm_set_vote_config) -- on the caller's own images, then the tile shape
(anchor rows per work item) of the winner.  The paper picks block size and
copy count from Eqs. 4-6 and by experiment (Sec. II.B); here the experiment
is automated.  The best configuration is applied to the context and kept in
a JSON cache keyed by GPU name and class, so later runs can apply it without
timing.

All timing is of the vote kernel alone, with CUDA events on the context's
stream (glcm_set_timing / glcm_get_timing).
"""
from __future__ import annotations

import json
import os

from . import binding as B

DEFAULT_CANDIDATES = tuple([(512, 5, 4)] + [(512, r, lay) for r in (5, 4, 3, 2, 1, 0) for lay in (1, 0, 2, 3)] +
                           [(256, 5, 1), (1024, 5, 1), (1024, 0, 3)])
# Anchor rows per work item tried for the winning configuration (0: the
# planner's choice); the general kernel's tiles hold at most 64.
BAND_CANDIDATES = {4: (0, 8, 16, 32, 64, 128), "general": (0, 16, 32, 64)}


def class_key(levels: int, n_offsets: int, dtype: int) -> str:
    return f"N{levels}_off{n_offsets}_{'u8' if dtype == B.GLCM_U8 else 'u16'}"


def _time_config(ctx, images, levels, offsets, flags, reps):
    """Vote-kernel milliseconds per pass over `images` (device tensors), run as
    one batch -- the way a batch of the class's images votes: one launch for
    all of them, its chunks spread over the GPU -- from a prepared (and after
    its first run, graph-captured) batch."""
    prepared = ctx.prepare([dict(image=im, levels=levels, offsets=offsets, flags=flags) for im in images])
    ctx.run(prepared)  # plan, attributes, capture
    ctx.synchronize()
    B.glcm_get_timing(ctx.ctx, reset=True)
    for _ in range(reps):
        ctx.run(prepared)
    ctx.synchronize()
    ms, _, _ = B.glcm_get_timing(ctx.ctx, reset=True)
    return ms / max(1, reps)


# A band height other than the planner's own choice (0) must be this much
# faster to be kept: the planner cuts bands for each launch's CTA count, a
# fixed height only for the tuning run's.
BAND_MARGIN = 0.03


def tune(ctx, images, levels: int, offsets, flags: int = 0, reps: int = 3, candidates=DEFAULT_CANDIDATES):
    """Time the candidates on `images` (a list of 2-D device tensors of one
    pixel type), apply the fastest to `ctx` and return
    {"threads", "log2_copies", "layout", "ms", "tried": [...]}."""
    from . import image_args
    dtype = image_args(images[0])[4]
    n_off = len(offsets)
    B.glcm_set_timing(ctx.ctx, True)
    tried = []
    best = None
    for threads, r, layout in candidates:
        try:
            B.glcm_set_vote_config(ctx.ctx, levels, n_off, dtype, threads, r, layout, 0)
        except B.GlcmError:
            continue  # histograms do not fit this configuration
        ms = _time_config(ctx, images, levels, offsets, flags, reps)
        tried.append({"threads": threads, "log2_copies": r, "layout": layout, "band_rows": 0, "ms": ms})
        if best is None or ms < best["ms"]:
            best = tried[-1]
    if best is None:
        B.glcm_set_vote_config(ctx.ctx, levels, n_off, dtype, 0, 0, 0, 0)
        return None
    # Tile shape of the winner.
    for band in BAND_CANDIDATES[4 if best["layout"] == 4 else "general"][1:]:
        try:
            B.glcm_set_vote_config(ctx.ctx, levels, n_off, dtype, best["threads"], best["log2_copies"],
                                   best["layout"], band)
        except B.GlcmError:
            continue
        ms = _time_config(ctx, images, levels, offsets, flags, reps)
        tried.append({"threads": best["threads"], "log2_copies": best["log2_copies"], "layout": best["layout"],
                      "band_rows": band, "ms": ms})
        if ms < best["ms"] * (1.0 - BAND_MARGIN):
            best = tried[-1]
    B.glcm_set_vote_config(ctx.ctx, levels, n_off, dtype, best["threads"], best["log2_copies"], best["layout"],
                           best["band_rows"])
    return dict(best, tried=tried)


def _time_batch(ctx, prepared, reps, trials: int = 3):
    """Milliseconds of one run of a prepared batch: the best of `trials`
    timings of `reps` back-to-back graph replays between two synchronizations
    of the context's stream (wall clock; the replays queue on the GPU, so their
    launches overlap the work), after one untimed run that captures the graph
    for the current configuration."""
    import time
    ctx.run(prepared)
    ctx.synchronize()
    best = None
    for _ in range(trials):
        t0 = time.perf_counter()
        for _ in range(reps):
            ctx.run(prepared)
        ctx.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / max(1, reps)
        best = ms if best is None else min(best, ms)
    return best


# A configuration replaces the incumbent of its class only if the whole
# batch gets at least this much faster (above the spread of repeated timings).
BATCH_MARGIN = 0.02


def tune_batch(ctx, jobs, reps: int = 10, candidates=DEFAULT_CANDIDATES, cache: "TuneCache | None" = None,
               gpu: str = ""):
    """Tune every vote class of a batch on the batch itself: for one class at
    a time (the others at their incumbents), every feasible (threads, copies,
    layout) and then the winner's band heights are timed as the whole
    prepared batch (`jobs`: the dicts of Context.prepare), so a class is tuned
    in the launch shape it has in that batch (e.g. on the SMs a split batch
    leaves to it).  The incumbent is the planner's default; a candidate
    replaces it only if the batch is BATCH_MARGIN faster.  Returns {class key:
    chosen config} and applies the choices to ctx."""
    from . import image_args
    classes = {}
    for j in jobs:
        dtype = image_args(j["image"])[4]
        classes[(j["levels"], len(j["offsets"]), dtype)] = True
    prepared = ctx.prepare(jobs)
    chosen = {}
    for (levels, n_off, dtype) in classes:
        key = class_key(levels, n_off, dtype)
        if cache is not None and cache.apply(ctx, gpu, levels, n_off, dtype):
            chosen[key] = cache.get(gpu, key)
            continue
        B.glcm_set_vote_config(ctx.ctx, levels, n_off, dtype, 0, 0, 0, 0)  # planner default
        best = {"threads": 0, "log2_copies": 0, "layout": 0, "band_rows": 0,
                "ms": _time_batch(ctx, prepared, reps)}
        default_ms = best["ms"]
        for threads, r, layout in candidates:
            try:
                B.glcm_set_vote_config(ctx.ctx, levels, n_off, dtype, threads, r, layout, 0)
            except B.GlcmError:
                continue
            ms = _time_batch(ctx, prepared, reps)
            if ms < best["ms"] * (1.0 - BATCH_MARGIN):
                best = {"threads": threads, "log2_copies": r, "layout": layout, "band_rows": 0, "ms": ms}
        if best["threads"]:
            for band in BAND_CANDIDATES[4 if best["layout"] == 4 else "general"][1:]:
                try:
                    B.glcm_set_vote_config(ctx.ctx, levels, n_off, dtype, best["threads"], best["log2_copies"],
                                           best["layout"], band)
                except B.GlcmError:
                    continue
                ms = _time_batch(ctx, prepared, reps)
                if ms < best["ms"] * (1.0 - BATCH_MARGIN):
                    best = dict(best, band_rows=band, ms=ms)
        B.glcm_set_vote_config(ctx.ctx, levels, n_off, dtype, best["threads"], best["log2_copies"],
                               best["layout"], best["band_rows"])
        best["default_ms"] = default_ms
        chosen[key] = best
        if cache is not None:
            cache.put(gpu, key, best)
    if cache is not None:
        cache.save()
    return chosen


class TuneCache:
    """JSON cache {gpu name: {class key: config}}."""

    def __init__(self, path: str):
        self.path = path
        self.data = {}
        if os.path.exists(path):
            with open(path) as f:
                self.data = json.load(f)

    def get(self, gpu: str, key: str):
        return self.data.get(gpu, {}).get(key)

    def put(self, gpu: str, key: str, cfg: dict):
        self.data.setdefault(gpu, {})[key] = {k: cfg.get(k, 0) for k in ("threads", "log2_copies", "layout",
                                                                           "band_rows", "ms")}

    def save(self):
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def apply(self, ctx, gpu: str, levels: int, n_offsets: int, dtype: int) -> bool:
        cfg = self.get(gpu, class_key(levels, n_offsets, dtype))
        if not cfg:
            return False
        B.glcm_set_vote_config(ctx.ctx, levels, n_offsets, dtype, cfg["threads"], cfg["log2_copies"],
                               cfg["layout"], cfg.get("band_rows", 0))
        return True


def tune_classes(ctx, groups, flags: int = 0, cache: TuneCache | None = None, gpu: str = "", reps: int = 2):
    """Tune every class in `groups`: {(levels, offsets tuple): [device images]}.
    Returns {class key: chosen config}."""
    from . import image_args
    chosen = {}
    for (levels, offsets), images in groups.items():
        dtype = image_args(images[0])[4]
        key = class_key(levels, len(offsets), dtype)
        if cache is not None and cache.apply(ctx, gpu, levels, len(offsets), dtype):
            chosen[key] = cache.get(gpu, key)
            continue
        res = tune(ctx, images, levels, list(offsets), flags, reps)
        if res is not None:
            chosen[key] = {k: res[k] for k in ("threads", "log2_copies", "layout", "band_rows", "ms")}
            if cache is not None:
                cache.put(gpu, key, res)
    if cache is not None:
        cache.save()
    return chosen
