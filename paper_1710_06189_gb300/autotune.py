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
    """Summed vote-kernel milliseconds per pass over `images` (device tensors)."""
    import torch
    outs = [torch.empty((len(offsets), levels, levels), dtype=torch.int32, device=im.device) for im in images]
    for im, out in zip(images, outs):  # warm-up (plans, attributes)
        ctx.compute(im, levels, offsets, flags, out=out)
    ctx.synchronize()
    B.glcm_get_timing(ctx.ctx, reset=True)
    for _ in range(reps):
        for im, out in zip(images, outs):
            ctx.compute(im, levels, offsets, flags, out=out)
    ms, _, _ = B.glcm_get_timing(ctx.ctx, reset=True)
    return ms / max(1, reps)


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
        if ms < best["ms"]:
            best = tried[-1]
    B.glcm_set_vote_config(ctx.ctx, levels, n_off, dtype, best["threads"], best["log2_copies"], best["layout"],
                           best["band_rows"])
    return dict(best, tried=tried)


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
