"""GB300 (sm_103a) gray-level co-occurrence matrices behind a C ABI.

``binding`` holds the ctypes functions with the C names of include/glcm.h.
``Context`` below is a thin convenience layer over them that takes and
returns torch tensors (PyTorch supplies device memory and streams only; all
computation runs in libglcm's CUDA kernels).  Counts are returned as int32
tensors holding the uint32 bit patterns (counts never exceed 2^31 for images
up to 46340^2).
"""
from __future__ import annotations

from . import binding
from .binding import (GLCM_ERR_BUSY, GLCM_ERR_NOMEM, GLCM_ERR_RANGE, GLCM_FLAT_WRAP, GLCM_INPUT_LEVELS, GLCM_NORMALIZE,
                      GLCM_OK,
                      GLCM_SYMMETRIC, GLCM_U8, GLCM_U16, GlcmError,
                      glcm_compute, glcm_compute_batch, glcm_compute_naive, glcm_create, glcm_destroy,
                      glcm_features, glcm_get_timing, glcm_last_error, glcm_offset_from_angle,
                      glcm_histogram, glcm_set_timing, glcm_set_vote_config, glcm_synchronize, glcm_windows)

__all__ = [
    "PreparedBatch",
    "binding", "Context", "Server", "GlcmError", "GLCM_OK", "GLCM_ERR_BUSY", "GLCM_ERR_NOMEM", "GLCM_ERR_RANGE", "GLCM_SYMMETRIC", "GLCM_NORMALIZE", "GLCM_INPUT_LEVELS", "GLCM_FLAT_WRAP", "GLCM_U8",
    "GLCM_U16", "glcm_compute", "glcm_compute_batch", "glcm_compute_naive", "glcm_create", "glcm_destroy",
    "glcm_features", "glcm_get_timing", "glcm_last_error", "glcm_offset_from_angle", "glcm_set_timing",
    "glcm_set_vote_config", "glcm_synchronize", "glcm_windows", "glcm_histogram",
]


def _torch():
    import torch
    return torch


def image_args(img):
    """(pointer source, width, height, pitch_bytes, dtype) of a 2-D image tensor or array."""
    torch = _torch()
    if isinstance(img, torch.Tensor):
        if img.dim() != 2 or img.stride(1) != 1:
            raise ValueError("image must be a 2-D tensor with unit column stride")
        if img.dtype == torch.uint8:
            dt = GLCM_U8
        elif img.dtype in (torch.uint16, torch.int16):
            dt = GLCM_U16
        else:
            raise ValueError("image must be uint8 or uint16")
        return img, img.shape[1], img.shape[0], img.stride(0) * img.element_size(), dt
    import numpy as np
    a = img
    if a.ndim != 2 or a.strides[1] != a.itemsize:
        raise ValueError("image must be a 2-D array with unit column stride")
    dt = {np.dtype(np.uint8): GLCM_U8, np.dtype(np.uint16): GLCM_U16}[a.dtype]
    return a, a.shape[1], a.shape[0], a.strides[0], dt


class PreparedBatch:
    """Descriptors of a batch (a ctypes glcm_desc array), the output buffers,
    and the offset arrays the descriptors point to (kept alive here)."""

    def __init__(self, descs, outs, keep):
        self.descs = descs
        self.outs = outs
        self._keep = keep


class Context:
    """A libglcm context on one device; results are torch tensors."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, stream=None):
        torch = _torch()
        self.device = device
        self.stream = stream
        handle = None
        if stream is not None:
            handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.ctx = glcm_create(device, hbm_budget_bytes, handle)
        self._torch_device = torch.device("cuda", device)

    def close(self):
        if self.ctx is not None:
            glcm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, shape, dtype, like_device=True):
        torch = _torch()
        return torch.empty(shape, dtype=dtype, device=self._torch_device if like_device else "cpu")

    def compute(self, img, levels: int, offsets, flags: int = 0, normalized: bool = False, out=None,
                norm_out=None):
        torch = _torch()
        src, w, h, pitch, dt = image_args(img)
        n = len(offsets)
        on_dev = isinstance(img, torch.Tensor) and img.is_cuda
        counts = out if out is not None else self._empty((n, levels, levels), torch.int32, on_dev)
        norm = None
        if normalized:
            flags |= GLCM_NORMALIZE
            norm = norm_out if norm_out is not None else self._empty((n, levels, levels), torch.float32, on_dev)
        glcm_compute(self.ctx, src, w, h, pitch, dt, levels, offsets, flags, counts, norm)
        return (counts, norm) if normalized else counts

    def features(self, counts, levels: int, symmetric: bool = False, out=None):
        torch = _torch()
        n = counts.numel() // (levels * levels)
        feats = out if out is not None else self._empty((n, 14), torch.float32, counts.is_cuda)
        glcm_features(self.ctx, counts, levels, n, GLCM_SYMMETRIC if symmetric else 0, feats)
        return feats.reshape(tuple(counts.shape[:-2]) + (14,))

    def batch(self, jobs):
        """jobs: list of dicts {image, levels, offsets, flags, counts, normalized, features};
        missing outputs are allocated (counts always; normalized / features when True)."""
        prepared = self.prepare(jobs)
        glcm_compute_batch(self.ctx, prepared.descs)
        return prepared.outs

    def prepare(self, jobs):
        """The descriptors of a batch, built once: run(prepared) then repeats the
        batch on the same buffers with a single call (no per-image Python work).
        Outputs are allocated as in batch()."""
        torch = _torch()
        descs = []
        outs = []
        for jb in jobs:
            src, w, h, pitch, dt = image_args(jb["image"])
            n, N = len(jb["offsets"]), jb["levels"]
            dev = isinstance(jb["image"], torch.Tensor) and jb["image"].is_cuda
            c = jb.get("counts")
            if c is None:
                c = self._empty((n, N, N), torch.int32, dev)
            nm = jb.get("normalized")
            if nm is True:
                nm = self._empty((n, N, N), torch.float32, dev)
            ft = jb.get("features")
            if ft is True:
                ft = self._empty((n, 14), torch.float32, dev)
            nm = nm if nm is not False else None
            ft = ft if ft is not False else None
            descs.append(binding.make_desc(src, w, h, pitch, dt, N, jb["offsets"], jb.get("flags", 0), c, nm, ft))
            outs.append((c, nm, ft))
        return PreparedBatch(binding.desc_array(descs), outs, descs)

    def run(self, prepared):
        """Run a batch from prepare() again (same images and output buffers)."""
        glcm_compute_batch(self.ctx, prepared.descs)
        return prepared.outs

    def prepare_batch_windows(self, jobs, windows):
        """A batch of images (as prepare()) plus sliding-window jobs -- dicts
        {image, levels, win, stride, offsets, flags, counts, maps} with counts /
        maps True (allocated here), False or a device tensor -- for
        run_batch_windows: one CUDA-graph launch per call.  Device buffers only."""
        torch = _torch()
        prepared = self.prepare(jobs)
        wdescs, wouts = [], []
        for w in windows:
            src, wd, ht, pitch, dt = image_args(w["image"])
            n_off, N = len(w["offsets"]), w["levels"]
            nwx, nwy = (wd - w["win"]) // w["stride"] + 1, (ht - w["win"]) // w["stride"] + 1
            c = w.get("counts", False)
            c = self._empty((nwy, nwx, n_off, N, N), torch.int32) if c is True else (c if c is not False else None)
            m = w.get("maps", True)
            m = self._empty((4, n_off, nwy, nwx), torch.float32) if m is True else (m if m is not False else None)
            wdescs.append(binding.make_window_desc(src, wd, ht, pitch, dt, N, w["win"], w["stride"], w["offsets"],
                                                   w.get("flags", 0), c, m))
            wouts.append((c, m))
        return PreparedBatch(prepared.descs, (prepared.outs, wouts), (prepared, wdescs))

    def run_batch_windows(self, prepared):
        """Run (first call: run and capture; then replay) a prepare_batch_windows batch:
        returns (image outputs, window outputs)."""
        _, wdescs = prepared._keep
        binding.glcm_compute_batch_windows(self.ctx, prepared.descs, wdescs)
        return prepared.outs

    def windows(self, img, levels: int, win: int, stride: int, offsets, flags: int = 0, counts: bool = True,
                maps: bool = True):
        torch = _torch()
        src, w, h, pitch, dt = image_args(img)
        nwx, nwy = (w - win) // stride + 1, (h - win) // stride + 1
        dev = isinstance(img, torch.Tensor) and img.is_cuda
        n = len(offsets)
        c = self._empty((nwy, nwx, n, levels, levels), torch.int32, dev) if counts else None
        m = self._empty((4, n, nwy, nwx), torch.float32, dev) if maps else None
        glcm_windows(self.ctx, src, w, h, pitch, dt, levels, win, stride, offsets, flags, c, m)
        return c, m

    def histogram(self, img, levels: int, flags: int = 0, out=None):
        """glcm_histogram: pixels per level, int32 view of uint32 [levels]."""
        torch = _torch()
        src, w, h, pitch, dt = image_args(img)
        on_dev = isinstance(img, torch.Tensor) and img.is_cuda
        hist = out if out is not None else self._empty((levels,), torch.int32, on_dev)
        glcm_histogram(self.ctx, src, w, h, pitch, dt, levels, flags, hist)
        return hist

    def enqueue_batch(self, jobs):
        """glcm_enqueue_batch: the batch launched directly, no graph, no sync;
        jobs as for batch() with device tensors only."""
        torch = _torch()
        descs, outs = [], []
        for jb in jobs:
            src, w, h, pitch, dt = image_args(jb["image"])
            n, N = len(jb["offsets"]), jb["levels"]
            c = jb.get("counts")
            if c is None:
                c = self._empty((n, N, N), torch.int32)
            nm = jb.get("normalized")
            nm = self._empty((n, N, N), torch.float32) if nm is True else (nm if nm is not False else None)
            ft = jb.get("features")
            ft = self._empty((n, 14), torch.float32) if ft is True else (ft if ft is not False else None)
            descs.append(binding.make_desc(src, w, h, pitch, dt, N, jb["offsets"], jb.get("flags", 0), c, nm, ft))
            outs.append((c, nm, ft))
        binding.glcm_enqueue_batch(self.ctx, descs)
        self._keep = descs
        return outs

    def synchronize(self):
        glcm_synchronize(self.ctx)


class Server:
    """Continuous-batching GLCM server on one device (glcm_server_*).

    submit() queues a host image and returns a ticket; wait() returns
    (status, latency_ms, (counts, normalized, features)).  Outputs are
    allocated in pinned host memory unless given.  The image and the outputs
    are kept referenced here until the request is waited for."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, lanes: int = 0, max_batch: int = 0,
                 max_queue: int = 0):
        self.server = binding.glcm_server_create(device, hbm_budget_bytes, lanes, max_batch, max_queue)
        self._live = {}

    def submit(self, image, levels: int, offsets, flags: int = 0, counts=None, normalized=False, features=False,
               pin: bool = True):
        torch = _torch()
        src, w, h, pitch, dt = image_args(image)
        n = len(offsets)

        def host(shape, dtype):
            t = torch.empty(shape, dtype=dtype)
            return t.pin_memory() if pin else t

        c = counts if counts is not None else host((n, levels, levels), torch.int32)
        nm = normalized if not isinstance(normalized, bool) else (host((n, levels, levels), torch.float32)
                                                                  if normalized else None)
        ft = features if not isinstance(features, bool) else (host((n, 14), torch.float32) if features else None)
        desc = binding.make_desc(src, w, h, pitch, dt, levels, offsets, flags, c, nm, ft)
        t = binding.glcm_server_submit(self.server, desc)
        self._live[t] = (desc, image, (c, nm, ft))
        return t

    def wait(self, ticket: int, timeout_ms: int = -1):
        st, lat = binding.glcm_server_wait(self.server, ticket, timeout_ms)
        if st == GLCM_ERR_BUSY:
            return st, None, None
        _, _, outs = self._live.pop(ticket)
        return st, lat, outs

    def stats(self):
        return binding.glcm_server_stats(self.server)

    def last_error(self):
        return binding.glcm_server_last_error(self.server)

    def close(self):
        if self.server is not None:
            binding.glcm_server_destroy(self.server)
            self.server = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
