"""ctypes binding of libglcm: the C ABI of include/glcm.h, same names.

Argument marshalling only -- every step of the GLCM path runs in the CUDA
library.  Pointers may be given as torch tensors (``data_ptr()``), numpy
arrays (host memory), plain integers or None.  A non-zero status raises
``GlcmError`` carrying the library's message.  There is no fallback: if the
shared library is missing the import of the functions fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

c_int, c_size_t, c_void_p, c_double, c_longlong = (ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p,
                                                   ctypes.c_double, ctypes.c_longlong)

GLCM_OK = 0
GLCM_ERR_ARG = -1
GLCM_ERR_RANGE = -2
GLCM_ERR_NOMEM = -3
GLCM_ERR_UNSUPPORTED = -4
GLCM_ERR_CUDA = -5
GLCM_ERR_TIMEOUT = -6
GLCM_ERR_BUSY = -7
GLCM_U8, GLCM_U16 = 0, 1
GLCM_SYMMETRIC, GLCM_NORMALIZE, GLCM_INPUT_LEVELS, GLCM_FLAT_WRAP = 1, 2, 4, 8
GLCM_N_FEATURES = 14
GLCM_N_WINDOW_MAPS = 4

HEADER = os.path.join(_build.ROOT, "include", "glcm.h")


class glcm_offset(ctypes.Structure):
    _fields_ = [("dx", c_int), ("dy", c_int)]


class glcm_desc(ctypes.Structure):
    _fields_ = [("image", c_void_p), ("width", c_int), ("height", c_int), ("pitch_bytes", c_size_t),
                ("dtype", c_int), ("levels", c_int), ("offsets", ctypes.POINTER(glcm_offset)),
                ("n_offsets", c_int), ("flags", c_int), ("counts", c_void_p), ("normalized", c_void_p),
                ("features", c_void_p)]


class glcm_window_desc(ctypes.Structure):
    _fields_ = [("image", c_void_p), ("width", c_int), ("height", c_int), ("pitch_bytes", c_size_t),
                ("dtype", c_int), ("levels", c_int), ("win", c_int), ("stride", c_int),
                ("offsets", ctypes.POINTER(glcm_offset)), ("n_offsets", c_int), ("flags", c_int),
                ("counts", c_void_p), ("maps", c_void_p)]


class glcm_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", c_longlong), ("completed", c_longlong), ("failed", c_longlong),
                ("batches", c_longlong), ("max_batch", c_longlong), ("kernel_launches", c_longlong),
                ("queue_peak", c_longlong), ("arena_bytes", c_size_t), ("arena_peak", c_size_t)]


class glcm_ceilings_t(ctypes.Structure):
    _fields_ = [("sm_count", c_int), ("red_interleaved_per_s", c_double), ("red_same_word_per_s", c_double),
                ("red_random_one_copy_per_s", c_double), ("hbm_read_gbs", c_double)]


class GlcmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"glcm status {status}: {message}")
        self.status = status


_PROTOS = {
    "glcm_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_size_t, c_void_p]),
    "glcm_destroy": (c_int, [c_void_p]),
    "glcm_last_error": (ctypes.c_char_p, [c_void_p]),
    "glcm_offset_from_angle": (c_int, [c_int, c_int, ctypes.POINTER(glcm_offset)]),
    "glcm_compute": (c_int, [c_void_p, c_void_p, c_int, c_int, c_size_t, c_int, c_int,
                             ctypes.POINTER(glcm_offset), c_int, c_int, c_void_p, c_void_p]),
    "glcm_features": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "glcm_compute_batch": (c_int, [c_void_p, ctypes.POINTER(glcm_desc), c_int]),
    "glcm_enqueue_batch": (c_int, [c_void_p, ctypes.POINTER(glcm_desc), c_int]),
    "glcm_server_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_size_t, c_int, c_int, c_int]),
    "glcm_server_submit": (c_int, [c_void_p, ctypes.POINTER(glcm_desc), ctypes.POINTER(c_longlong)]),
    "glcm_server_wait": (c_int, [c_void_p, c_longlong, c_int, ctypes.POINTER(c_double)]),
    "glcm_server_stats": (c_int, [c_void_p, ctypes.POINTER(glcm_server_stats_t)]),
    "glcm_server_last_error": (ctypes.c_char_p, [c_void_p]),
    "glcm_server_destroy": (c_int, [c_void_p]),
    "glcm_windows": (c_int, [c_void_p, c_void_p, c_int, c_int, c_size_t, c_int, c_int, c_int, c_int,
                             ctypes.POINTER(glcm_offset), c_int, c_int, c_void_p, c_void_p]),
    "glcm_histogram": (c_int, [c_void_p, c_void_p, c_int, c_int, c_size_t, c_int, c_int, c_int, c_void_p]),
    "glcm_synchronize": (c_int, [c_void_p]),
    "glcm_set_timing": (c_int, [c_void_p, c_int]),
    "glcm_get_timing": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_longlong),
                                ctypes.POINTER(c_longlong), c_int]),
    "glcm_set_vote_config": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, c_int]),
    "glcm_compute_naive": (c_int, [c_void_p, c_void_p, c_int, c_int, c_size_t, c_int, c_int, glcm_offset,
                                   c_int, c_void_p]),
    "glcm_compute_noalloc": (c_int, [c_void_p, c_int, c_int, c_size_t, c_int, c_int, ctypes.POINTER(glcm_offset),
                                     c_int, c_int, c_void_p, c_void_p, ctypes.c_char_p, c_size_t]),
    "glcm_measure_ceilings": (c_int, [c_int, ctypes.POINTER(glcm_ceilings_t)]),
    "glcm_compute_batch_windows": (c_int, [c_void_p, ctypes.POINTER(glcm_desc), c_int,
                                           ctypes.POINTER(glcm_window_desc), c_int]),
}

_lib = None


def declared_functions() -> list[str]:
    """Names of the functions include/glcm.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(glcm_[a-z_0-9]+)\s*\(", text)
    return sorted(set(n for n in names if n not in ("glcm_offset", "glcm_desc", "glcm_status")))


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libglcm.so; raise if it is missing and cannot be built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"libglcm.so is not built ({_build.LIB}); run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _PROTOS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _offsets(offsets):
    arr = (glcm_offset * len(offsets))()
    for k, (dx, dy) in enumerate(offsets):
        arr[k].dx, arr[k].dy = int(dx), int(dy)
    return arr


def _check(ctx, status: int):
    if status != GLCM_OK:
        msg = load().glcm_last_error(ctx)
        raise GlcmError(status, msg.decode() if msg else "")
    return status


def glcm_create(device: int = 0, hbm_budget_bytes: int = 0, stream=None):
    lib = load()
    out = c_void_p()
    st = lib.glcm_create(ctypes.byref(out), int(device), int(hbm_budget_bytes),
                         None if not stream else int(stream))
    _check(None, st)
    return out


def glcm_destroy(ctx):
    return _check(ctx, load().glcm_destroy(ctx))


def glcm_last_error(ctx) -> str:
    m = load().glcm_last_error(ctx)
    return m.decode() if m else ""


def glcm_offset_from_angle(d: int, theta_deg: int):
    o = glcm_offset()
    _check(None, load().glcm_offset_from_angle(int(d), int(theta_deg), ctypes.byref(o)))
    return (o.dx, o.dy)


def glcm_compute(ctx, image, width, height, pitch_bytes, dtype, levels, offsets, flags, counts,
                 normalized=None):
    offs = _offsets(offsets)
    return _check(ctx, load().glcm_compute(ctx, _ptr(image), int(width), int(height), int(pitch_bytes),
                                           int(dtype), int(levels), offs, len(offsets), int(flags),
                                           _ptr(counts), _ptr(normalized)))


def glcm_features(ctx, counts, levels, n_glcm, flags, features):
    return _check(ctx, load().glcm_features(ctx, _ptr(counts), int(levels), int(n_glcm), int(flags),
                                            _ptr(features)))


def make_desc(image, width, height, pitch_bytes, dtype, levels, offsets, flags, counts, normalized=None,
              features=None):
    """One glcm_desc; keep the returned tuple alive while the batch runs."""
    offs = _offsets(offsets)
    d = glcm_desc(_ptr(image), int(width), int(height), int(pitch_bytes), int(dtype), int(levels),
                  ctypes.cast(offs, ctypes.POINTER(glcm_offset)), len(offsets), int(flags), _ptr(counts),
                  _ptr(normalized), _ptr(features))
    return d, offs


def desc_array(descs):
    """A ctypes glcm_desc array of make_desc results, reusable across calls."""
    return (glcm_desc * len(descs))(*[d[0] if isinstance(d, tuple) else d for d in descs])


def glcm_compute_batch(ctx, descs):
    """descs: make_desc results, or an array from desc_array (reused as is)."""
    arr = descs if isinstance(descs, ctypes.Array) else desc_array(descs)
    return _check(ctx, load().glcm_compute_batch(ctx, arr, len(arr)))


def glcm_enqueue_batch(ctx, descs):
    """Direct (graph-free, unsynchronized) batch launch; device pointers only."""
    arr = (glcm_desc * len(descs))(*[d[0] if isinstance(d, tuple) else d for d in descs])
    return _check(ctx, load().glcm_enqueue_batch(ctx, arr, len(descs)))


def _check_server(server, status: int):
    if status != GLCM_OK:
        msg = load().glcm_server_last_error(server)
        raise GlcmError(status, msg.decode() if msg else "")
    return status


def glcm_server_create(device=0, hbm_budget_bytes=0, lanes=0, max_batch=0, max_queue=0):
    out = c_void_p()
    _check_server(None, load().glcm_server_create(ctypes.byref(out), int(device), int(hbm_budget_bytes),
                                                  int(lanes), int(max_batch), int(max_queue)))
    return out


def glcm_server_submit(server, desc):
    """Queue one request (a make_desc tuple with host pointers); returns its ticket."""
    t = c_longlong()
    d = desc[0] if isinstance(desc, tuple) else desc
    _check_server(server, load().glcm_server_submit(server, ctypes.byref(d), ctypes.byref(t)))
    return t.value


def glcm_server_wait(server, ticket, timeout_ms=-1):
    """(status, latency_ms); status GLCM_ERR_BUSY means still in flight.  A
    failed request's status is returned, not raised."""
    lat = c_double()
    st = load().glcm_server_wait(server, int(ticket), int(timeout_ms), ctypes.byref(lat))
    if st == GLCM_ERR_ARG:
        _check_server(server, st)
    return st, lat.value


def glcm_server_stats(server):
    st = glcm_server_stats_t()
    _check_server(server, load().glcm_server_stats(server, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in st._fields_}


def glcm_server_last_error(server) -> str:
    m = load().glcm_server_last_error(server)
    return m.decode() if m else ""


def glcm_server_destroy(server):
    return load().glcm_server_destroy(server)


def glcm_windows(ctx, image, width, height, pitch_bytes, dtype, levels, win, stride, offsets, flags,
                 counts=None, maps=None):
    offs = _offsets(offsets)
    return _check(ctx, load().glcm_windows(ctx, _ptr(image), int(width), int(height), int(pitch_bytes),
                                           int(dtype), int(levels), int(win), int(stride), offs, len(offsets),
                                           int(flags), _ptr(counts), _ptr(maps)))


def glcm_histogram(ctx, image, width, height, pitch_bytes, dtype, levels, flags, hist):
    return _check(ctx, load().glcm_histogram(ctx, _ptr(image), int(width), int(height), int(pitch_bytes),
                                             int(dtype), int(levels), int(flags), _ptr(hist)))


def glcm_synchronize(ctx):
    return _check(ctx, load().glcm_synchronize(ctx))


def glcm_set_timing(ctx, enable: bool):
    return _check(ctx, load().glcm_set_timing(ctx, int(bool(enable))))


def glcm_get_timing(ctx, reset: bool = False):
    ms, nv, nk = c_double(), c_longlong(), c_longlong()
    _check(ctx, load().glcm_get_timing(ctx, ctypes.byref(ms), ctypes.byref(nv), ctypes.byref(nk), int(reset)))
    return ms.value, nv.value, nk.value


def glcm_set_vote_config(ctx, levels, n_offsets, dtype, threads, log2_copies, layout, band_rows=0):
    return _check(ctx, load().glcm_set_vote_config(ctx, int(levels), int(n_offsets), int(dtype), int(threads),
                                                   int(log2_copies), int(layout), int(band_rows)))


def glcm_compute_naive(ctx, image, width, height, pitch_bytes, dtype, levels, offset, flags, counts):
    o = glcm_offset(int(offset[0]), int(offset[1]))
    return _check(ctx, load().glcm_compute_naive(ctx, _ptr(image), int(width), int(height), int(pitch_bytes),
                                                 int(dtype), int(levels), o, int(flags), _ptr(counts)))


def glcm_compute_noalloc(image, width, height, pitch_bytes, dtype, levels, offsets, flags, counts, stream=None):
    """GLCM counts with no allocation (static device scratch); device pointers only."""
    offs = _offsets(offsets)
    buf = ctypes.create_string_buffer(256)
    st = load().glcm_compute_noalloc(_ptr(image), int(width), int(height), int(pitch_bytes), int(dtype),
                                     int(levels), offs, len(offsets), int(flags), _ptr(counts),
                                     None if not stream else int(stream), buf, 256)
    if st != GLCM_OK:
        raise GlcmError(st, buf.value.decode())
    return st


def glcm_measure_ceilings(device: int = 0) -> dict:
    """Measured shared-reduction and HBM-read ceilings of a device (see glcm.h)."""
    out = glcm_ceilings_t()
    st = load().glcm_measure_ceilings(int(device), ctypes.byref(out))
    if st != GLCM_OK:
        raise GlcmError(st, "glcm_measure_ceilings failed")
    return {k: getattr(out, k) for k, _ in glcm_ceilings_t._fields_}


def make_window_desc(image, width, height, pitch_bytes, dtype, levels, win, stride, offsets, flags, counts, maps):
    """A glcm_window_desc (keeps its offsets array alive on the struct)."""
    d = glcm_window_desc()
    offs = _offsets(offsets)
    d.image, d.width, d.height, d.pitch_bytes = _ptr(image), int(width), int(height), int(pitch_bytes)
    d.dtype, d.levels, d.win, d.stride = int(dtype), int(levels), int(win), int(stride)
    d.offsets, d.n_offsets, d.flags = offs, len(offsets), int(flags)
    d.counts, d.maps = _ptr(counts), _ptr(maps)
    d._keep = offs
    return d


def glcm_compute_batch_windows(ctx, descs, wins):
    """One graph launch of a batch of images (make_desc results or a desc_array)
    and sliding-window jobs (make_window_desc results), device buffers only."""
    if isinstance(descs, ctypes.Array):
        da, n = descs, len(descs)
    else:
        n = len(descs)
        da = desc_array(descs) if n else (glcm_desc * 1)()
    wa = (glcm_window_desc * max(1, len(wins)))(*wins) if wins else (glcm_window_desc * 1)()
    return _check(ctx, load().glcm_compute_batch_windows(ctx, da, n, wa, len(wins)))
