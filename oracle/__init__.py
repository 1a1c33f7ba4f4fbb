"""CPU oracle for the GLCM library -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg (``bench.py``'s ``cpu_baseline`` and ``--impl reference``) may import
this package.  The CUDA product path never imports, links or calls it, and
the two share no code: the oracle is plain C loops (``glcm_oracle.c``) for
the counts of Eq. (1) and plain numpy in float64 (``haralick.py``) for the
symmetrize/normalize epilogue and the 14 Haralick features.

Functions
---------
``glcm(img, levels, offsets, levels_mode=False)``
    uint32 counts, shape (n_offsets, N, N), row-major [i][j] with i the
    anchor level (Eq. 1, partner by Eq. 2, bin by Eq. 3 with the anchor as
    the row).
``glcm_flat(img, levels, offsets, levels_mode=False)``
    the same counts with Eq. 2 read literally on the row-major buffer: pixel
    p = y W + x pairs with p + dy W + dx whenever that index is in [0, W H),
    so pairs may run across row ends (the flat-wrap mode).
``window_glcm(img, levels, offsets, win, stride, windows)``
    local GLCMs of win x win windows (pairs with both pixels inside).
``histogram(img, levels, levels_mode=False)``
    uint32 pixels per level, shape (N,) (the one-pixel statistic, Sec. I).
``symmetrize_normalize`` / ``haralick`` / ``window_maps``
    float64 epilogue and features, see ``haralick.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .haralick import (FEATURE_NAMES, haralick, haralick_batch, normalize, symmetrize,
                       window_maps)  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glcm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc -O2 (no SIMD intrinsics) into _build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64 = ctypes.c_longlong
            vp = ctypes.c_void_p
            ci = ctypes.c_int
            sz = ctypes.c_size_t
            lib.oracle_glcm.restype = i64
            lib.oracle_glcm.argtypes = [vp, ci, ci, sz, ci, ci, ci, ci, ci, vp]
            lib.oracle_glcm_multi.restype = i64
            lib.oracle_glcm_multi.argtypes = [vp, ci, ci, sz, ci, ci, ci, ci, vp, vp]
            lib.oracle_glcm_flat_multi.restype = i64
            lib.oracle_glcm_flat_multi.argtypes = [vp, ci, ci, sz, ci, ci, ci, ci, vp, vp]
            lib.oracle_window_glcm.restype = i64
            lib.oracle_window_glcm.argtypes = [vp, ci, ci, sz, ci, ci, ci, ci, ci, ci, vp, ci, vp, vp, vp]
            lib.oracle_histogram.restype = i64
            lib.oracle_histogram.argtypes = [vp, ci, ci, sz, ci, ci, ci, vp]
            _lib = lib
    return _lib


def _img_args(img: np.ndarray):
    if img.ndim != 2 or img.dtype not in (np.uint8, np.uint16):
        raise ValueError("image must be a 2-D uint8 or uint16 array")
    if img.strides[1] != img.itemsize:
        img = np.ascontiguousarray(img)
    return img, img.shape[1], img.shape[0], img.strides[0], img.itemsize


def glcm(img: np.ndarray, levels: int, offsets, levels_mode: bool = False, return_skipped: bool = False):
    """Counts of Eq. (1) for each (dx, dy) in ``offsets``: (n_off, N, N) uint32."""
    lib = _load()
    img, w, h, pitch, bpp = _img_args(img)
    offs = np.asarray(offsets, dtype=np.int32).reshape(-1, 2)
    out = np.zeros((len(offs), levels, levels), dtype=np.uint32)
    dxy = np.ascontiguousarray(offs.reshape(-1))
    s = lib.oracle_glcm_multi(img.ctypes.data, w, h, pitch, bpp, levels, int(levels_mode),
                              len(offs), dxy.ctypes.data, out.ctypes.data)
    if s < 0:
        raise ValueError("oracle_glcm_multi: bad arguments")
    return (out, int(s)) if return_skipped else out


def glcm_flat(img: np.ndarray, levels: int, offsets, levels_mode: bool = False, return_skipped: bool = False):
    """Flat-wrap counts (Eq. 2 on the row-major buffer): (n_off, N, N) uint32."""
    lib = _load()
    img, w, h, pitch, bpp = _img_args(img)
    offs = np.asarray(offsets, dtype=np.int32).reshape(-1, 2)
    out = np.zeros((len(offs), levels, levels), dtype=np.uint32)
    dxy = np.ascontiguousarray(offs.reshape(-1))
    s = lib.oracle_glcm_flat_multi(img.ctypes.data, w, h, pitch, bpp, levels, int(levels_mode),
                                   len(offs), dxy.ctypes.data, out.ctypes.data)
    if s < 0:
        raise ValueError("oracle_glcm_flat_multi: bad arguments")
    return (out, int(s)) if return_skipped else out


def window_glcm(img: np.ndarray, levels: int, offsets, win: int, stride: int, windows=None,
                levels_mode: bool = False):
    """Local GLCMs of win x win windows at (wx*stride, wy*stride).

    ``windows`` is an array of (wy, wx) window indices; None means every
    window that fits inside the image, in row-major (wy, wx) order.
    Returns (n_win, n_off, N, N) uint32."""
    lib = _load()
    img, w, h, pitch, bpp = _img_args(img)
    if windows is None:
        nwy = (h - win) // stride + 1 if h >= win else 0
        nwx = (w - win) // stride + 1 if w >= win else 0
        gy, gx = np.meshgrid(np.arange(nwy), np.arange(nwx), indexing="ij")
        windows = np.stack([gy.reshape(-1), gx.reshape(-1)], axis=1)
    windows = np.asarray(windows, dtype=np.int32).reshape(-1, 2)
    wy = np.ascontiguousarray(windows[:, 0])
    wx = np.ascontiguousarray(windows[:, 1])
    offs = np.asarray(offsets, dtype=np.int32).reshape(-1, 2)
    dxy = np.ascontiguousarray(offs.reshape(-1))
    out = np.zeros((len(windows), len(offs), levels, levels), dtype=np.uint32)
    s = lib.oracle_window_glcm(img.ctypes.data, w, h, pitch, bpp, levels, int(levels_mode), win,
                               stride, len(offs), dxy.ctypes.data, len(windows), wx.ctypes.data,
                               wy.ctypes.data, out.ctypes.data)
    if s < 0:
        raise ValueError("oracle_window_glcm: bad arguments or window outside the image")
    return out


def histogram(img: np.ndarray, levels: int, levels_mode: bool = False, return_skipped: bool = False):
    """Pixels per level over the whole image: (N,) uint32."""
    lib = _load()
    img, w, h, pitch, bpp = _img_args(img)
    out = np.zeros(levels, dtype=np.uint32)
    s = lib.oracle_histogram(img.ctypes.data, w, h, pitch, bpp, levels, int(levels_mode), out.ctypes.data)
    if s < 0:
        raise ValueError("oracle_histogram: bad arguments")
    return (out, int(s)) if return_skipped else out


def pair_count(w: int, h: int, dx: int, dy: int) -> int:
    """Number of in-bounds anchor/partner pairs (closed form)."""
    return max(0, w - abs(dx)) * max(0, h - abs(dy))
