"""FP64 CPU oracle for the relativistic line-of-sight sum -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it and
shares no code with it; see ``oracle.c`` for what is computed and which
passage of the paper each step follows.

The C source is compiled on first use (``build()``) with gcc, optimisation
level 2, no fast-math and no floating-point contraction, into
``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_F64, ORC_F32 = 0, 1


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("origin", ctypes.c_double * 3), ("dx", ctypes.c_double * 3),
                ("n_epochs", ctypes.c_int32), ("t0", ctypes.c_double), ("dt", ctypes.c_double)]


class _Fields(ctypes.Structure):
    _fields_ = [("j", ctypes.c_void_p), ("beta", ctypes.c_void_p), ("dtype", ctypes.c_int32)]


class _View(ctypes.Structure):
    _fields_ = [("dir", ctypes.c_double * 3), ("up", ctypes.c_double * 3), ("center", ctypes.c_double * 3),
                ("t_obs", ctypes.c_double), ("c", ctypes.c_double), ("alpha", ctypes.c_double),
                ("nu_ratio", ctypes.c_double), ("beaming", ctypes.c_int32), ("lookback", ctypes.c_int32),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fov_u", ctypes.c_double),
                ("fov_v", ctypes.c_double), ("split_at_nodes", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into a shared library; returns its path."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        ptr = ctypes.POINTER
        lib.orc_render.argtypes = [ptr(_Grid), ptr(_Fields), ptr(_View), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_int32]
        lib.orc_render.restype = ctypes.c_int
        lib.orc_render_pixels.argtypes = [ptr(_Grid), ptr(_Fields), ptr(_View), ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        lib.orc_render_pixels.restype = ctypes.c_int
        lib.orc_max_threads.restype = ctypes.c_int32
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().orc_max_threads())


def _grid(g) -> _Grid:
    out = _Grid()
    out.n[:] = [int(v) for v in g.n]
    out.origin[:] = [float(v) for v in g.origin]
    out.dx[:] = [float(v) for v in g.dx]
    out.n_epochs = int(g.n_epochs)
    out.t0 = float(g.t0)
    out.dt = float(g.dt)
    return out


def _view(v, split_at_nodes: bool) -> _View:
    out = _View()
    out.dir[:] = [float(x) for x in v.dir]
    out.up[:] = [float(x) for x in v.up]
    out.center[:] = [float(x) for x in v.center]
    out.t_obs = float(v.t_obs)
    out.c = float(v.c)
    out.alpha = float(v.alpha)
    out.nu_ratio = float(v.nu_ratio)
    out.beaming = int(bool(v.beaming))
    out.lookback = int(bool(v.lookback))
    out.width = int(v.width)
    out.height = int(v.height)
    out.fov_u = float(v.fov_u)
    out.fov_v = float(v.fov_v)
    out.split_at_nodes = int(bool(split_at_nodes))
    return out


def _fields(grid, j, beta):
    nx, ny, nz = (int(v) for v in grid.n)
    M = int(grid.n_epochs)
    dtype = j.dtype
    if dtype not in (np.float64, np.float32):
        raise TypeError("oracle fields must be float64 or float32")
    j = np.ascontiguousarray(j).reshape(M, nz, ny, nx)
    if beta is None:
        beta = np.zeros((M, nz, ny, nx, 3), dtype=dtype)
    beta = np.ascontiguousarray(beta, dtype=dtype).reshape(M, nz, ny, nx, 3)
    f = _Fields()
    f.j = j.ctypes.data
    f.beta = beta.ctypes.data
    f.dtype = ORC_F64 if dtype == np.float64 else ORC_F32
    return f, (j, beta)


def render(grid, j, beta, view, *, threads: int = 0, counts: bool = False, split_at_nodes: bool = False):
    """Image ``[height][width]`` (float64) of one view; with ``counts`` also
    the per-pixel number of cell-samples (int64)."""
    lib = _load()
    f, keep = _fields(grid, j, beta)
    img = np.zeros((int(view.height), int(view.width)), dtype=np.float64)
    cnt = np.zeros(img.shape, dtype=np.int64) if counts else None
    g, v = _grid(grid), _view(view, split_at_nodes)
    rc = lib.orc_render(ctypes.byref(g), ctypes.byref(f), ctypes.byref(v), img.ctypes.data,
                        cnt.ctypes.data if cnt is not None else None, int(threads))
    del keep
    if rc != 0:
        raise ValueError(f"oracle rejected the input (code {rc})")
    return (img, cnt) if counts else img


def render_pixels(grid, j, beta, view, pixels, *, threads: int = 0, counts: bool = False,
                  split_at_nodes: bool = False):
    """Values of the pixels listed as rows (p, q) of ``pixels``."""
    lib = _load()
    f, keep = _fields(grid, j, beta)
    pq = np.ascontiguousarray(np.asarray(pixels, dtype=np.int32).reshape(-1, 2))
    out = np.zeros(pq.shape[0], dtype=np.float64)
    cnt = np.zeros(pq.shape[0], dtype=np.int64) if counts else None
    g, v = _grid(grid), _view(view, split_at_nodes)
    rc = lib.orc_render_pixels(ctypes.byref(g), ctypes.byref(f), ctypes.byref(v), pq.ctypes.data,
                               int(pq.shape[0]), out.ctypes.data,
                               cnt.ctypes.data if cnt is not None else None, int(threads))
    del keep
    if rc != 0:
        raise ValueError(f"oracle rejected the input (code {rc})")
    return (out, cnt) if counts else out


def pixel_area(view) -> float:
    """Area of one pixel on the image plane (for flux = area * sum(I))."""
    return (float(view.fov_u) / int(view.width)) * (float(view.fov_v) / int(view.height))


__all__ = ["build", "render", "render_pixels", "pixel_area", "max_threads", "ORC_F64", "ORC_F32", "math"]
