"""Python binding of the gbdart C ABI (include/gbdart.h).

Argument marshalling only: every step of a render runs in the CUDA kernels of
the shared library.  PyTorch provides device memory (output tensors) and
streams.  If the compiled library is missing the import fails loudly; there
is no fallback implementation.

Views are any objects with the attributes ``dir, up, center, t_obs, c,
alpha, nu_ratio, beaming, lookback, width, height, fov_u, fov_v``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK, ERR_INVALID, ERR_NOMEM, ERR_BUDGET, ERR_NOTFOUND, ERR_TIMEOUT, ERR_CUDA, ERR_CANCELLED, ERR_BUSY = range(9)
IN_F64, IN_F32 = 0, 1
STORE_F32, STORE_BF16_F16U = 0, 1
BEAMING, LOOKBACK = 1, 2

_STORES = {"f32": STORE_F32, "bf16": STORE_BF16_F16U, STORE_F32: STORE_F32, STORE_BF16_F16U: STORE_BF16_F16U}


class GbdError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"gbdart error {code}: {message}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("origin", ctypes.c_double * 3), ("dx", ctypes.c_double * 3),
                ("n_epochs", ctypes.c_int32), ("t0", ctypes.c_double), ("dt", ctypes.c_double)]


class Fields(ctypes.Structure):
    _fields_ = [("j", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("dtype_in", ctypes.c_int32),
                ("store", ctypes.c_int32), ("on_device", ctypes.c_int32), ("brick", ctypes.c_int32),
                ("super_brick", ctypes.c_int32), ("paired", ctypes.c_int32), ("morton_cells", ctypes.c_int32)]


class StreamInfo(ctypes.Structure):
    _fields_ = [("slab", ctypes.c_int32), ("flexload", ctypes.c_int32), ("slabs", ctypes.c_int32),
                ("bytes_uploaded", ctypes.c_uint64), ("bytes_total", ctypes.c_uint64)]


class CView(ctypes.Structure):
    _fields_ = [("dir", ctypes.c_double * 3), ("up", ctypes.c_double * 3), ("center", ctypes.c_double * 3),
                ("t_obs", ctypes.c_double), ("c", ctypes.c_double), ("alpha", ctypes.c_double),
                ("nu_ratio", ctypes.c_double), ("flags", ctypes.c_uint32)]


class ImageSpec(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fov_u", ctypes.c_double),
                ("fov_v", ctypes.c_double), ("out", ctypes.c_void_p), ("samples", ctypes.c_void_p),
                ("out_on_host", ctypes.c_int32)]


class Launch(ctypes.Structure):
    _fields_ = [("packet_w", ctypes.c_int32), ("packet_h", ctypes.c_int32), ("cta_warps", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("persistent", ctypes.c_int32), ("regcap", ctypes.c_int32),
                ("region", ctypes.c_int32), ("group", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("launch", Launch), ("brick", ctypes.c_int32), ("super_brick", ctypes.c_int32),
                ("paired", ctypes.c_int32), ("morton_cells", ctypes.c_int32), ("ms", ctypes.c_float),
                ("candidates", ctypes.c_int32)]


TUNE_LAUNCH, TUNE_LAYOUT = 1, 2


class Request(ctypes.Structure):
    _fields_ = [("volume", ctypes.c_uint64), ("view", CView), ("spec", ImageSpec), ("priority", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("device_ms", ctypes.c_double)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("max_waves", ctypes.c_int32), ("max_requests_per_wave", ctypes.c_int32),
                ("max_requests_in_flight", ctypes.c_int32), ("request_budget_bytes", ctypes.c_uint64),
                ("launch", Launch)]


class ServeSummary(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("requests_per_s", ctypes.c_double), ("waves", ctypes.c_uint64),
                ("mean_requests_per_wave", ctypes.c_double), ("max_waves_in_flight", ctypes.c_int32),
                ("pending", ctypes.c_int32), ("in_flight", ctypes.c_int32)]


class VolumeDesc(ctypes.Structure):
    _fields_ = [("grid", Grid), ("store", ctypes.c_int32), ("brick", ctypes.c_int32),
                ("super_brick", ctypes.c_int32), ("paired", ctypes.c_int32), ("morton_cells", ctypes.c_int32),
                ("bytes", ctypes.c_uint64),
                ("record_bytes", ctypes.c_uint64), ("n_channels", ctypes.c_int32), ("channel_bytes", ctypes.c_uint64)]


_lock = threading.Lock()
_libs: dict[bool, ctypes.CDLL] = {}

_SIGNATURES = {
    "gbd_error_string": ([ctypes.c_int], ctypes.c_char_p),
    "gbd_last_error": ([], ctypes.c_char_p),
    "gbd_last_launch_count": ([], ctypes.c_int32),
    "gbd_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_uint64], ctypes.c_int),
    "gbd_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "gbd_load_snapshots": ([ctypes.c_void_p, ctypes.POINTER(Grid), ctypes.POINTER(Fields),
                            ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "gbd_unload": ([ctypes.c_void_p, ctypes.c_uint64], ctypes.c_int),
    "gbd_volume_info": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(VolumeDesc)], ctypes.c_int),
    "gbd_render": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(CView), ctypes.POINTER(ImageSpec),
                    ctypes.POINTER(Launch), ctypes.c_void_p], ctypes.c_int),
    "gbd_bounds_violations": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "gbd_render_batch_noalloc": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(CView), ctypes.c_int32,
                                  ctypes.POINTER(ImageSpec), ctypes.POINTER(Launch), ctypes.c_void_p], ctypes.c_int),
    "gbd_render_streamed": ([ctypes.c_void_p, ctypes.POINTER(Grid), ctypes.POINTER(Fields), ctypes.POINTER(CView),
                             ctypes.c_int32, ctypes.POINTER(ImageSpec), ctypes.POINTER(Launch),
                             ctypes.POINTER(StreamInfo), ctypes.c_void_p], ctypes.c_int),
    "gbd_render_labelled": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32, ctypes.POINTER(CView),
                             ctypes.c_int32, ctypes.POINTER(ImageSpec), ctypes.POINTER(Launch), ctypes.c_void_p],
                            ctypes.c_int),
    "gbd_load_channels": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                           ctypes.c_int32], ctypes.c_int),
    "gbd_render_vector": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(CView), ctypes.c_int32,
                           ctypes.POINTER(ImageSpec), ctypes.POINTER(Launch), ctypes.c_void_p], ctypes.c_int),
    "gbd_touched_records": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(CView), ctypes.c_int32,
                             ctypes.POINTER(ImageSpec), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "gbd_serve_start": ([ctypes.c_void_p, ctypes.POINTER(ServeConfig)], ctypes.c_int),
    "gbd_serve_stop": ([ctypes.c_void_p], ctypes.c_int),
    "gbd_submit": ([ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "gbd_poll": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(Stats)],
                 ctypes.c_int),
    "gbd_wait": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(Stats)], ctypes.c_int),
    "gbd_cancel": ([ctypes.c_void_p, ctypes.c_uint64], ctypes.c_int),
    "gbd_serve_stats": ([ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ServeSummary)], ctypes.c_int),
    "gbd_tune": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(CView), ctypes.c_int32,
                  ctypes.POINTER(ImageSpec), ctypes.c_uint32, ctypes.c_void_p, ctypes.POINTER(TuneResult)],
                 ctypes.c_int),
    "gbd_relayout": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                      ctypes.c_int32], ctypes.c_int),
    "gbd_render_batch": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(CView), ctypes.c_int32,
                          ctypes.POINTER(ImageSpec), ctypes.POINTER(Launch), ctypes.c_void_p], ctypes.c_int),
}


def load_library(checked: bool = False, build_if_missing: bool = True) -> ctypes.CDLL:
    """The compiled library (built in-tree by ``build.build`` if absent)."""
    with _lock:
        if checked in _libs:
            return _libs[checked]
        path = _build.lib_path(checked)
        if not os.path.exists(path):
            if not build_if_missing:
                raise ImportError(f"gbdart library not built: {path}")
            _build.build(checked=checked)
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _libs[checked] = lib
        return lib


def declared_symbols() -> list[str]:
    return list(_SIGNATURES)


def _check(lib, rc: int):
    if rc != OK:
        raise GbdError(rc, lib.gbd_last_error().decode(errors="replace"))


def _cview(v) -> CView:
    out = CView()
    out.dir[:] = [float(x) for x in v.dir]
    out.up[:] = [float(x) for x in v.up]
    out.center[:] = [float(x) for x in v.center]
    out.t_obs = float(v.t_obs)
    out.c = float(v.c)
    out.alpha = float(v.alpha)
    out.nu_ratio = float(v.nu_ratio)
    out.flags = (BEAMING if v.beaming else 0) | (LOOKBACK if v.lookback else 0)
    return out


def _launch(launch) -> ctypes.POINTER(Launch) | None:
    if launch is None:
        return None
    if isinstance(launch, Launch):
        return ctypes.pointer(launch)
    lw = Launch()
    lw.packet_w, lw.packet_h = launch.get("packet", (0, 0))
    lw.cta_warps = launch.get("cta_warps", 0)
    lw.depth = launch.get("depth", 0)
    lw.persistent = int(launch.get("persistent", 1))
    lw.regcap = int(launch.get("regcap", 0))
    lw.region = int(launch.get("region", 0))
    lw.group = int(launch.get("group", 0))
    return ctypes.pointer(lw)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """A gbdart context on one CUDA device."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, checked: bool = False):
        self.lib = load_library(checked)
        self.device = device
        h = ctypes.c_void_p()
        _check(self.lib, self.lib.gbd_create(ctypes.byref(h), int(device), int(budget_bytes)))
        self.handle = h

    # -- lifetime
    def close(self):
        if self.handle:
            self.lib.gbd_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- volumes
    def load_snapshots(self, grid, j, beta, *, store="f32", brick: int = 0, super_brick: int = 0,
                       paired: bool = False, morton_cells: bool = False) -> int:
        """Pack snapshots j[M][nz][ny][nx] and beta[M][nz][ny][nx][3] (numpy
        arrays or torch tensors, float64 or float32) into a resident volume."""
        import torch
        g = Grid()
        g.n[:] = [int(x) for x in grid.n]
        g.origin[:] = [float(x) for x in grid.origin]
        g.dx[:] = [float(x) for x in grid.dx]
        g.n_epochs = int(grid.n_epochs)
        g.t0 = float(grid.t0)
        g.dt = float(grid.dt)
        keep = []
        on_device = isinstance(j, torch.Tensor) and j.is_cuda
        if on_device:
            jj = j.contiguous()
            bb = beta.contiguous().to(jj.dtype)
            if jj.dtype not in (torch.float64, torch.float32):
                raise TypeError("fields must be float64 or float32")
            dtype_in = IN_F64 if jj.dtype == torch.float64 else IN_F32
            jp, bp = jj.data_ptr(), bb.data_ptr()
            keep += [jj, bb]
        else:
            jj = j.cpu().numpy() if isinstance(j, torch.Tensor) else np.asarray(j)
            bb = beta.cpu().numpy() if isinstance(beta, torch.Tensor) else np.asarray(beta)
            if jj.dtype not in (np.float64, np.float32):
                raise TypeError("fields must be float64 or float32")
            jj = np.ascontiguousarray(jj)
            bb = np.ascontiguousarray(bb, dtype=jj.dtype)
            dtype_in = IN_F64 if jj.dtype == np.float64 else IN_F32
            jp, bp = jj.ctypes.data, bb.ctypes.data
            keep += [jj, bb]
        M, nz, ny, nx = int(grid.n_epochs), int(grid.n[2]), int(grid.n[1]), int(grid.n[0])
        if tuple(jj.shape) != (M, nz, ny, nx) or tuple(bb.shape) != (M, nz, ny, nx, 3):
            raise ValueError(f"field shapes {tuple(jj.shape)}, {tuple(bb.shape)} do not match the grid")
        f = Fields()
        f.j, f.vel = jp, bp
        f.dtype_in = dtype_in
        f.store = _STORES[store]
        f.on_device = int(on_device)
        f.brick = int(brick)
        f.super_brick = int(super_brick)
        f.paired = int(bool(paired))
        f.morton_cells = int(bool(morton_cells))
        vid = ctypes.c_uint64()
        rc = self.lib.gbd_load_snapshots(self.handle, ctypes.byref(g), ctypes.byref(f), ctypes.byref(vid))
        del keep
        _check(self.lib, rc)
        return int(vid.value)

    def touched_records(self, vol: int, views) -> int:
        """Distinct (cell, snapshot) records a batch render of ``views`` reads."""
        views = list(views)
        arr = (CView * len(views))(*[_cview(v) for v in views])
        spec = self._spec(views[0], None, None)
        out = ctypes.c_uint64()
        _check(self.lib, self.lib.gbd_touched_records(self.handle, int(vol), arr, len(views), ctypes.byref(spec),
                                                      ctypes.byref(out)))
        return int(out.value)

    def load_channels(self, vol: int, channels):
        """Attach extra emissivity channels [K][M][nz][ny][nx] (K = 1 or 3;
        numpy or torch, float32 or float64) to a volume for vector renders."""
        import torch
        if isinstance(channels, torch.Tensor) and channels.is_cuda:
            cc = channels.contiguous()
            if cc.dtype not in (torch.float64, torch.float32):
                raise TypeError("channels must be float64 or float32")
            dtype_in, ptr, on_device = (IN_F64 if cc.dtype == torch.float64 else IN_F32), cc.data_ptr(), 1
        else:
            cc = np.ascontiguousarray(channels.cpu().numpy() if isinstance(channels, torch.Tensor) else channels)
            if cc.dtype not in (np.float64, np.float32):
                raise TypeError("channels must be float64 or float32")
            dtype_in, ptr, on_device = (IN_F64 if cc.dtype == np.float64 else IN_F32), cc.ctypes.data, 0
        info = self.volume_info(vol)
        want = (int(info["n_epochs"]), int(info["n"][2]), int(info["n"][1]), int(info["n"][0]))
        if cc.ndim != 5 or tuple(cc.shape[1:]) != want:
            raise ValueError(f"channels must be [K]{list(want)}, got {tuple(cc.shape)}")
        _check(self.lib, self.lib.gbd_load_channels(self.handle, int(vol), ptr, int(cc.shape[0]), dtype_in, on_device))

    def render_vector(self, vol: int, views, *, out=None, launch=None, stream=None):
        """Images [n][1 + K][H][W]: component 0 of j', components 1.. of the
        volume's extra channels, all marched along each ray at once."""
        import torch
        views = list(views)
        v0 = views[0]
        k = int(self.volume_info(vol).get("channels", 0))
        if out is None:
            out = torch.empty((len(views), 1 + k, int(v0.height), int(v0.width)), dtype=torch.float32,
                              device=torch.device("cuda", self.device))
        arr = (CView * len(views))(*[_cview(v) for v in views])
        spec = self._spec(v0, out.data_ptr(), None)
        rc = self.lib.gbd_render_vector(self.handle, int(vol), arr, len(views), ctypes.byref(spec), _launch(launch),
                                        _stream_handle(stream))
        _check(self.lib, rc)
        return out

    def render_labelled(self, vols, views, *, out=None, samples: bool = False, launch=None, stream=None):
        """Images [n][H][W] of ``views`` over a scene of several resident
        volumes (non-overlapping sub-domains, each with its own grid): the
        sum of each ray's sums through every sub-domain."""
        import torch
        views = list(views)
        v0 = views[0]
        dev = torch.device("cuda", self.device)
        shape = (len(views), int(v0.height), int(v0.width))
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=dev)
        cnt = torch.empty(shape, dtype=torch.int32, device=dev) if samples else None
        ids = (ctypes.c_uint64 * len(vols))(*[int(v) for v in vols])
        arr = (CView * len(views))(*[_cview(v) for v in views])
        spec = self._spec(v0, out.data_ptr(), cnt.data_ptr() if cnt is not None else None)
        rc = self.lib.gbd_render_labelled(self.handle, ids, len(vols), arr, len(views), ctypes.byref(spec),
                                          _launch(launch), _stream_handle(stream))
        _check(self.lib, rc)
        return (out, cnt) if samples else out

    def render_streamed(self, grid, j, beta, views, *, out=None, store="f32", slab: int = 0, flexload: bool = True,
                        launch=None, stream=None, brick: int = 0, super_brick: int = 0):
        """Images [n][H][W] of ``views`` rendered from host-resident fields
        j[M][nz][ny][nx], beta[M][nz][ny][nx][3] (numpy, float32 or float64)
        slab by slab along z, uploading with ``flexload`` only the snapshots
        each slab's rays can reach.  Returns (images, info) with info the
        slab and upload counts."""
        import torch
        views = list(views)
        v0 = views[0]
        g = Grid()
        g.n[:] = [int(x) for x in grid.n]
        g.origin[:] = [float(x) for x in grid.origin]
        g.dx[:] = [float(x) for x in grid.dx]
        g.n_epochs = int(grid.n_epochs)
        g.t0 = float(grid.t0)
        g.dt = float(grid.dt)
        jj = np.ascontiguousarray(j.cpu().numpy() if isinstance(j, torch.Tensor) else j)
        if jj.dtype not in (np.float64, np.float32):
            raise TypeError("fields must be float64 or float32")
        bb = np.ascontiguousarray(beta.cpu().numpy() if isinstance(beta, torch.Tensor) else beta, dtype=jj.dtype)
        M, nz, ny, nx = int(grid.n_epochs), int(grid.n[2]), int(grid.n[1]), int(grid.n[0])
        if tuple(jj.shape) != (M, nz, ny, nx) or tuple(bb.shape) != (M, nz, ny, nx, 3):
            raise ValueError(f"field shapes {tuple(jj.shape)}, {tuple(bb.shape)} do not match the grid")
        f = Fields()
        f.j, f.vel = jj.ctypes.data, bb.ctypes.data
        f.dtype_in = IN_F64 if jj.dtype == np.float64 else IN_F32
        f.store = _STORES[store]
        f.on_device = 0
        f.brick = int(brick)
        f.super_brick = int(super_brick)
        dev = torch.device("cuda", self.device)
        if out is None:
            out = torch.empty((len(views), int(v0.height), int(v0.width)), dtype=torch.float32, device=dev)
        arr = (CView * len(views))(*[_cview(v) for v in views])
        spec = self._spec(v0, out.data_ptr(), None)
        info = StreamInfo()
        info.slab = int(slab)
        info.flexload = int(bool(flexload))
        rc = self.lib.gbd_render_streamed(self.handle, ctypes.byref(g), ctypes.byref(f), arr, len(views),
                                          ctypes.byref(spec), _launch(launch), ctypes.byref(info),
                                          _stream_handle(stream))
        _check(self.lib, rc)
        return out, dict(slabs=info.slabs, bytes_uploaded=info.bytes_uploaded, bytes_total=info.bytes_total)

    def unload(self, vol: int):
        _check(self.lib, self.lib.gbd_unload(self.handle, int(vol)))

    def volume_info(self, vol: int) -> dict:
        d = VolumeDesc()
        _check(self.lib, self.lib.gbd_volume_info(self.handle, int(vol), ctypes.byref(d)))
        return dict(n=tuple(d.grid.n), n_epochs=d.grid.n_epochs, store=d.store, brick=d.brick,
                    super_brick=d.super_brick, paired=d.paired, morton_cells=d.morton_cells, bytes=int(d.bytes),
                    record_bytes=int(d.record_bytes), channels=int(d.n_channels), channel_bytes=int(d.channel_bytes))

    # -- rendering
    def _spec(self, view, out_ptr, samples_ptr, on_host=False) -> ImageSpec:
        s = ImageSpec()
        s.width, s.height = int(view.width), int(view.height)
        s.fov_u, s.fov_v = float(view.fov_u), float(view.fov_v)
        s.out = out_ptr
        s.samples = samples_ptr
        s.out_on_host = int(on_host)
        return s

    def render(self, vol: int, view, *, out=None, samples: bool = False, launch=None, stream=None):
        """Image [height][width] (float32 device tensor); with ``samples`` also
        the per-pixel cell-sample counts (int32 tensor, values are uint32)."""
        import torch
        dev = torch.device("cuda", self.device)
        if out is None:
            out = torch.empty((int(view.height), int(view.width)), dtype=torch.float32, device=dev)
        cnt = torch.empty(out.shape, dtype=torch.int32, device=dev) if samples else None
        spec = self._spec(view, out.data_ptr(), cnt.data_ptr() if cnt is not None else None)
        cv = _cview(view)
        rc = self.lib.gbd_render(self.handle, int(vol), ctypes.byref(cv), ctypes.byref(spec), _launch(launch),
                                 _stream_handle(stream))
        _check(self.lib, rc)
        return (out, cnt) if samples else out

    def render_batch(self, vol: int, views, *, out=None, samples: bool = False, launch=None, stream=None):
        """Images [n][height][width] of views sharing one image geometry, in
        one call (up to 128 views per kernel launch, replayed from a cached
        CUDA graph)."""
        import torch
        views = list(views)
        v0 = views[0]
        for v in views[1:]:
            if (v.width, v.height, v.fov_u, v.fov_v) != (v0.width, v0.height, v0.fov_u, v0.fov_v):
                raise ValueError("render_batch needs one image geometry for all views")
        dev = torch.device("cuda", self.device)
        shape = (len(views), int(v0.height), int(v0.width))
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=dev)
        cnt = torch.empty(shape, dtype=torch.int32, device=dev) if samples else None
        arr = (CView * len(views))(*[_cview(v) for v in views])
        spec = self._spec(v0, out.data_ptr(), cnt.data_ptr() if cnt is not None else None)
        rc = self.lib.gbd_render_batch(self.handle, int(vol), arr, len(views), ctypes.byref(spec), _launch(launch),
                                       _stream_handle(stream))
        _check(self.lib, rc)
        return (out, cnt) if samples else out

    def render_batch_noalloc(self, vol: int, views, out, *, launch=None, stream=None):
        """``render_batch`` into the caller's device tensor ``out`` [n][H][W]
        without any allocation by the library (its scratch is a fixed
        device array; at most 1024 views per call).  ``out`` must be a
        contiguous float32 tensor of shape [n][H][W] on this context's device:
        the library writes n * H * W floats from its first element."""
        import torch
        views = list(views)
        if not views:
            raise ValueError("render_batch_noalloc needs at least one view")
        v0 = views[0]
        for v in views[1:]:
            if (v.width, v.height, v.fov_u, v.fov_v) != (v0.width, v0.height, v0.fov_u, v0.fov_v):
                raise ValueError("render_batch_noalloc needs one image geometry for all views")
        shape = (len(views), int(v0.height), int(v0.width))
        if not isinstance(out, torch.Tensor) or out.dtype != torch.float32 or not out.is_contiguous():
            raise ValueError("render_batch_noalloc writes into a contiguous float32 torch tensor")
        if out.device != torch.device("cuda", self.device):
            raise ValueError(f"out must be on cuda:{self.device}, not {out.device}")
        if tuple(out.shape) != shape:
            raise ValueError(f"out must have shape {shape}, not {tuple(out.shape)}")
        arr = (CView * len(views))(*[_cview(v) for v in views])
        spec = self._spec(views[0], out.data_ptr(), None)
        rc = self.lib.gbd_render_batch_noalloc(self.handle, int(vol), arr, len(views), ctypes.byref(spec),
                                               _launch(launch), _stream_handle(stream))
        _check(self.lib, rc)
        return out

    def render_batch_host(self, vol: int, views, out_host, *, launch=None, stream=None):
        """Like ``render_batch`` but the images land in ``out_host``, a host
        (preferably pinned) float32 tensor or array of shape [n][H][W]; the
        device-to-host copy is enqueued on the stream."""
        views = list(views)
        v0 = views[0]
        ptr = out_host.data_ptr() if hasattr(out_host, "data_ptr") else out_host.ctypes.data
        arr = (CView * len(views))(*[_cview(v) for v in views])
        spec = self._spec(v0, ptr, None, on_host=True)
        rc = self.lib.gbd_render_batch(self.handle, int(vol), arr, len(views), ctypes.byref(spec), _launch(launch),
                                       _stream_handle(stream))
        _check(self.lib, rc)
        return out_host

    def tune(self, vol: int, views, *, launch: bool = True, layout: bool = False, stream=None) -> dict:
        """Autotune the batch render of ``views`` (launch configuration and,
        with ``layout``, the volume's brick layout).  Later calls of the same
        class without an explicit launch use the result."""
        import torch
        views = list(views)
        v0 = views[0]
        out = torch.empty((len(views), int(v0.height), int(v0.width)), dtype=torch.float32,
                          device=torch.device("cuda", self.device))
        arr = (CView * len(views))(*[_cview(v) for v in views])
        spec = self._spec(v0, out.data_ptr(), None)
        res = TuneResult()
        what = (TUNE_LAUNCH if launch else 0) | (TUNE_LAYOUT if layout else 0)
        _check(self.lib, self.lib.gbd_tune(self.handle, int(vol), arr, len(views), ctypes.byref(spec), what,
                                           _stream_handle(stream), ctypes.byref(res)))
        lw = res.launch
        return dict(packet=(lw.packet_w, lw.packet_h), cta_warps=lw.cta_warps, depth=lw.depth,
                    persistent=lw.persistent, regcap=lw.regcap, region=lw.region, group=lw.group, brick=res.brick,
                    super_brick=res.super_brick,
                    paired=res.paired, morton_cells=res.morton_cells, ms=res.ms, candidates=res.candidates)

    def relayout(self, vol: int, brick: int, super_brick: int, paired: bool = False, morton_cells: bool = False):
        _check(self.lib, self.lib.gbd_relayout(self.handle, int(vol), int(brick), int(super_brick),
                                               int(bool(paired)), int(bool(morton_cells))))

    def bounds_violations(self) -> int:
        """Device error word (waits for the device and clears it): bit 0 a
        bounds-check violation of the checked library, bit 1 a region ray
        list that ran out of room; 0 when neither happened."""
        w = ctypes.c_int32()
        _check(self.lib, self.lib.gbd_bounds_violations(self.handle, ctypes.byref(w)))
        return int(w.value)

    # -- serving
    def serve_start(self, *, max_waves: int = 0, max_requests_per_wave: int = 0, max_requests_in_flight: int = 0,
                    request_budget_bytes: int = 0, launch=None):
        cfg = ServeConfig()
        cfg.max_waves = int(max_waves)
        cfg.max_requests_per_wave = int(max_requests_per_wave)
        cfg.max_requests_in_flight = int(max_requests_in_flight)
        cfg.request_budget_bytes = int(request_budget_bytes)
        lp = _launch(launch)
        if lp is not None:
            cfg.launch = lp.contents
        _check(self.lib, self.lib.gbd_serve_start(self.handle, ctypes.byref(cfg)))

    def serve_stop(self):
        _check(self.lib, self.lib.gbd_serve_stop(self.handle))
        self._served = {}

    def submit(self, vol: int, view, out, *, priority: int = 0) -> int:
        """Queue a render of ``view`` into ``out`` (device tensor, or pinned
        host tensor) [height][width]; returns the ticket.  ``out`` is kept
        alive until the request is reported done."""
        r = Request()
        r.volume = int(vol)
        r.view = _cview(view)
        on_host = not (hasattr(out, "is_cuda") and out.is_cuda)
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        r.spec = self._spec(view, ptr, None, on_host=on_host)
        r.priority = int(priority)
        t = ctypes.c_uint64()
        _check(self.lib, self.lib.gbd_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        if not hasattr(self, "_served"):
            self._served = {}
        self._served[int(t.value)] = out
        return int(t.value)

    @staticmethod
    def _stats(st: Stats) -> dict:
        return dict(status=st.status, queue_ms=st.queue_ms, latency_ms=st.latency_ms, device_ms=st.device_ms)

    def poll(self, ticket: int):
        """(done, stats); raises GbdError if the request ended with an error."""
        done = ctypes.c_int32()
        st = Stats()
        rc = self.lib.gbd_poll(self.handle, int(ticket), ctypes.byref(done), ctypes.byref(st))
        if done.value:
            getattr(self, "_served", {}).pop(int(ticket), None)
        _check(self.lib, rc)
        return bool(done.value), self._stats(st)

    def wait(self, ticket: int, timeout_ms: int = 60000) -> dict:
        st = Stats()
        rc = self.lib.gbd_wait(self.handle, int(ticket), int(timeout_ms), ctypes.byref(st))
        if rc != ERR_TIMEOUT:
            getattr(self, "_served", {}).pop(int(ticket), None)
        _check(self.lib, rc)
        return self._stats(st)

    def cancel(self, ticket: int):
        _check(self.lib, self.lib.gbd_cancel(self.handle, int(ticket)))

    def serve_stats(self, reset: bool = False) -> dict:
        s = ServeSummary()
        _check(self.lib, self.lib.gbd_serve_stats(self.handle, int(bool(reset)), ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServeSummary._fields_}

    def last_launch_count(self) -> int:
        return int(self.lib.gbd_last_launch_count())


def error_string(code: int) -> str:
    return load_library().gbd_error_string(int(code)).decode()
