"""ctypes binding of libfdk with the C ABI's names (include/fdk.h).

Tensors are passed as raw pointers; shapes give dims, det and n_views; the
stream is PyTorch's current stream unless one is given.  Nothing here
computes: every step of the back-projection runs in the library's kernels.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import threading
from typing import Optional

import numpy as np
import torch

from . import build as _build

FDK_OK, FDK_ERR_INVALID_ARG, FDK_ERR_UNSUPPORTED, FDK_ERR_OOM, FDK_ERR_CUDA, FDK_ERR_TIMEOUT = range(6)
FDK_F32, FDK_BF16, FDK_F16 = 0, 1, 2
FETCH_AUTO, FETCH_LDG, FETCH_TEX, FETCH_QUAD, FETCH_STAGE = 0, 1, 2, 3, 4
_STATUS = {0: "FDK_OK", 1: "FDK_ERR_INVALID_ARG", 2: "FDK_ERR_UNSUPPORTED", 3: "FDK_ERR_OOM",
           4: "FDK_ERR_CUDA", 5: "FDK_ERR_TIMEOUT"}
_DTYPES = {torch.float32: FDK_F32, torch.bfloat16: FDK_BF16, torch.float16: FDK_F16}


class FdkError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class fdk_opts(ctypes.Structure):
    _fields_ = [("proj_dtype", ctypes.c_int32), ("matrices_on_device", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("fetch", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("overwrite", ctypes.c_int32), ("reserved", ctypes.c_int32 * 8)]


class fdk_scan(ctypes.Structure):
    _fields_ = [("volume", ctypes.c_void_p), ("dims", ctypes.c_int32 * 3),
                ("voxel_size", ctypes.c_float * 3), ("origin", ctypes.c_float * 3),
                ("projections", ctypes.c_void_p), ("det", ctypes.c_int32 * 2),
                ("matrices", ctypes.c_void_p), ("n_views", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None
_i32_3 = ctypes.c_int32 * 3
_i32_2 = ctypes.c_int32 * 2
_f32_3 = ctypes.c_float * 3


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB) or not _build.up_to_date():
                _build.build()
            lib = ctypes.CDLL(_build.LIB)
            vp, fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)
            i3 = ctypes.POINTER(ctypes.c_int32)
            f3 = ctypes.POINTER(ctypes.c_float)
            op = ctypes.POINTER(fdk_opts)
            lib.fdk_backproject.argtypes = [vp, i3, f3, f3, vp, i3, vp, ctypes.c_int32, op]
            lib.fdk_forwardproject_adjoint.argtypes = [vp, i3, vp, i3, f3, f3, vp, ctypes.c_int32, op]
            lib.fdk_backproject_static.argtypes = [vp, i3, f3, f3, vp, i3, vp, ctypes.c_int32, op]
            lib.fdk_backproject_static.restype = ctypes.c_int
            lib.fdk_backproject_host.argtypes = [vp, i3, f3, f3, vp, i3, vp, ctypes.c_int32, op]
            lib.fdk_backproject_host.restype = ctypes.c_int
            lib.fdk_count_updates.argtypes = [ctypes.POINTER(ctypes.c_int64), i3, f3, f3, i3, vp,
                                              ctypes.c_int32, op]
            for fn in (lib.fdk_backproject, lib.fdk_forwardproject_adjoint, lib.fdk_count_updates):
                fn.restype = ctypes.c_int
            sp = ctypes.POINTER(fdk_scan)
            pp = ctypes.POINTER(ctypes.c_void_p)
            lib.fdk_batch_plan_create.argtypes = [pp, sp, ctypes.c_int32, op]
            lib.fdk_batch_plan_create.restype = ctypes.c_int
            lib.fdk_batch_plan_execute.argtypes = [vp, vp]
            lib.fdk_batch_plan_execute.restype = ctypes.c_int
            lib.fdk_batch_plan_tile.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
            lib.fdk_batch_plan_tile.restype = ctypes.c_int
            lib.fdk_batch_plan_scan_fetch.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
            lib.fdk_batch_plan_scan_fetch.restype = ctypes.c_int
            lib.fdk_batch_plan_destroy.argtypes = [vp]
            lib.fdk_batch_plan_destroy.restype = None
            lib.fdk_backproject_batched.argtypes = [sp, ctypes.c_int32, op]
            lib.fdk_backproject_batched.restype = ctypes.c_int
            lib.fdk_preweight_filter.argtypes = [vp, vp, i3, vp, ctypes.c_int32, ctypes.c_float, op]
            lib.fdk_preweight_filter.restype = ctypes.c_int
            lib.fdk_last_error.restype = ctypes.c_char_p
            lib.fdk_last_error.argtypes = []
            lib.fdk_version.restype = ctypes.c_int32
            lib.fdk_release.restype = None
            lib.fdk_device_status.argtypes = []
            lib.fdk_device_status.restype = ctypes.c_int
            lib.fdk_microbench.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
            lib.fdk_microbench.restype = ctypes.c_int
            lib.fdk_testing_set_wait_limit.argtypes = [ctypes.c_int64]
            lib.fdk_testing_set_wait_limit.restype = ctypes.c_int
            lib.fdk_testing_fail_allocations.argtypes = [ctypes.c_int32]
            lib.fdk_testing_fail_allocations.restype = ctypes.c_int
            _lib = lib
    return _lib


def fdk_last_error() -> str:
    return _load().fdk_last_error().decode()


def fdk_version() -> int:
    return int(_load().fdk_version())


def fdk_release() -> None:
    _load().fdk_release()


def fdk_device_status() -> None:
    """Synchronise the current device; raise FdkError if a bounded
    device-side wait of an earlier call gave up (FDK_ERR_TIMEOUT) or the
    device reported an error."""
    _check(_load().fdk_device_status())


MICRO_LDG, MICRO_LDS, MICRO_TLD4, MICRO_RCP, MICRO_CHASE = 1, 2, 3, 4, 5


def fdk_microbench(which: int, param: int = 0) -> float:
    """One gather micro-benchmark of the current device (see include/fdk.h):
    warp operations per SM per cycle, or cycles per load for MICRO_CHASE."""
    out = ctypes.c_double(0.0)
    _check(_load().fdk_microbench(int(which), int(param), ctypes.byref(out)))
    return float(out.value)


def _check(st: int):
    if st != FDK_OK:
        raise FdkError(st, fdk_last_error())


def fdk_testing_set_wait_limit(polls: int) -> None:
    """Testing hook (include/fdk_testing.h): poll limit of the consumer
    waits of later launches (0: give up at once; < 0: the built-in limit)."""
    _check(_load().fdk_testing_set_wait_limit(int(polls)))


def fdk_testing_fail_allocations(n: int) -> None:
    """Testing hook (include/fdk_testing.h): the library's next n device
    allocations fail as on a device out of memory."""
    _check(_load().fdk_testing_fail_allocations(int(n)))


def _device_of(*tensors):
    """The one CUDA device that every CUDA tensor among ``tensors`` lives on
    (None if none is a CUDA tensor: the library then refuses the call).  The
    library launches on the current device, so each call runs with this
    device current, and tensors on different devices are refused here,
    before any call."""
    devs = {t.device for t in tensors if getattr(t, "is_cuda", False)}
    if len(devs) > 1:
        raise ValueError(f"tensors on different devices: {sorted(str(d) for d in devs)}")
    return devs.pop() if devs else None


def _on(*tensors):
    """Context that makes the tensors' CUDA device current for one call."""
    dev = _device_of(*tensors)
    return torch.cuda.device(dev) if dev is not None else contextlib.nullcontext()


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _mats(matrices, n_views: int):
    """Host FP32 (n,12) numpy array, or a CUDA FP32 tensor (device matrices)."""
    if isinstance(matrices, torch.Tensor) and matrices.is_cuda:
        m = matrices.reshape(-1, 12)
        if m.dtype != torch.float32 or not m.is_contiguous():
            raise ValueError("device matrices must be contiguous float32")
        if m.shape[0] != n_views:
            raise ValueError("need one 3x4 matrix per view")
        return m, m.data_ptr(), 1
    if isinstance(matrices, torch.Tensor):
        matrices = matrices.numpy()
    m = np.ascontiguousarray(np.asarray(matrices, dtype=np.float32).reshape(-1, 12))
    if m.shape[0] != n_views:
        raise ValueError("need one 3x4 matrix per view")
    return m, m.ctypes.data, 0


def _opts(dtype: int, mats_dev: int, stream, fetch: int, tile: int) -> fdk_opts:
    o = fdk_opts()
    o.proj_dtype = dtype
    o.matrices_on_device = mats_dev
    o.stream = stream if isinstance(stream, int) else (
        (stream or torch.cuda.current_stream()).cuda_stream)
    o.fetch = fetch
    o.tile = tile
    return o


def _geom(voxel_size, origin):
    vs = np.asarray(voxel_size, dtype=np.float32).reshape(3)
    org = np.asarray(origin, dtype=np.float32).reshape(3)
    return _f32_3(*vs.tolist()), _f32_3(*org.tolist())


def fdk_backproject(volume: torch.Tensor, projections: torch.Tensor, matrices, voxel_size, origin,
                    *, fetch: int = FETCH_AUTO, tile: int = 0, stream=None) -> torch.Tensor:
    """volume[nz,ny,nx] (CUDA FP32) += back-projection of projections[n,H,W]
    (CUDA FP32/BF16/FP16) with per-view row-major 3x4 matrices (host array or
    CUDA tensor).  Returns ``volume``."""
    if volume.dtype != torch.float32 or volume.dim() != 3 or not volume.is_contiguous():
        raise ValueError("volume must be a contiguous float32 (nz, ny, nx) tensor")
    if projections.dim() != 3 or not projections.is_contiguous():
        raise ValueError("projections must be a contiguous (n_views, H, W) tensor")
    if projections.dtype not in _DTYPES:
        raise ValueError(f"unsupported projection dtype {projections.dtype}")
    n = projections.shape[0]
    m, mptr, mdev = _mats(matrices, n)
    nz, ny, nx = volume.shape
    vs, org = _geom(voxel_size, origin)
    lib = _load()
    with _on(volume, projections, m):
        o = _opts(_DTYPES[projections.dtype], mdev, stream, fetch, tile)
        st = lib.fdk_backproject(_ptr(volume), _i32_3(nx, ny, nz), vs, org, _ptr(projections),
                                 _i32_2(projections.shape[2], projections.shape[1]), mptr, n,
                                 ctypes.byref(o))
    _check(st)
    return volume


def fdk_backproject_host(volume: torch.Tensor, projections: torch.Tensor, matrices, voxel_size, origin,
                         *, fetch: int = FETCH_AUTO, tile: int = 0, stream=None,
                         overwrite: bool = False) -> torch.Tensor:
    """fdk_backproject for host (CPU) tensors: volume[nz,ny,nx] FP32 +=
    back-projection of projections[n,H,W] (FP32/BF16/FP16), host matrices.
    The library copies in chunks of views, overlapping copies with the
    back-projection (pinned tensors overlap; pageable ones copy
    synchronously), and synchronises before returning.  With
    ``overwrite=True`` the result replaces ``volume`` (which is then not
    copied to the device).  Returns ``volume``."""
    if volume.is_cuda or projections.is_cuda:
        raise ValueError("fdk_backproject_host takes host tensors (use fdk_backproject for CUDA tensors)")
    if volume.dtype != torch.float32 or volume.dim() != 3 or not volume.is_contiguous():
        raise ValueError("volume must be a contiguous float32 (nz, ny, nx) tensor")
    if projections.dim() != 3 or not projections.is_contiguous():
        raise ValueError("projections must be a contiguous (n_views, H, W) tensor")
    if projections.dtype not in _DTYPES:
        raise ValueError(f"unsupported projection dtype {projections.dtype}")
    n = projections.shape[0]
    m, mptr, mdev = _mats(matrices, n)
    if mdev:
        raise ValueError("fdk_backproject_host takes host matrices")
    nz, ny, nx = volume.shape
    vs, org = _geom(voxel_size, origin)
    o = _opts(_DTYPES[projections.dtype], False, stream, fetch, tile)
    o.overwrite = 1 if overwrite else 0
    st = _load().fdk_backproject_host(_ptr(volume), _i32_3(nx, ny, nz), vs, org, _ptr(projections),
                                      _i32_2(projections.shape[2], projections.shape[1]), mptr, n,
                                      ctypes.byref(o))
    _check(st)
    return volume


def fdk_backproject_static(volume: torch.Tensor, projections: torch.Tensor, matrices, voxel_size,
                           origin, *, tile: int = 0, stream=None) -> torch.Tensor:
    """fdk_backproject for callers that must not allocate device memory: the
    library stages the images in its fixed 64 MiB array (see include/fdk.h).
    Same arguments and result as :func:`fdk_backproject`."""
    if volume.dtype != torch.float32 or volume.dim() != 3 or not volume.is_contiguous():
        raise ValueError("volume must be a contiguous float32 (nz, ny, nx) tensor")
    if projections.dim() != 3 or not projections.is_contiguous():
        raise ValueError("projections must be a contiguous (n_views, H, W) tensor")
    if projections.dtype not in _DTYPES:
        raise ValueError(f"unsupported projection dtype {projections.dtype}")
    n = projections.shape[0]
    m, mptr, mdev = _mats(matrices, n)
    nz, ny, nx = volume.shape
    vs, org = _geom(voxel_size, origin)
    lib = _load()
    with _on(volume, projections, m):
        o = _opts(_DTYPES[projections.dtype], mdev, stream, FETCH_AUTO, tile)
        st = lib.fdk_backproject_static(_ptr(volume), _i32_3(nx, ny, nz), vs, org, _ptr(projections),
                                        _i32_2(projections.shape[2], projections.shape[1]), mptr, n,
                                        ctypes.byref(o))
    _check(st)
    return volume


def fdk_forwardproject_adjoint(projections: torch.Tensor, volume: torch.Tensor, matrices,
                               voxel_size, origin, *, stream=None) -> torch.Tensor:
    """projections[n,H,W] (CUDA FP32) += transpose of the back-projection
    applied to volume[nz,ny,nx] (CUDA FP32).  Returns ``projections``."""
    if projections.dtype != torch.float32 or projections.dim() != 3 or not projections.is_contiguous():
        raise ValueError("projections must be a contiguous float32 (n_views, H, W) tensor")
    if volume.dtype != torch.float32 or volume.dim() != 3 or not volume.is_contiguous():
        raise ValueError("volume must be a contiguous float32 (nz, ny, nx) tensor")
    n = projections.shape[0]
    m, mptr, mdev = _mats(matrices, n)
    nz, ny, nx = volume.shape
    vs, org = _geom(voxel_size, origin)
    lib = _load()
    with _on(projections, volume, m):
        o = _opts(FDK_F32, mdev, stream, FETCH_AUTO, 0)
        st = lib.fdk_forwardproject_adjoint(_ptr(projections),
                                            _i32_2(projections.shape[2], projections.shape[1]),
                                            _ptr(volume), _i32_3(nx, ny, nz), vs, org, mptr, n,
                                            ctypes.byref(o))
    _check(st)
    return projections


def fdk_count_updates(dims, det, matrices, voxel_size, origin, *, stream=None) -> int:
    """Clipped update count: voxel/view pairs with w > 0, -1 < u < W, -1 < v < H."""
    n = int(np.asarray(matrices).reshape(-1, 12).shape[0]) if not isinstance(matrices, torch.Tensor) \
        else int(matrices.reshape(-1, 12).shape[0])
    m, mptr, mdev = _mats(matrices, n)
    vs, org = _geom(voxel_size, origin)
    with _on(m):
        o = _opts(FDK_F32, mdev, stream, FETCH_AUTO, 0)
    out = ctypes.c_int64(0)
    d = [int(x) for x in dims]
    lib = _load()
    with _on(m):
        st = lib.fdk_count_updates(ctypes.byref(out), _i32_3(*d), vs, org,
                                   _i32_2(int(det[0]), int(det[1])), mptr, n, ctypes.byref(o))
    _check(st)
    return int(out.value)


def _scan_array(scans):
    """scans: sequence of (volume, projections, matrices, voxel_size, origin)."""
    arr = (fdk_scan * len(scans))()
    keep = []
    for s, (vol, proj, mats, vs, org) in zip(arr, scans):
        if vol.dtype != torch.float32 or vol.dim() != 3 or not vol.is_contiguous():
            raise ValueError("volume must be a contiguous float32 (nz, ny, nx) tensor")
        if proj.dtype != torch.float32 or proj.dim() != 3 or not proj.is_contiguous():
            raise ValueError("projections must be a contiguous float32 (n, H, W) tensor")
        m = np.ascontiguousarray(np.asarray(mats.cpu() if isinstance(mats, torch.Tensor) else mats,
                                            dtype=np.float32).reshape(-1, 12))
        if m.shape[0] != proj.shape[0]:
            raise ValueError("need one 3x4 matrix per view")
        keep.append(m)
        nz, ny, nx = vol.shape
        s.volume = vol.data_ptr()
        s.dims[:] = [nx, ny, nz]
        s.voxel_size[:] = [float(x) for x in np.asarray(vs, dtype=np.float32).reshape(3)]
        s.origin[:] = [float(x) for x in np.asarray(org, dtype=np.float32).reshape(3)]
        s.projections = proj.data_ptr()
        s.det[:] = [proj.shape[2], proj.shape[1]]
        s.matrices = m.ctypes.data
        s.n_views = proj.shape[0]
    return arr, keep


class BatchPlan:
    """fdk_batch_plan_create / _execute / _tile / _destroy.  The tensors of
    every scan must outlive the plan."""

    def __init__(self, scans, *, tile: int = 0, autotune: bool = False, fetch: int = FETCH_AUTO):
        arr, keep = _scan_array(scans)
        o = fdk_opts()
        o.tile = tile
        o.autotune = 1 if autotune else 0
        o.fetch = fetch
        h = ctypes.c_void_p()
        lib = _load()
        self._tensors = [t for sc in scans for t in (sc[0], sc[1])]
        with _on(*self._tensors):
            _check(lib.fdk_batch_plan_create(ctypes.byref(h), arr, len(scans), ctypes.byref(o)))
        self._h = h
        self._lib = lib
        self.scans = list(scans)

    @property
    def tile(self) -> int:
        t = ctypes.c_int32(0)
        _check(self._lib.fdk_batch_plan_tile(self._h, ctypes.byref(t)))
        return int(t.value)

    def scan_fetch(self, scan: int) -> int:
        """FETCH_STAGE or FETCH_LDG: the fetch path the plan uses for scan ``scan``."""
        f = ctypes.c_int32(0)
        _check(self._lib.fdk_batch_plan_scan_fetch(self._h, int(scan), ctypes.byref(f)))
        return int(f.value)

    def execute(self, stream=None):
        with _on(*self._tensors):
            s = stream if isinstance(stream, int) else (stream or torch.cuda.current_stream()).cuda_stream
            _check(self._lib.fdk_batch_plan_execute(self._h, ctypes.c_void_p(s)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fdk_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fdk_batch_plan_create(scans, *, tile: int = 0, autotune: bool = False, fetch: int = FETCH_AUTO) -> BatchPlan:
    return BatchPlan(scans, tile=tile, autotune=autotune, fetch=fetch)


def fdk_backproject_batched(scans, *, tile: int = 0, fetch: int = FETCH_AUTO, stream=None):
    """One-shot batch: create a plan, execute it, synchronise, destroy."""
    arr, keep = _scan_array(scans)
    o = fdk_opts()
    o.tile = tile
    o.fetch = fetch
    lib = _load()
    with _on(*[t for sc in scans for t in (sc[0], sc[1])]):
        o.stream = stream if isinstance(stream, int) else (stream or torch.cuda.current_stream()).cuda_stream
        st = lib.fdk_backproject_batched(arr, len(scans), ctypes.byref(o))
    _check(st)


def fdk_preweight_filter(out: torch.Tensor, raw: torch.Tensor, matrices, scale: float = 1.0,
                         *, stream=None) -> torch.Tensor:
    """out[n, H, W] = cosine pre-weighted, Ram-Lak row-filtered raw[n, H, W]
    (CUDA FP32; out may be raw).  Returns ``out``."""
    for t, name in ((out, "out"), (raw, "raw")):
        if t.dtype != torch.float32 or t.dim() != 3 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 (n_views, H, W) tensor")
    if out.shape != raw.shape:
        raise ValueError("out and raw must have the same shape")
    n = raw.shape[0]
    m, mptr, mdev = _mats(matrices, n)
    lib = _load()
    with _on(out, raw, m):
        o = _opts(FDK_F32, mdev, stream, FETCH_AUTO, 0)
        st = lib.fdk_preweight_filter(_ptr(out), _ptr(raw), _i32_2(raw.shape[2], raw.shape[1]), mptr, n,
                                      float(scale), ctypes.byref(o))
    _check(st)
    return out
