"""FP64 CPU oracle for the cone-beam back-projection (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package.  It compiles ``fdk_oracle.c`` with gcc (no fused
multiply-add contraction, so x86 and Arm give the same bits) and wraps its
entry points for numpy arrays.  It shares nothing with the CUDA library.

Functions follow Listing 1 and Sec. IV of the paper; see ``fdk_oracle.c``
for the definition and the readings taken where the listing is ambiguous.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdk_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libfdk_oracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # FDK_ORACLE_LIB names another build of fdk_oracle.c to load instead;
            # the mutation tests use it to run the pins against planted mistakes
            lib = ctypes.CDLL(os.environ.get("FDK_ORACLE_LIB") or build())
            lib.oracle_backproject.argtypes = [_f64p, _i64p, _f64p, _f64p, _f32p, ctypes.c_int64,
                                               ctypes.c_int64, _f32p, ctypes.c_int64,
                                               ctypes.c_int, ctypes.c_int]
            lib.oracle_backproject_voxels.argtypes = [_f64p, _i64p, ctypes.c_int64, _f64p, _f64p,
                                                      _f32p, ctypes.c_int64, ctypes.c_int64,
                                                      _f32p, ctypes.c_int64]
            lib.oracle_adjoint.argtypes = [_f64p, _i64p, _f64p, _f64p, _f32p, ctypes.c_int64,
                                           ctypes.c_int64, _f32p, ctypes.c_int64, ctypes.c_int]
            lib.oracle_bruteforce.argtypes = [_f64p, _i64p, _f64p, _f64p, _f32p, ctypes.c_int64,
                                              ctypes.c_int64, _f32p, ctypes.c_int64]
            lib.oracle_camera.argtypes = [_f32p, ctypes.c_int64, _f64p]
            lib.oracle_preweight_filter.argtypes = [_f64p, _f32p, ctypes.c_int64, ctypes.c_int64,
                                                    _f32p, ctypes.c_int64, ctypes.c_double]
            lib.oracle_count_updates.argtypes = [_i64p, _i64p, _i64p, _f64p, _f64p, ctypes.c_int64,
                                                 ctypes.c_int64, _f32p, ctypes.c_int64, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_int]
            for fn in (lib.oracle_backproject, lib.oracle_backproject_voxels,
                       lib.oracle_adjoint, lib.oracle_bruteforce, lib.oracle_camera,
                       lib.oracle_preweight_filter, lib.oracle_count_updates):
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _geom(dims, voxel_size, origin):
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64).reshape(3))
    # the library takes voxel size and origin as FP32; promote those values
    vs = np.ascontiguousarray(np.asarray(voxel_size, dtype=np.float32).astype(np.float64).reshape(3))
    org = np.ascontiguousarray(np.asarray(origin, dtype=np.float32).astype(np.float64).reshape(3))
    return d, vs, org


def _proj(proj):
    p = np.ascontiguousarray(np.asarray(proj, dtype=np.float32))
    if p.ndim != 3:
        raise ValueError("projections must be (n_views, H, W)")
    return p


def _mats(mats, n_views):
    m = np.ascontiguousarray(np.asarray(mats, dtype=np.float32).reshape(-1, 12))
    if m.shape[0] != n_views:
        raise ValueError("need one 3x4 matrix per view")
    return m


def backproject(proj, mats, dims, voxel_size, origin, vol=None, threads: int = 1,
                literal_trunc: bool = False) -> np.ndarray:
    """FP64 back-projection: returns vol (nz, ny, nx) float64 (accumulated
    into ``vol`` when given).  ``threads`` splits (z, y) lines; the result is
    bit-identical for any thread count."""
    p = _proj(proj)
    n, H, W = p.shape
    m = _mats(mats, n)
    d, vs, org = _geom(dims, voxel_size, origin)
    if vol is None:
        vol = np.zeros((int(d[2]), int(d[1]), int(d[0])), dtype=np.float64)
    assert vol.dtype == np.float64 and vol.flags.c_contiguous
    rc = _load().oracle_backproject(_p(vol, _f64p), _p(d, _i64p), _p(vs, _f64p), _p(org, _f64p),
                                    _p(p, _f32p), W, H, _p(m, _f32p), n, int(threads),
                                    int(bool(literal_trunc)))
    if rc != 0:
        raise RuntimeError(f"oracle_backproject failed ({rc})")
    return vol


def backproject_voxels(proj, mats, voxel_size, origin, xyz) -> np.ndarray:
    """FP64 back-projection at selected voxels; xyz is (n, 3) int (x, y, z)."""
    p = _proj(proj)
    n, H, W = p.shape
    m = _mats(mats, n)
    _, vs, org = _geom((1, 1, 1), voxel_size, origin)
    q = np.ascontiguousarray(np.asarray(xyz, dtype=np.int64).reshape(-1, 3))
    out = np.zeros(q.shape[0], dtype=np.float64)
    rc = _load().oracle_backproject_voxels(_p(out, _f64p), _p(q, _i64p), q.shape[0],
                                           _p(vs, _f64p), _p(org, _f64p), _p(p, _f32p), W, H,
                                           _p(m, _f32p), n)
    if rc != 0:
        raise RuntimeError(f"oracle_backproject_voxels failed ({rc})")
    return out


def adjoint(vol, mats, dims, voxel_size, origin, det_w: int, det_h: int, proj=None,
            threads: int = 1) -> np.ndarray:
    """FP64 transpose of :func:`backproject`: returns (n_views, H, W) float64."""
    v = np.ascontiguousarray(np.asarray(vol, dtype=np.float32))
    d, vs, org = _geom(dims, voxel_size, origin)
    m = np.ascontiguousarray(np.asarray(mats, dtype=np.float32).reshape(-1, 12))
    n = m.shape[0]
    if v.shape != (int(d[2]), int(d[1]), int(d[0])):
        raise ValueError("volume shape must be (nz, ny, nx)")
    if proj is None:
        proj = np.zeros((n, det_h, det_w), dtype=np.float64)
    assert proj.dtype == np.float64 and proj.flags.c_contiguous
    rc = _load().oracle_adjoint(_p(proj, _f64p), _p(d, _i64p), _p(vs, _f64p), _p(org, _f64p),
                                _p(v, _f32p), det_w, det_h, _p(m, _f32p), n, int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_adjoint failed ({rc})")
    return proj


def bruteforce(proj, mats, dims, voxel_size, origin) -> np.ndarray:
    """FP64 tent-sum evaluation over every pixel (tiny cases only)."""
    p = _proj(proj)
    n, H, W = p.shape
    m = _mats(mats, n)
    d, vs, org = _geom(dims, voxel_size, origin)
    vol = np.zeros((int(d[2]), int(d[1]), int(d[0])), dtype=np.float64)
    rc = _load().oracle_bruteforce(_p(vol, _f64p), _p(d, _i64p), _p(vs, _f64p), _p(org, _f64p),
                                   _p(p, _f32p), W, H, _p(m, _f32p), n)
    if rc != 0:
        raise RuntimeError(f"oracle_bruteforce failed ({rc})")
    return vol


def camera(mats) -> np.ndarray:
    """(n, 3) array of (f, u0, v0) per view, read off each matrix through
    M M^T (square pixels, no skew)."""
    m = np.ascontiguousarray(np.asarray(mats, dtype=np.float32).reshape(-1, 12))
    out = np.zeros((m.shape[0], 3), dtype=np.float64)
    if _load().oracle_camera(_p(m, _f32p), m.shape[0], _p(out, _f64p)) != 0:
        raise ValueError("matrix is not a camera with square pixels")
    return out


def preweight_filter(proj, mats, scale: float = 1.0) -> np.ndarray:
    """FP64 cosine pre-weighting and Ram-Lak row filtering of raw line
    integrals (n, H, W) (direct linear convolution, small cases)."""
    p = _proj(proj)
    n, H, W = p.shape
    m = _mats(mats, n)
    out = np.zeros((n, H, W), dtype=np.float64)
    rc = _load().oracle_preweight_filter(_p(out, _f64p), _p(p, _f32p), W, H, _p(m, _f32p), n,
                                         float(scale))
    if rc != 0:
        raise RuntimeError(f"oracle_preweight_filter failed ({rc})")
    return out


def count_updates(mats, dims, voxel_size, origin, det_w: int, det_h: int, eps: float = 1e-3,
                  eps_w: float = 1e-5, threads: int = 1):
    """The clipped update count: (voxel, view) pairs with w > 0, -1 < u < W
    and -1 < v < H (Sec. VII).  Returns (count, band), band being the pairs
    within eps pixels (eps_w in w) of one of those decisions, which a lower
    precision evaluation may decide either way."""
    d, vs, org = _geom(dims, voxel_size, origin)
    m = np.ascontiguousarray(np.asarray(mats, dtype=np.float32).reshape(-1, 12))
    c = np.zeros(1, dtype=np.int64)
    b = np.zeros(1, dtype=np.int64)
    rc = _load().oracle_count_updates(_p(c, _i64p), _p(b, _i64p), _p(d, _i64p), _p(vs, _f64p), _p(org, _f64p),
                                      int(det_w), int(det_h), _p(m, _f32p), m.shape[0], float(eps),
                                      float(eps_w), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_count_updates failed ({rc})")
    return int(c[0]), int(b[0])
