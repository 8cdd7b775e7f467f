"""Host-side checks of the C ABI: the library builds, loads and exports every
declared entry point, and argument validation rejects bad calls before any
CUDA work (these run without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1401_3615_gb300 import build as fdk_build
from paper_1401_3615_gb300 import fdk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"FDK_API\s+[\w\s\*]+?\b(fdk_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    path = fdk_build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "fdk_backproject" in names and "fdk_forwardproject_adjoint" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert fdk.fdk_version() == 1


def _raw():
    return fdk._load()


def _call_bp(vol=1, dims=(4, 4, 4), vs=(1, 1, 1), org=(0, 0, 0), proj=2, det=(8, 8),
             mats=None, n=1, opts=None):
    lib = _raw()
    m = (ctypes.c_float * 12)(*([1.0] * 12)) if mats is None else mats
    d = None if dims is None else (ctypes.c_int32 * 3)(*dims)
    v = None if vs is None else (ctypes.c_float * 3)(*vs)
    o = None if org is None else (ctypes.c_float * 3)(*org)
    dt = None if det is None else (ctypes.c_int32 * 2)(*det)
    op = ctypes.byref(opts) if opts is not None else None
    # pointers are never dereferenced: every case fails validation first
    return lib.fdk_backproject(ctypes.c_void_p(vol * 256) if vol else None, d, v, o,
                               ctypes.c_void_p(proj * 256) if proj else None, dt, m, n, op)


@pytest.mark.parametrize("kw,msg", [
    (dict(vol=0), "volume"),
    (dict(proj=0), "projections"),
    (dict(dims=None), "null"),
    (dict(dims=(0, 4, 4)), "dims"),
    (dict(dims=(4, -1, 4)), "dims"),
    (dict(vs=(1, 0, 1)), "voxel_size"),
    (dict(vs=(1, float("nan"), 1)), "voxel_size"),
    (dict(org=(float("inf"), 0, 0)), "origin"),
    (dict(det=(0, 8)), "det"),
    (dict(det=(70000, 70000)), "detector too large"),
    (dict(n=-1), "n_views"),
    (dict(dims=(1 << 20, 1 << 20, 1 << 20)), "volume too large"),
])
def test_invalid_arguments_rejected(kw, msg):
    st = _call_bp(**kw)
    assert st == fdk.FDK_ERR_INVALID_ARG
    assert msg in fdk.fdk_last_error()


def test_bad_options_rejected():
    for field, val, msg in [("proj_dtype", 7, "proj_dtype"), ("matrices_on_device", 2, "matrices_on_device"),
                            ("fetch", 9, "fetch"), ("tile", 8, "tile"), ("tile", -1, "tile")]:
        o = fdk.fdk_opts()
        setattr(o, field, val)
        assert _call_bp(opts=o) == fdk.FDK_ERR_INVALID_ARG
        assert msg in fdk.fdk_last_error()
    o = fdk.fdk_opts()
    o.reserved[3] = 1
    assert _call_bp(opts=o) == fdk.FDK_ERR_INVALID_ARG
    o = fdk.fdk_opts()
    o.overwrite = 1                      # only fdk_backproject_host takes it
    assert _call_bp(opts=o) == fdk.FDK_ERR_INVALID_ARG and "overwrite" in fdk.fdk_last_error()


def test_nonfinite_matrix_rejected():
    m = (ctypes.c_float * 12)(*([1.0] * 11 + [float("nan")]))
    assert _call_bp(mats=m) == fdk.FDK_ERR_INVALID_ARG
    assert "finite" in fdk.fdk_last_error()


def test_misaligned_pointer_rejected():
    lib = _raw()
    d = (ctypes.c_int32 * 3)(4, 4, 4)
    f3 = (ctypes.c_float * 3)(1, 1, 1)
    m = (ctypes.c_float * 12)(*([1.0] * 12))
    st = lib.fdk_backproject(ctypes.c_void_p(4098), d, f3, f3, ctypes.c_void_p(4096),
                             (ctypes.c_int32 * 2)(8, 8), m, 1, None)
    assert st == fdk.FDK_ERR_INVALID_ARG and "aligned" in fdk.fdk_last_error()


def test_zero_views_is_noop_without_gpu():
    assert _call_bp(n=0, proj=0, mats=None) == fdk.FDK_OK
    assert fdk.fdk_last_error() == ""


def test_host_entry_point_validates_before_cuda():
    """fdk_backproject_host shares the argument checks of fdk_backproject
    and refuses device matrices, all before any CUDA call."""
    lib = _raw()
    d = (ctypes.c_int32 * 3)(4, 4, 4)
    f3 = (ctypes.c_float * 3)(1, 1, 1)
    m = (ctypes.c_float * 12)(*([1.0] * 12))
    det = (ctypes.c_int32 * 2)(8, 8)
    st = lib.fdk_backproject_host(None, d, f3, f3, ctypes.c_void_p(256), det, m, 1, None)
    assert st == fdk.FDK_ERR_INVALID_ARG and "volume" in fdk.fdk_last_error()
    o = fdk.fdk_opts()
    o.matrices_on_device = 1
    st = lib.fdk_backproject_host(ctypes.c_void_p(256), d, f3, f3, ctypes.c_void_p(256), det, m, 1,
                                  ctypes.byref(o))
    assert st == fdk.FDK_ERR_INVALID_ARG and "host matrices" in fdk.fdk_last_error()
    bad = (ctypes.c_int32 * 3)(4, 0, 4)
    st = lib.fdk_backproject_host(ctypes.c_void_p(256), bad, f3, f3, ctypes.c_void_p(256), det, m, 1, None)
    assert st == fdk.FDK_ERR_INVALID_ARG and "dims" in fdk.fdk_last_error()
    assert lib.fdk_backproject_host(ctypes.c_void_p(256), d, f3, f3, None, det, m, 0, None) == fdk.FDK_OK


def test_microbench_validates_before_cuda():
    lib = _raw()
    out = ctypes.c_double(0.0)
    for which, param, msg in [(fdk.MICRO_LDG, 3, "divide 32"), (fdk.MICRO_LDS, 0, "divide 32"),
                              (fdk.MICRO_TLD4, 1, "texture size"), (fdk.MICRO_CHASE, 0, "ring"),
                              (42, 1, "unknown")]:
        assert lib.fdk_microbench(which, param, ctypes.byref(out)) == fdk.FDK_ERR_INVALID_ARG
        assert msg in fdk.fdk_last_error()
    assert lib.fdk_microbench(fdk.MICRO_RCP, 0, None) == fdk.FDK_ERR_INVALID_ARG


def test_staged_fetch_checks_before_cuda():
    """The staged path's own requirements are checked on the host: tile 0
    only, rows of a multiple of 16 bytes (W a multiple of 4 for FP32, of 8 for
    BF16 / FP16) and a 16-byte aligned image base."""
    for field, val, kw, msg in [("proj_dtype", fdk.FDK_BF16, dict(det=(12, 8)), "W % 8"),
                                ("tile", 2, {}, "tile 0"),
                                (None, None, dict(det=(10, 8)), "W % 4")]:
        o = fdk.fdk_opts()
        o.fetch = fdk.FETCH_STAGE
        if field:
            setattr(o, field, val)
        st = _call_bp(opts=o, **kw)
        assert st != fdk.FDK_OK and msg in fdk.fdk_last_error(), (field, fdk.fdk_last_error())


def test_host_memory_is_refused_no_cpu_fallback():
    """The device entry points never compute on the host: CPU tensors are
    refused by the library's pointer check (here, without a GPU, the check
    itself cannot succeed), and the call raises instead of falling back."""
    import numpy as np
    import torch
    vol = torch.zeros((4, 4, 4), dtype=torch.float32)
    proj = torch.ones((1, 8, 8), dtype=torch.float32)
    mats = np.eye(3, 4, dtype=np.float32).reshape(1, 12)
    with pytest.raises(fdk.FdkError) as e:
        fdk.fdk_backproject(vol, proj, mats, (1, 1, 1), (0, 0, 0), stream=0)
    assert e.value.status == fdk.FDK_ERR_INVALID_ARG and "volume" in str(e.value)
    with pytest.raises(fdk.FdkError) as e:
        fdk.fdk_forwardproject_adjoint(proj, vol, mats, (1, 1, 1), (0, 0, 0), stream=0)
    assert e.value.status == fdk.FDK_ERR_INVALID_ARG
    assert float(vol.abs().sum()) == 0.0 and float(proj.sum()) == 64.0   # nothing written


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """With no library and no way to build one, the first call raises; the
    binding has nothing to fall back on."""
    monkeypatch.setattr(fdk, "_lib", None)
    monkeypatch.setattr(fdk_build, "OUT", str(tmp_path / "_build"))
    monkeypatch.setattr(fdk_build, "LIB", str(tmp_path / "_build" / "libfdk.so"))

    def no_nvcc():
        raise RuntimeError("nvcc not found")
    monkeypatch.setattr(fdk_build, "nvcc", no_nvcc)
    with pytest.raises(RuntimeError, match="nvcc not found"):
        fdk.fdk_version()
    assert fdk._lib is None


def _geom_args(dims=(4, 4, 4), det=(8, 8)):
    return ((ctypes.c_int32 * 3)(*dims), (ctypes.c_float * 3)(1, 1, 1), (ctypes.c_float * 3)(0, 0, 0),
            (ctypes.c_int32 * 2)(*det), (ctypes.c_float * 12)(*([1.0] * 12)))


def test_adjoint_and_count_validate_before_cuda():
    lib = _raw()
    d, vs, org, det, m = _geom_args()
    o = fdk.fdk_opts()
    o.proj_dtype = fdk.FDK_BF16
    st = lib.fdk_forwardproject_adjoint(ctypes.c_void_p(256), det, ctypes.c_void_p(256), d, vs, org, m, 1,
                                        ctypes.byref(o))
    assert st == fdk.FDK_ERR_INVALID_ARG and "FP32" in fdk.fdk_last_error()
    st = lib.fdk_forwardproject_adjoint(ctypes.c_void_p(256), det, None, d, vs, org, m, 1, None)
    assert st == fdk.FDK_ERR_INVALID_ARG and "volume" in fdk.fdk_last_error()
    bad = (ctypes.c_int32 * 3)(4, 4, 0)
    st = lib.fdk_forwardproject_adjoint(ctypes.c_void_p(256), det, ctypes.c_void_p(256), bad, vs, org, m, 1, None)
    assert st == fdk.FDK_ERR_INVALID_ARG and "dims" in fdk.fdk_last_error()
    assert lib.fdk_forwardproject_adjoint(None, det, ctypes.c_void_p(256), d, vs, org, m, 0, None) == fdk.FDK_OK
    st = lib.fdk_count_updates(None, d, vs, org, det, m, 1, None)
    assert st == fdk.FDK_ERR_INVALID_ARG and "count" in fdk.fdk_last_error()
    cnt = ctypes.c_int64(-1)
    assert lib.fdk_count_updates(ctypes.byref(cnt), d, vs, org, det, m, 0, None) == fdk.FDK_OK
    assert cnt.value == 0


def test_filter_validates_before_cuda():
    lib = _raw()
    m = (ctypes.c_float * 12)(*([1.0] * 12))
    p = ctypes.c_void_p(256)
    for det, n, scale, mats, msg in [((5000, 8), 1, 1.0, m, "4096"), ((0, 8), 1, 1.0, m, "det"),
                                     ((64, 8), -1, 1.0, m, "n_views"),
                                     ((64, 8), 1, float("inf"), m, "scale"),
                                     ((64, 8), 1, 1.0, None, "null"),
                                     ((64, 8), 1, 1.0, (ctypes.c_float * 12)(*([1.0] * 8 + [0.0] * 4)),
                                      "not a camera")]:
        st = lib.fdk_preweight_filter(p, p, (ctypes.c_int32 * 2)(*det), mats, n, scale, None)
        assert st == fdk.FDK_ERR_INVALID_ARG and msg in fdk.fdk_last_error(), (det, n, scale, fdk.fdk_last_error())
    assert lib.fdk_preweight_filter(p, p, (ctypes.c_int32 * 2)(64, 8), m, 0, 1.0, None) == fdk.FDK_OK


def test_batch_plan_validates_before_cuda():
    lib = _raw()
    plan = ctypes.c_void_p(0)
    sc = fdk.fdk_scan()
    sc.volume, sc.projections = 256, 256
    sc.dims[:] = (4, 4, 4)
    sc.voxel_size[:] = (1, 1, 1)
    sc.det[:] = (8, 8)
    mats = (ctypes.c_float * 12)(*([1.0] * 12))
    sc.matrices = ctypes.cast(mats, ctypes.c_void_p).value
    sc.n_views = 1
    assert lib.fdk_batch_plan_create(None, ctypes.byref(sc), 1, None) == fdk.FDK_ERR_INVALID_ARG
    for field, val, msg in [("proj_dtype", fdk.FDK_F16, "FP32"), ("fetch", fdk.FETCH_STAGE, "LDG"),
                            ("matrices_on_device", 1, "host matrices"), ("tile", 6, "tile"),
                            ("autotune", 2, "autotune")]:
        o = fdk.fdk_opts()
        setattr(o, field, val)
        st = lib.fdk_batch_plan_create(ctypes.byref(plan), ctypes.byref(sc), 1, ctypes.byref(o))
        assert st == fdk.FDK_ERR_INVALID_ARG and msg in fdk.fdk_last_error(), (field, fdk.fdk_last_error())
        assert not plan.value
    assert lib.fdk_batch_plan_create(ctypes.byref(plan), ctypes.byref(sc), 0, None) == fdk.FDK_ERR_INVALID_ARG
    sc.dims[1] = 0
    st = lib.fdk_batch_plan_create(ctypes.byref(plan), ctypes.byref(sc), 1, None)
    assert st == fdk.FDK_ERR_INVALID_ARG and "scan 0: dims" in fdk.fdk_last_error()
    sc.dims[1] = 4
    sc.volume = None
    st = lib.fdk_batch_plan_create(ctypes.byref(plan), ctypes.byref(sc), 1, None)
    assert st == fdk.FDK_ERR_INVALID_ARG and "null buffer" in fdk.fdk_last_error()
    assert lib.fdk_backproject_batched(ctypes.byref(sc), 0, None) == fdk.FDK_ERR_INVALID_ARG


def test_static_entry_point_validates_before_cuda():
    """The allocation-free variant refuses other fetch paths and detectors
    whose quad image exceeds its fixed array, before any CUDA call."""
    lib = _raw()
    d, vs, org, det, m = _geom_args()
    o = fdk.fdk_opts()
    o.fetch = fdk.FETCH_LDG
    st = lib.fdk_backproject_static(ctypes.c_void_p(256), d, vs, org, ctypes.c_void_p(256), det, m, 1,
                                    ctypes.byref(o))
    assert st == fdk.FDK_ERR_INVALID_ARG and "FDK_FETCH_QUAD" in fdk.fdk_last_error()
    big = (ctypes.c_int32 * 2)(2600, 2600)          # (W+3)(H+3) * 16 B = 108 MB > 64 MiB
    st = lib.fdk_backproject_static(ctypes.c_void_p(256), d, vs, org, ctypes.c_void_p(256), big, m, 1, None)
    assert st == fdk.FDK_ERR_INVALID_ARG and "static staging array" in fdk.fdk_last_error()
    o = fdk.fdk_opts()
    o.proj_dtype = fdk.FDK_F16                     # 8 B cells: 54 MB fits
    st = lib.fdk_backproject_static(ctypes.c_void_p(256), d, vs, org, ctypes.c_void_p(256), big, m, 0,
                                    ctypes.byref(o))
    # past the size check: a zero-view call only does the set-up (the array's
    # device address), which needs a device
    assert st != fdk.FDK_ERR_INVALID_ARG
    import torch
    if not torch.cuda.is_available():
        assert st == fdk.FDK_ERR_CUDA and "cudaGetDevice" in fdk.fdk_last_error()


def test_host_entry_point_retries_failed_setup():
    """Without a GPU, the host-buffer path gets through its argument checks
    and fails creating its copy stream.  A second call must try that set-up
    again and fail the same way, rather than run on with the null handles
    the first call left in its cache."""
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a CUDA device")
    lib = _raw()
    vol = np.zeros((4, 4, 4), np.float32)
    proj = np.ones((1, 8, 8), np.float32)
    d, vs, org, det, m = _geom_args()
    for _ in range(2):
        st = lib.fdk_backproject_host(vol.ctypes.data, d, vs, org, proj.ctypes.data, det, m, 1, None)
        assert st == fdk.FDK_ERR_CUDA and "copy stream creation failed" in fdk.fdk_last_error()
    assert not vol.any()


def test_count_reports_a_failed_buffer_allocation():
    """Without a GPU the clipped count gets through its argument checks and
    its device buffer cannot be allocated: the failure is a CUDA error (not
    out of memory), named in the message, and *count stays 0."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a CUDA device")
    lib = _raw()
    d, vs, org, det, m = _geom_args()
    cnt = ctypes.c_int64(-1)
    st = lib.fdk_count_updates(ctypes.byref(cnt), d, vs, org, det, m, 1, None)
    assert st == fdk.FDK_ERR_CUDA and "count buffer" in fdk.fdk_last_error()
    assert cnt.value == 0


def test_python_binding_refuses_tensors_on_two_devices():
    """The library launches on the current device, so the binding runs each
    call with its tensors' device current and refuses tensors that live on
    different devices before any library call."""
    from types import SimpleNamespace
    import torch
    a = SimpleNamespace(is_cuda=True, device=torch.device("cuda", 0))
    b = SimpleNamespace(is_cuda=True, device=torch.device("cuda", 1))
    host = SimpleNamespace(is_cuda=False, device=torch.device("cpu"))
    with pytest.raises(ValueError, match="different devices"):
        fdk._device_of(a, b)
    assert fdk._device_of(a, host, None) == torch.device("cuda", 0)
    assert fdk._device_of(host, None) is None


def test_testing_hooks_validate_and_inject_allocation_failures():
    """fdk_testing_fail_allocations makes the library's next allocation fail
    as on a device out of memory: the clipped count, which allocates its
    result word on every call, reports FDK_ERR_OOM.  The injection is used
    up by that one call: without a GPU the next call fails for real, with a
    CUDA error."""
    import torch
    lib = _raw()
    assert lib.fdk_testing_fail_allocations(-1) == fdk.FDK_ERR_INVALID_ARG
    assert lib.fdk_testing_set_wait_limit(0) == fdk.FDK_OK
    assert lib.fdk_testing_set_wait_limit(-1) == fdk.FDK_OK
    if torch.cuda.is_available():
        pytest.skip("the second half needs a machine without a CUDA device")
    d, vs, org, det, m = _geom_args()
    cnt = ctypes.c_int64(-1)
    assert lib.fdk_testing_fail_allocations(1) == fdk.FDK_OK
    st = lib.fdk_count_updates(ctypes.byref(cnt), d, vs, org, det, m, 1, None)
    assert st == fdk.FDK_ERR_OOM and "count buffer" in fdk.fdk_last_error()
    st = lib.fdk_count_updates(ctypes.byref(cnt), d, vs, org, det, m, 1, None)
    assert st == fdk.FDK_ERR_CUDA
    assert lib.fdk_testing_fail_allocations(0) == fdk.FDK_OK
