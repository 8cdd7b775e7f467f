"""The allocation-free entry point, fdk_backproject_static.

Some callers may not allocate device memory at all: host programs that hand
the GPU's memory to their own pool at start-up, reconstruction loops with a
fixed memory budget, plugins inside frameworks that own the device memory.
fdk_backproject_static serves them by staging its quad images in a fixed
64 MiB array inside the library instead of a buffer it allocates.  These
tests call it through the C ABI and check it against fdk_backproject on two
calls in a row (the array is shared by calls and keeps the previous call's
contents, which must not leak into the next result).  The file name sorts
last so that a run stopping at the first failure has run every other test.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import REL_TOL, assert_parity
from paper_1401_3615_gb300 import fdk

pytestmark = pytest.mark.gpu


def _static_call(vol, proj, mats, vs, org, fetch=0):
    """fdk_backproject_static through the raw C ABI (ctypes), default stream.
    ``mats`` is a host array, or a CUDA tensor (device matrices)."""
    lib = fdk._load()
    o = fdk.fdk_opts()
    o.proj_dtype = fdk._DTYPES[proj.dtype]
    o.fetch = fetch
    if isinstance(mats, torch.Tensor):
        o.matrices_on_device = 1
        mptr = ctypes.c_void_p(mats.data_ptr())
    else:
        m = np.ascontiguousarray(np.asarray(mats, dtype=np.float32).reshape(-1, 12))
        mptr = m.ctypes.data_as(ctypes.c_void_p)
    nz, ny, nx = vol.shape
    st = lib.fdk_backproject_static(
        ctypes.c_void_p(vol.data_ptr()), (ctypes.c_int32 * 3)(nx, ny, nz),
        (ctypes.c_float * 3)(*[float(x) for x in vs]), (ctypes.c_float * 3)(*[float(x) for x in org]),
        ctypes.c_void_p(proj.data_ptr()), (ctypes.c_int32 * 2)(proj.shape[2], proj.shape[1]),
        mptr, proj.shape[0], ctypes.byref(o))
    return st


@pytest.mark.parametrize("case", ["multi_pass_small_detector", "full_detector"])
def test_static_matches_allocating_entry_point_twice(case):
    if case == "multi_pass_small_detector":
        # 640 x 480 quad images take 4.97 MB: 13 per pass, 40 views = 4 passes
        cfg = synth.preset("small", nx=40, ny=36, nz=20, voxel=6.0, n_views=40,
                           det_w=640, det_h=480, pixel=0.308 * 1.95)
    else:
        # 1248 x 960 quad images take 19.3 MB: 3 per pass, 7 views = 3 passes
        cfg = synth.preset("fdk128", nx=48, ny=40, nz=24, voxel=4.0, n_views=7)
    s = synth.make_scan(cfg, device="cuda")
    shape = (cfg.nz, cfg.ny, cfg.nx)
    ref = torch.zeros(shape, device="cuda")
    fdk.fdk_backproject(ref, s["proj"], s["mats"], s["voxel_size"], s["origin"])
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    assert np.abs(ref).max() > 0
    for call in range(2):
        # different projections on the first call, so stale staging would show
        proj = s["proj"] if call == 1 else (s["proj"] * 3.0).contiguous()
        vol = torch.zeros(shape, device="cuda")
        assert _static_call(vol, proj, s["mats"], s["voxel_size"], s["origin"]) == fdk.FDK_OK, \
            fdk.fdk_last_error()
        torch.cuda.synchronize()
        got = vol.cpu().numpy()
        expect = ref if call == 1 else 3.0 * ref
        assert_parity(expect, got, rel_tol=REL_TOL, what=f"{case} call {call}")


def test_static_rejects_oversized_detector_and_ldg_fetch():
    vol = torch.zeros((2, 2, 2), device="cuda")
    # 2048 x 2048 FP32 quad image: 2051 * 2051 * 16 B > 64 MiB
    big = torch.zeros((1, 2048, 2048), device="cuda")
    P = np.zeros((1, 12), np.float32)
    P[0, 0] = P[0, 5] = P[0, 11] = 1.0
    assert _static_call(vol, big, P, (1, 1, 1), (0, 0, 0)) == fdk.FDK_ERR_INVALID_ARG
    assert "static staging array" in fdk.fdk_last_error()
    small = torch.zeros((1, 8, 8), device="cuda")
    assert _static_call(vol, small, P, (1, 1, 1), (0, 0, 0), fetch=fdk.FETCH_LDG) == fdk.FDK_ERR_INVALID_ARG
    # the same detector in FP16 (8 B cells) fits
    big16 = torch.zeros((1, 2048, 2048), device="cuda", dtype=torch.float16)
    assert _static_call(vol, big16, P, (1, 1, 1), (0, 0, 0)) == fdk.FDK_OK, fdk.fdk_last_error()
    torch.cuda.synchronize()


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("device_matrices", [False, True])
def test_static_half_storage_and_device_matrices_twice(dtype, device_matrices):
    """FP16/BF16 images (8-byte quad cells) with non-zero values, host or
    device matrices, several passes through the array: equal to the
    allocating entry point on the same stored values, on two calls in a row."""
    # 640 x 480 quad images of 8 B cells take 2.49 MB: 26 per pass, 60 views = 3 passes
    cfg = synth.preset("small", nx=40, ny=36, nz=20, voxel=6.0, n_views=60,
                       det_w=640, det_h=480, pixel=0.308 * 1.95)
    s = synth.make_scan(cfg, device="cuda")
    p16 = s["proj"].to(dtype)
    mats = torch.from_numpy(np.ascontiguousarray(s["mats"].reshape(-1, 12))).cuda() if device_matrices \
        else s["mats"]
    shape = (cfg.nz, cfg.ny, cfg.nx)
    ref = torch.zeros(shape, device="cuda")
    fdk.fdk_backproject(ref, p16, mats, s["voxel_size"], s["origin"], fetch=fdk.FETCH_QUAD)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    assert np.abs(ref).max() > 0
    for call in range(2):
        proj = p16 if call == 1 else (p16 * 2).contiguous()
        vol = torch.zeros(shape, device="cuda")
        assert _static_call(vol, proj, mats, s["voxel_size"], s["origin"]) == fdk.FDK_OK, fdk.fdk_last_error()
        torch.cuda.synchronize()
        expect = ref if call == 1 else 2.0 * ref
        assert_parity(expect, vol.cpu().numpy(), rel_tol=REL_TOL, what=f"{dtype} device={device_matrices} call {call}")


def test_static_against_oracle():
    """The allocation-free entry point against the FP64 oracle directly, on
    a ragged 37 x 29 x 21 volume (FP32 images)."""
    s = synth.make_scan(synth.preset("small", nx=37, ny=29, nz=21), device="cuda")
    ref = oracle.backproject(s["proj"].cpu().numpy(), s["mats"], s["dims"], s["voxel_size"], s["origin"],
                             threads=os.cpu_count() or 1)
    vol = torch.zeros(ref.shape, device="cuda")
    assert _static_call(vol, s["proj"], s["mats"], s["voxel_size"], s["origin"]) == fdk.FDK_OK, \
        fdk.fdk_last_error()
    torch.cuda.synchronize()
    assert_parity(ref, vol.cpu().numpy(), what="static vs oracle")


def test_static_call_allocates_nothing():
    """Once set up on a device (the first call; under CUDA's lazy module
    loading that is when the array itself is allocated), a call leaves the
    device's free memory unchanged."""
    cfg = synth.preset("small", nx=37, ny=29, nz=21)
    s = synth.make_scan(cfg, device="cuda")
    vol = torch.zeros((cfg.nz, cfg.ny, cfg.nx), device="cuda")
    assert _static_call(vol, s["proj"], s["mats"], s["voxel_size"], s["origin"]) == fdk.FDK_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _static_call(vol, s["proj"], s["mats"], s["voxel_size"], s["origin"]) == fdk.FDK_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
