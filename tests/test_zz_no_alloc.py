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

import numpy as np
import pytest
import torch

import synth
from _helpers import REL_TOL, assert_parity
from paper_1401_3615_gb300 import fdk

pytestmark = pytest.mark.gpu


def _static_call(vol, proj, mats, vs, org, fetch=0):
    """fdk_backproject_static through the raw C ABI (ctypes), default stream."""
    lib = fdk._load()
    o = fdk.fdk_opts()
    o.proj_dtype = fdk._DTYPES[proj.dtype]
    o.fetch = fetch
    m = np.ascontiguousarray(np.asarray(mats, dtype=np.float32).reshape(-1, 12))
    nz, ny, nx = vol.shape
    st = lib.fdk_backproject_static(
        ctypes.c_void_p(vol.data_ptr()), (ctypes.c_int32 * 3)(nx, ny, nz),
        (ctypes.c_float * 3)(*[float(x) for x in vs]), (ctypes.c_float * 3)(*[float(x) for x in org]),
        ctypes.c_void_p(proj.data_ptr()), (ctypes.c_int32 * 2)(proj.shape[2], proj.shape[1]),
        m.ctypes.data_as(ctypes.c_void_p), proj.shape[0], ctypes.byref(o))
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
