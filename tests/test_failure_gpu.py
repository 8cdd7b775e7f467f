"""Failure paths on the GPU, driven by the library's testing hooks
(include/fdk_testing.h) rather than by a fault.

* A bounded device-side wait that gives up: with a poll limit of 0 every
  consumer wait of the staged back-projection, and of the row filter's
  staged rows, gives up without polling.  The CTA records the timeout, waits
  (with the full limit) for its copies in flight and returns with its tile or
  rows unwritten; fdk_device_status() reports FDK_ERR_TIMEOUT once, and the
  next normal call gives the right result.
* A device allocation that fails: the library's next allocation fails as on
  a device out of memory; the call reports FDK_ERR_OOM, and a retry
  allocates again and gives the right result.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import assert_parity
from paper_1401_3615_gb300 import fdk

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1
SENTINEL = 7.0


@pytest.fixture(autouse=True)
def _restore_hooks():
    yield
    fdk.fdk_testing_set_wait_limit(-1)
    fdk.fdk_testing_fail_allocations(0)


@pytest.fixture(scope="module")
def fine():
    """0.5 mm voxels on the 1248 x 960 detector (the pitch of the 512^3
    workload), a 64 x 64 x 48 block, 24 views: the staged path applies and
    the block has 4 x 4 x 3 tiles of 16^3."""
    cfg = synth.preset("fdk512", nx=64, ny=64, nz=48, n_views=24)
    s = synth.make_scan(cfg, device="cuda")
    ref = oracle.backproject(s["proj"].cpu().numpy(), s["mats"], s["dims"], s["voxel_size"], s["origin"],
                             threads=NCPU)
    return s, ref


def _status():
    try:
        fdk.fdk_device_status()
        return fdk.FDK_OK
    except fdk.FdkError as e:
        return e.status


def test_staged_wait_gives_up_then_recovers(fine):
    """Device matrices, so that each tile is one CTA of one launch over all
    views (host matrices split the views into two launches by ray
    orientation)."""
    s, ref = fine
    shape = ref.shape
    mats = torch.from_numpy(np.ascontiguousarray(s["mats"].reshape(-1, 12))).cuda()
    vol = torch.full(shape, SENTINEL, device="cuda")
    fdk.fdk_testing_set_wait_limit(0)
    fdk.fdk_backproject(vol, s["proj"], mats, s["voxel_size"], s["origin"], fetch=fdk.FETCH_STAGE)
    fdk.fdk_testing_set_wait_limit(-1)
    assert _status() == fdk.FDK_ERR_TIMEOUT
    assert "gave up" in fdk.fdk_last_error()
    assert _status() == fdk.FDK_OK          # the record is cleared once reported
    got = vol.cpu().numpy().astype(np.float64)
    # every 16^3 tile is either untouched (its CTA gave up on its first
    # staged view) or complete (it had no staged view to wait for)
    untouched = 0
    for z0 in range(0, shape[0], 16):
        for y0 in range(0, shape[1], 16):
            for x0 in range(0, shape[2], 16):
                t = got[z0:z0 + 16, y0:y0 + 16, x0:x0 + 16]
                r = ref[z0:z0 + 16, y0:y0 + 16, x0:x0 + 16]
                if np.all(t == SENTINEL):
                    untouched += 1
                else:
                    assert np.abs(t - SENTINEL - r).max() <= 1e-4 * np.abs(ref).max(), (z0, y0, x0)
    assert untouched > 0
    # the next call, with the built-in limit, is complete and correct
    vol.zero_()
    fdk.fdk_backproject(vol, s["proj"], mats, s["voxel_size"], s["origin"], fetch=fdk.FETCH_STAGE)
    assert _status() == fdk.FDK_OK
    assert_parity(ref, vol.cpu().numpy(), what="staged, after a timeout")


def test_filter_wait_gives_up_then_recovers():
    cfg = synth.preset("small", n_views=3, det_w=1248, det_h=6, pixel=0.308)
    geo = synth.geometry(cfg)
    raw = synth.projections(cfg, geo, synth.phantom(cfg), device="cuda", filtered=False)
    out = torch.full_like(raw, SENTINEL)
    fdk.fdk_testing_set_wait_limit(0)
    fdk.fdk_preweight_filter(out, raw, geo["mats"], scale=1.0)
    fdk.fdk_testing_set_wait_limit(-1)
    assert _status() == fdk.FDK_ERR_TIMEOUT
    # every CTA waits for its first row pair, so nothing was written
    assert torch.all(out == SENTINEL)
    fdk.fdk_preweight_filter(out, raw, geo["mats"], scale=1.0)
    assert _status() == fdk.FDK_OK
    ref = oracle.preweight_filter(raw.cpu().numpy(), geo["mats"])
    assert_parity(ref, out.cpu().numpy(), rel_tol=3e-5, psnr_min=100.0, what="filter, after a timeout")


def test_count_allocation_failure_then_retry(fine):
    s, _ = fine
    args = (s["dims"], (s["cfg"].det_w, s["cfg"].det_h), s["mats"], s["voxel_size"], s["origin"])
    expect = fdk.fdk_count_updates(*args)
    fdk.fdk_testing_fail_allocations(1)
    with pytest.raises(fdk.FdkError) as e:
        fdk.fdk_count_updates(*args)
    assert e.value.status == fdk.FDK_ERR_OOM and "count buffer" in str(e.value)
    assert fdk.fdk_count_updates(*args) == expect


@pytest.mark.parametrize("what", ["staged error word", "quad staging", "host-path buffers"])
def test_allocation_failure_then_retry(fine, what):
    """After fdk_release() the next call must allocate its cached device
    buffers again; the first of those allocations fails, the call reports
    FDK_ERR_OOM and enqueues nothing that writes the volume; the retry
    allocates and is correct."""
    s, ref = fine
    torch.cuda.synchronize()
    fdk.fdk_release()
    vol = torch.zeros(ref.shape, device="cuda")

    def call(v):
        if what == "staged error word":
            fdk.fdk_backproject(v, s["proj"], s["mats"], s["voxel_size"], s["origin"], fetch=fdk.FETCH_STAGE)
        elif what == "quad staging":
            fdk.fdk_backproject(v, s["proj"], s["mats"], s["voxel_size"], s["origin"], fetch=fdk.FETCH_QUAD)
        else:
            h = torch.zeros(ref.shape)
            fdk.fdk_backproject_host(h, s["proj"].cpu(), s["mats"], s["voxel_size"], s["origin"],
                                     overwrite=True)
            v.copy_(h)

    fdk.fdk_testing_fail_allocations(1)
    with pytest.raises(fdk.FdkError) as e:
        call(vol)
    assert e.value.status == fdk.FDK_ERR_OOM, str(e.value)
    torch.cuda.synchronize()
    assert not torch.any(vol != 0)
    call(vol)
    torch.cuda.synchronize()
    assert _status() == fdk.FDK_OK
    assert_parity(ref, vol.cpu().numpy(), what=f"{what}, retry after a failed allocation")
