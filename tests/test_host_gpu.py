"""fdk_backproject_host: the back-projection of host buffers through the C
ABI, with the projections copied in chunks of views that overlap the
back-projection of the previous chunk.

One chunk is one fdk_backproject pass, so with fewer than 64 views the
result equals the device entry point bit for bit, also when the volume is
tall enough (nz >= 64) for the last chunk to run as z-slabs that are copied
back one by one.  With more views each chunk is its own pass and the result
matches the FP64 oracle within the accuracy bar.
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


def _oracle(s, proj=None):
    p = (s["proj"] if proj is None else proj).float().cpu().numpy()
    return oracle.backproject(p, s["mats"], s["dims"], s["voxel_size"], s["origin"], threads=NCPU)


def _shape(s):
    return (s["cfg"].nz, s["cfg"].ny, s["cfg"].nx)


def test_one_chunk_equals_device_path_bitwise():
    s = synth.make_scan(synth.preset("small", nx=37, ny=29, nz=21), device="cuda")
    dev = torch.zeros(_shape(s), device="cuda")
    fdk.fdk_backproject(dev, s["proj"], s["mats"], s["voxel_size"], s["origin"])
    host = torch.zeros(_shape(s)).pin_memory()
    fdk.fdk_backproject_host(host, s["proj"].cpu().pin_memory(), s["mats"], s["voxel_size"], s["origin"])
    assert torch.equal(host, dev.cpu())


@pytest.mark.parametrize("fetch", [fdk.FETCH_AUTO, fdk.FETCH_LDG])
def test_one_chunk_in_z_slabs_equals_device_path_bitwise(fetch):
    """80 slices: the single chunk runs as slabs of 32, 32 and 16 slices
    (whole 16-voxel tile layers, exact FP32 slab origins), each copied back
    while the next is computed; the volume equals one device call's."""
    s = synth.make_scan(synth.preset("small", nx=40, ny=36, nz=80, voxel=4.0, n_views=40), device="cuda")
    dev = torch.zeros(_shape(s), device="cuda")
    fdk.fdk_backproject(dev, s["proj"], s["mats"], s["voxel_size"], s["origin"], fetch=fetch)
    for pinned in (True, False):
        host = torch.full(_shape(s), 3.0)
        host = host.pin_memory() if pinned else host
        fdk.fdk_backproject_host(host, s["proj"].cpu().pin_memory(), s["mats"], s["voxel_size"], s["origin"],
                                 fetch=fetch, overwrite=True)
        assert torch.equal(host, dev.cpu()), f"pinned={pinned}"


@pytest.mark.parametrize("pinned", [True, False])
def test_chunks_accumulate_against_oracle(pinned):
    """300 views go in chunks of 19, 38, 76 and 167 views; the host volume
    starts at 0.5 and is accumulated twice."""
    s = synth.make_scan(synth.preset("small", n_views=300, det_w=40, det_h=32, nx=20, ny=18, nz=10))
    ref = _oracle(s)
    vol = torch.full(_shape(s), 0.5)
    proj = s["proj"].float().contiguous()
    if pinned:
        vol, proj = vol.pin_memory(), proj.pin_memory()
    for _ in range(2):
        fdk.fdk_backproject_host(vol, proj, s["mats"], s["voxel_size"], s["origin"])
    assert_parity(2 * ref + 0.5, vol.numpy().astype(np.float64), what=f"pinned={pinned}")


def test_overwrite_replaces_the_host_volume():
    s = synth.make_scan(synth.preset("small", n_views=300, det_w=40, det_h=32, nx=20, ny=18, nz=10))
    ref = _oracle(s)
    vol = torch.full(_shape(s), 7.0).pin_memory()
    fdk.fdk_backproject_host(vol, s["proj"].float().contiguous().pin_memory(), s["mats"], s["voxel_size"],
                             s["origin"], overwrite=True)
    assert_parity(ref, vol.numpy().astype(np.float64), what="overwrite")


def test_full_128_cube_496_views_and_half_storage():
    s = synth.make_scan(synth.PRESETS["fdk128"], device="cuda")
    ref = _oracle(s)
    vol = torch.zeros(_shape(s)).pin_memory()
    fdk.fdk_backproject_host(vol, s["proj"].cpu().pin_memory(), s["mats"], s["voxel_size"], s["origin"])
    assert_parity(ref, vol.numpy().astype(np.float64), what="fdk128 host")
    p16 = s["proj"].to(torch.float16)
    vol16 = torch.zeros(_shape(s)).pin_memory()
    fdk.fdk_backproject_host(vol16, p16.cpu().pin_memory(), s["mats"], s["voxel_size"], s["origin"])
    assert_parity(_oracle(s, proj=p16), vol16.numpy().astype(np.float64), what="fdk128 host fp16")


def test_rejects_device_buffers_and_device_matrices():
    s = synth.make_scan(synth.preset("small", nx=8, ny=8, nz=8), device="cuda")
    with pytest.raises(ValueError):
        fdk.fdk_backproject_host(torch.zeros((8, 8, 8), device="cuda"), s["proj"], s["mats"],
                                 s["voxel_size"], s["origin"])
    with pytest.raises(ValueError):
        fdk.fdk_backproject_host(torch.zeros((8, 8, 8)), s["proj"].cpu(), torch.from_numpy(s["mats"]).cuda(),
                                 s["voxel_size"], s["origin"])
