"""GPU parity of the staged fetch path (FDK_FETCH_STAGE) through the C ABI.

The staged path reads each tile's taps from a shared-memory copy of its
footprint that the tensor-memory accelerator fills (zeros outside the image).
Its arithmetic is that of the global-load path on the same tap values, so
besides matching the FP64 oracle within the accuracy bar it must equal the
LDG path with the same 16 x 16 x 16 tiles (tile variant 7) bit for bit.
Every run ends with fdk_device_status(), which fails if a bounded wait in
the kernel gave up.
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
LDG_SAME_TILE = 7      # 16 x 16 x 16, the staged path's tile


def _bp(scan, fetch, proj=None, mats=None, tile=0):
    p = scan["proj"] if proj is None else proj
    dims = scan["dims"]
    vol = torch.zeros((int(dims[2]), int(dims[1]), int(dims[0])), dtype=torch.float32, device="cuda")
    fdk.fdk_backproject(vol, p, scan["mats"] if mats is None else mats, scan["voxel_size"],
                        scan["origin"], fetch=fetch, tile=tile)
    fdk.fdk_device_status()
    return vol


def _oracle(scan):
    return oracle.backproject(scan["proj"].float().cpu().numpy(), scan["mats"], scan["dims"],
                              scan["voxel_size"], scan["origin"], threads=NCPU)


def _check(scan, what, mats=None):
    got = _bp(scan, fdk.FETCH_STAGE, mats=mats)
    ldg = _bp(scan, fdk.FETCH_LDG, mats=mats, tile=LDG_SAME_TILE)
    assert_parity(_oracle(scan), got.cpu().numpy(), what=what)
    assert torch.equal(got, ldg), f"{what}: staged != LDG (max diff {float((got - ldg).abs().max()):.3e})"


def test_ragged():
    s = synth.make_scan(synth.preset("small", nx=37, ny=29, nz=21), device="cuda")
    _check(s, "ragged 37x29x21")


def test_boundary_tiles_field_larger_than_detector():
    """A 480 mm volume whose footprint overruns the 64 x 48 detector: most
    tiles are boundary tiles, whose boxes extend past the image edge and are
    zero-filled by the copy."""
    s = synth.make_scan(synth.preset("small", nx=48, ny=48, nz=24, voxel=10.0), device="cuda")
    _check(s, "boundary-heavy")


@pytest.mark.parametrize("device_mats", [False, True])
def test_more_views_than_one_pass(device_mats):
    s = synth.make_scan(synth.preset("small", n_views=600, det_w=40, det_h=32, nx=20, ny=18, nz=10),
                        device="cuda")
    mats = torch.from_numpy(s["mats"]).cuda() if device_mats else None
    _check(s, "600 views", mats=mats)


def test_source_inside_volume():
    """Tiles that straddle the source plane keep the checked global-load path
    next to staged tiles."""
    s = synth.make_scan(synth.preset("small", nx=40, ny=40, nz=8, voxel=10.0, sid=150.0, sdd=300.0),
                        device="cuda")
    _check(s, "source inside")


def test_orthographic_identity_exact():
    """w = 1, u = x, v = y: each z slice is a copy of the image (zero past
    the detector edge, where the boxes read the copy's fill)."""
    rng = np.random.default_rng(0)
    W, H = 72, 50
    img = torch.from_numpy(rng.standard_normal((1, H, W)).astype(np.float32)).cuda()
    P = np.zeros((1, 12), np.float32)
    P[0, 0] = 1.0
    P[0, 5] = 1.0
    P[0, 11] = 1.0
    vol = torch.zeros((9, 60, 80), device="cuda")
    fdk.fdk_backproject(vol, img, P, (1, 1, 1), (0, 0, 0), fetch=fdk.FETCH_STAGE)
    fdk.fdk_device_status()
    v = vol.cpu().numpy()
    for z in range(9):
        np.testing.assert_allclose(v[z, :H, :W], img[0].cpu().numpy(), rtol=0, atol=1e-6)
        assert np.all(v[z, H:, :] == 0) and np.all(v[z, :, W:] == 0)


def test_full_128_cube_496_views():
    """The 128^3 x 496-view, 1248 x 960 workload, whole volume."""
    s = synth.make_scan(synth.PRESETS["fdk128"], device="cuda")
    _check(s, "fdk128")


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_half_storage_staged_equals_ldg_and_oracle(dtype):
    """16-bit images are staged as 16-bit boxes (half the bytes, twice the
    pixels per stage) and widened to FP32 on each tap read: the result equals
    the LDG path's on the same stored values bit for bit, and the oracle's
    given those values within the accuracy bar; AUTO stages them."""
    s = synth.make_scan(synth.preset("fdk512", nx=96, ny=80, nz=64, n_views=40, seed=71), device="cuda")
    p16 = s["proj"].to(dtype)
    got = _bp(s, fdk.FETCH_STAGE, proj=p16)
    ldg = _bp(s, fdk.FETCH_LDG, proj=p16, tile=LDG_SAME_TILE)
    assert torch.equal(got, ldg), float((got - ldg).abs().max())
    auto = _bp(s, fdk.FETCH_AUTO, proj=p16)
    assert torch.equal(got, auto)
    ref = oracle.backproject(p16.float().cpu().numpy(), s["mats"], s["dims"], s["voxel_size"], s["origin"],
                             threads=NCPU)
    assert_parity(ref, got.cpu().numpy(), what=f"staged {dtype}")


def test_512_cube_equals_ldg_bitwise():
    """The 512^3 x 496-view workload: the staged result equals the LDG
    result with the same tiles bit for bit, and its sampled parity against
    the oracle is tested with the benchmark's launch configuration (AUTO)."""
    s = synth.make_scan(synth.PRESETS["fdk512"], device="cuda")
    got = _bp(s, fdk.FETCH_STAGE)
    ldg = _bp(s, fdk.FETCH_LDG, tile=LDG_SAME_TILE)
    assert torch.equal(got, ldg), float((got - ldg).abs().max())


def test_sampled_1024_cube_fp32():
    """The 1024^3 x 496-view workload with FP32 projections, which AUTO runs
    on the staged path: 4000 seeded random voxels, a strided 32^3 sub-grid
    and the eight corners are checked one by one against the oracle, and
    the whole volume equals the LDG result with the same tiles bit for bit."""
    cfg = synth.PRESETS["fdk1024"]
    s = synth.make_scan(cfg, device="cuda")
    got = _bp(s, fdk.FETCH_AUTO)
    n = cfg.nx
    g32 = np.arange(5, n, 32)
    zz, yy, xx = np.meshgrid(g32, g32, g32, indexing="ij")
    corners = [[(c & 1) * (n - 1), ((c >> 1) & 1) * (n - 1), ((c >> 2) & 1) * (n - 1)] for c in range(8)]
    xyz = np.concatenate([np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1),
                          np.random.default_rng(1024).integers(0, n, size=(4000, 3)),
                          np.array(corners)]).astype(np.int64)
    proj = s["proj"].cpu().numpy()
    import concurrent.futures as cf
    chunks = np.array_split(np.arange(len(xyz)), NCPU)
    with cf.ThreadPoolExecutor(NCPU) as ex:
        ref = np.concatenate(list(ex.map(lambda idx: oracle.backproject_voxels(
            proj, s["mats"], s["voxel_size"], s["origin"], xyz[idx]), chunks)))
    g = got[xyz[:, 2], xyz[:, 1], xyz[:, 0]].cpu().numpy().astype(np.float64)
    peak = float(np.abs(ref).max())
    err = float(np.abs(g - ref).max())
    assert np.all(np.isfinite(g))
    assert err <= 1e-4 * peak, f"max|diff| {err:.3e} > 1e-4 * {peak:.3e}"
    ldg = _bp(s, fdk.FETCH_LDG, tile=LDG_SAME_TILE)
    assert torch.equal(got, ldg), float((got - ldg).abs().max())


def test_two_streams():
    s = synth.make_scan(synth.preset("small", nx=37, ny=29, nz=21), device="cuda")
    p2 = (s["proj"] * -0.5).contiguous()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    v1 = torch.zeros((21, 29, 37), device="cuda")
    v2 = torch.zeros_like(v1)
    torch.cuda.synchronize()
    for _ in range(3):
        with torch.cuda.stream(s1):
            fdk.fdk_backproject(v1, s["proj"], s["mats"], s["voxel_size"], s["origin"], fetch=fdk.FETCH_STAGE)
        with torch.cuda.stream(s2):
            fdk.fdk_backproject(v2, p2, s["mats"], s["voxel_size"], s["origin"], fetch=fdk.FETCH_STAGE)
    fdk.fdk_device_status()
    ref = _oracle(s)
    assert_parity(3 * ref, v1.cpu().numpy())
    assert_parity(-1.5 * ref, v2.cpu().numpy())


def test_rejections():
    s = synth.make_scan(synth.preset("small", nx=8, ny=8, nz=8, det_w=66), device="cuda")
    vol = torch.zeros((8, 8, 8), device="cuda")
    args = (s["mats"], s["voxel_size"], s["origin"])
    with pytest.raises(fdk.FdkError, match="W % 4"):
        fdk.fdk_backproject(vol, s["proj"], *args, fetch=fdk.FETCH_STAGE)
    s = synth.make_scan(synth.preset("small", nx=8, ny=8, nz=8), device="cuda")
    args = (s["mats"], s["voxel_size"], s["origin"])
    with pytest.raises(fdk.FdkError, match="tile 0"):
        fdk.fdk_backproject(vol, s["proj"], *args, fetch=fdk.FETCH_STAGE, tile=2)
    s68 = synth.make_scan(synth.preset("small", nx=8, ny=8, nz=8, det_w=68), device="cuda")
    with pytest.raises(fdk.FdkError, match="W % 8"):               # 16-bit rows of 136 bytes
        fdk.fdk_backproject(vol, s68["proj"].to(torch.bfloat16), s68["mats"], s68["voxel_size"], s68["origin"],
                            fetch=fdk.FETCH_STAGE)
    flat = torch.zeros(s["proj"].numel() + 1, device="cuda")
    shifted = flat[1:].view(s["proj"].shape)          # 4-byte but not 16-byte aligned
    shifted.copy_(s["proj"])
    with pytest.raises(fdk.FdkError, match="aligned"):
        fdk.fdk_backproject(vol, shifted, *args, fetch=fdk.FETCH_STAGE)
    fdk.fdk_device_status()
