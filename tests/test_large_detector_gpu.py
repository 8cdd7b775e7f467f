"""GPU parity on a detector of more than 2^23 pixels.

Below 2^23 pixels (W * (H + 1) < 2^23) the global-load paths form the flat
tap index in FP32 and use its bits as the address offset; from there on the
index is no longer an exact FP32 integer and every path that reads the image
directly (the LDG kernels, the staged kernel's fallback views, the batched
kernel) switches to integer index arithmetic.  A 3072 x 2816 detector
(8.65e6 cells, 0.0625 mm at the isocentre) takes that branch.  Volumes:
- 0.5 mm voxels (8 pixels per voxel) over a field larger than the
  detector's, so interior and boundary tiles both read the image directly;
- 0.25 mm voxels, whose boxes fit a stage;
- 3 mm voxels (48 pixels per voxel), far coarser than the detector.
Each result is compared with the oracle on every voxel (Listing 1, Sec. IV),
the adjoint with the oracle's transpose, and the paths that must agree bit
for bit are compared with each other.
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
W, H = 3072, 2816
PIXEL = 0.308 * 1248.0 / W
LDG_SAME_TILE = 7      # 16 x 16 x 16, the staged path's tile


def _scan(nx, ny, nz, voxel, seed):
    cfg = synth.preset("fdk512", nx=nx, ny=ny, nz=nz, voxel=voxel, n_views=8, det_w=W, det_h=H,
                       pixel=PIXEL, seed=seed)
    assert W * (H + 1) >= 2 ** 23
    return synth.make_scan(cfg, device="cuda")


def _bp(s, proj=None, fetch=fdk.FETCH_AUTO, tile=0):
    d = s["dims"]
    vol = torch.zeros((int(d[2]), int(d[1]), int(d[0])), dtype=torch.float32, device="cuda")
    fdk.fdk_backproject(vol, s["proj"] if proj is None else proj, s["mats"], s["voxel_size"], s["origin"],
                        fetch=fetch, tile=tile)
    fdk.fdk_device_status()
    return vol


def _oracle(s, proj=None):
    p = (s["proj"] if proj is None else proj).float().cpu().numpy()
    return oracle.backproject(p, s["mats"], s["dims"], s["voxel_size"], s["origin"], threads=NCPU)


@pytest.fixture(scope="module")
def coarse():
    s = _scan(416, 400, 368, 0.5, 3070)
    s["ref"] = _oracle(s)
    return s


@pytest.fixture(scope="module")
def very_coarse():
    return _scan(80, 72, 48, 3.0, 3072)


@pytest.fixture(scope="module")
def fine():
    return _scan(64, 64, 48, 0.25, 2816)


@pytest.mark.parametrize("fetch,tile", [(fdk.FETCH_AUTO, 0), (fdk.FETCH_LDG, 0), (fdk.FETCH_LDG, LDG_SAME_TILE),
                                        (fdk.FETCH_TEX, 0), (fdk.FETCH_STAGE, 0)])
def test_coarse_volume(coarse, fetch, tile):
    """FETCH_STAGE here runs the staged kernel with most boxes too large for
    a stage, so its views fall back to its own direct reads."""
    got = _bp(coarse, fetch=fetch, tile=tile).cpu().numpy()
    rel, p = assert_parity(coarse["ref"], got, what=f"fetch {fetch} tile {tile}")
    print(f"fetch {fetch} tile {tile}: max|diff|/max|f| {rel:.3e}, PSNR {p:.1f} dB")


def test_very_coarse_volume(very_coarse):
    """48 pixels per voxel.  The default options (here the 8-voxel z-run of
    LDG tile variant 0) and the texture path meet the bar.  The 16-voxel
    z-run variant (tile 7, the staged path's tiling) does not: its FP32
    detector positions, relative to a cell up to 400 pixels away and stepped
    along the run, carry about 1e-4 pixel of rounding, and on a detector this
    fine against the voxel that moves the result by about 2e-4 of its peak
    (measured 2.07e-4, 114.7 dB).  That variant is held to the bound its
    arithmetic gives here, 4e-4 and 100 dB.  (The staged path itself never
    sees such a footprint: its boxes are at most 128 pixels wide.)"""
    ref = _oracle(very_coarse)
    for fetch, tile in ((fdk.FETCH_AUTO, 0), (fdk.FETCH_LDG, 0), (fdk.FETCH_TEX, 0)):
        got = _bp(very_coarse, fetch=fetch, tile=tile).cpu().numpy()
        rel, p = assert_parity(ref, got, what=f"fetch {fetch} tile {tile}")
        print(f"48 px/voxel, fetch {fetch} tile {tile}: max|diff|/max|f| {rel:.3e}, PSNR {p:.1f} dB")
    got = _bp(very_coarse, fetch=fdk.FETCH_LDG, tile=LDG_SAME_TILE).cpu().numpy()
    rel, p = assert_parity(ref, got, rel_tol=4e-4, psnr_min=100.0, what="16-voxel z-run")
    print(f"48 px/voxel, 16-voxel z-run: max|diff|/max|f| {rel:.3e}, PSNR {p:.1f} dB")


def test_coarse_volume_half_storage(coarse):
    for dtype in (torch.bfloat16, torch.float16):
        p16 = coarse["proj"].to(dtype)
        got = _bp(coarse, proj=p16, fetch=fdk.FETCH_LDG).cpu().numpy()
        assert_parity(_oracle(coarse, p16), got, what=f"LDG {dtype}")


def test_quad_images_refused(coarse):
    d = coarse["dims"]
    vol = torch.zeros((int(d[2]), int(d[1]), int(d[0])), device="cuda")
    with pytest.raises(fdk.FdkError, match="quad"):
        fdk.fdk_backproject(vol, coarse["proj"], coarse["mats"], coarse["voxel_size"], coarse["origin"],
                            fetch=fdk.FETCH_QUAD)


def test_fine_volume_staged(fine):
    staged = _bp(fine, fetch=fdk.FETCH_STAGE)
    ldg = _bp(fine, fetch=fdk.FETCH_LDG, tile=LDG_SAME_TILE)
    assert torch.equal(staged, ldg), float((staged - ldg).abs().max())
    assert torch.equal(staged, _bp(fine))
    rel, p = assert_parity(_oracle(fine), staged.cpu().numpy(), what="staged")
    print(f"staged: max|diff|/max|f| {rel:.3e}, PSNR {p:.1f} dB")
    for dtype in (torch.bfloat16, torch.float16):
        p16 = fine["proj"].to(dtype)
        s16 = _bp(fine, proj=p16, fetch=fdk.FETCH_STAGE)
        assert torch.equal(s16, _bp(fine, proj=p16, fetch=fdk.FETCH_LDG, tile=LDG_SAME_TILE)), dtype
        assert_parity(_oracle(fine, p16), s16.cpu().numpy(), what=f"staged {dtype}")


def test_adjoint(coarse, fine):
    for s, seed in ((coarse, 5), (fine, 6)):
        x = synth.gaussian_volume(s["dims"], seed=seed)
        out = torch.zeros((8, H, W), dtype=torch.float32, device="cuda")
        fdk.fdk_forwardproject_adjoint(out, torch.from_numpy(x).cuda(), s["mats"], s["voxel_size"], s["origin"])
        fdk.fdk_device_status()
        ref = oracle.adjoint(x, s["mats"], s["dims"], s["voxel_size"], s["origin"], W, H, threads=NCPU)
        rel, p = assert_parity(ref, out.cpu().numpy(), what="adjoint")
        print(f"adjoint: max|diff|/max|q| {rel:.3e}, PSNR {p:.1f} dB")


def test_batch(coarse, fine):
    """Both scans in one batch equal the sequential calls on the plan's paths."""
    scans = []
    for s in (coarse, fine):
        d = s["dims"]
        scans.append((torch.zeros((int(d[2]), int(d[1]), int(d[0])), device="cuda"), s["proj"], s["mats"],
                      s["voxel_size"], s["origin"]))
    plan = fdk.fdk_batch_plan_create(scans)
    plan.execute()
    torch.cuda.synchronize()
    fdk.fdk_device_status()
    for i, (s, sc) in enumerate(zip((coarse, fine), scans)):
        if plan.scan_fetch(i) == fdk.FETCH_STAGE:
            ref = _bp(s, fetch=fdk.FETCH_STAGE)
        else:
            ref = _bp(s, fetch=fdk.FETCH_LDG, tile=plan.tile)
        assert torch.equal(sc[0], ref), (i, float((sc[0] - ref).abs().max()))
    plan.close()
