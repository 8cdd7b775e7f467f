"""GPU parity past 2^31 voxels: the 64-bit volume offsets of every path
that reads or writes the volume.

A 2048 x 2048 x 520 volume of 0.125 mm voxels holds 2.18e9 voxels (8.7 GB
in FP32): from slice z = 512 on, a voxel's flat index exceeds 2^31.  Eight
views of the 1248 x 960 C-arm scan keep each call short.  The back-projection
(staged and LDG paths, and the host-buffer schedule, whose slabs start past
2^31 elements) is checked voxel by voxel against the oracle on a seeded
sample that includes the last slices and the far corners; the adjoint reads
a volume that is zero except for two Gaussian blocks, one across the 2^31
boundary and one in the far corner, so its result is the oracle's transpose
of those blocks alone (Listing 1, Sec. IV, and its transpose).
"""
import concurrent.futures as cf
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
CFG = synth.preset("fdk512", nx=2048, ny=2048, nz=520, voxel=0.125, n_views=8, seed=2048)
LDG_SAME_TILE = 7      # 16 x 16 x 16, the staged path's tile


@pytest.fixture(scope="module")
def scan():
    s = synth.make_scan(CFG, device="cuda")
    assert CFG.nx * CFG.ny * CFG.nz > 2 ** 31
    yield s
    torch.cuda.empty_cache()


def _bp(s, fetch, tile=0):
    vol = torch.zeros((CFG.nz, CFG.ny, CFG.nx), dtype=torch.float32, device="cuda")
    fdk.fdk_backproject(vol, s["proj"], s["mats"], s["voxel_size"], s["origin"], fetch=fetch, tile=tile)
    fdk.fdk_device_status()
    return vol


def _sample():
    """Seeded voxels: random ones, a strided grid of the last 8 slices (all
    past 2^31), the 8 corners and a run across the 2^31 boundary."""
    rng = np.random.default_rng(31)
    n, nz = CFG.nx, CFG.nz
    rand = np.stack([rng.integers(0, n, 3000), rng.integers(0, n, 3000), rng.integers(0, nz, 3000)], 1)
    g = np.arange(3, n, 97)
    yy, xx = np.meshgrid(g, g, indexing="ij")
    tail = np.concatenate([np.stack([xx.ravel(), yy.ravel(), np.full(xx.size, z)], 1) for z in range(nz - 8, nz)])
    corners = np.array([[(c & 1) * (n - 1), ((c >> 1) & 1) * (n - 1), ((c >> 2) & 1) * (nz - 1)] for c in range(8)])
    flat = 2 ** 31 + np.arange(-64, 64) * 4099                   # flat indices around 2^31
    across = np.stack([flat % n, (flat // n) % n, flat // (n * n)], 1)
    return np.concatenate([rand, tail, corners, across]).astype(np.int64)


def _oracle_at(s, xyz):
    proj = s["proj"].cpu().numpy()
    chunks = np.array_split(np.arange(len(xyz)), NCPU)
    with cf.ThreadPoolExecutor(NCPU) as ex:
        return np.concatenate(list(ex.map(lambda idx: oracle.backproject_voxels(
            proj, s["mats"], s["voxel_size"], s["origin"], xyz[idx]), chunks)))


def _check_sampled(vol, ref, xyz, what):
    got = vol[xyz[:, 2], xyz[:, 1], xyz[:, 0]].cpu().numpy().astype(np.float64)
    peak = float(np.abs(ref).max())
    err = float(np.abs(got - ref).max())
    assert peak > 0 and np.all(np.isfinite(got))
    assert err <= 1e-4 * peak, f"{what}: max|diff| {err:.3e} > 1e-4 * {peak:.3e}"
    return err / peak


def test_backproject_past_2_31_voxels(scan):
    xyz = _sample()
    ref = _oracle_at(scan, xyz)
    staged = _bp(scan, fdk.FETCH_STAGE)
    print(f"staged: max|diff|/peak {_check_sampled(staged, ref, xyz, 'staged'):.3e} on {len(xyz)} voxels")
    ldg = _bp(scan, fdk.FETCH_LDG, tile=LDG_SAME_TILE)
    assert torch.equal(staged, ldg), float((staged - ldg).abs().max())
    del ldg
    auto = _bp(scan, fdk.FETCH_AUTO)
    assert torch.equal(staged, auto)
    del auto
    # the host-buffer schedule: its last chunk runs as z-slabs whose device
    # and host offsets pass 2^31 elements, and it equals one device call
    host = torch.empty((CFG.nz, CFG.ny, CFG.nx), dtype=torch.float32, pin_memory=True)
    fdk.fdk_backproject_host(host, scan["proj"].cpu().contiguous(), scan["mats"], scan["voxel_size"],
                             scan["origin"], overwrite=True)
    assert torch.equal(host.cuda(), staged)


def test_adjoint_past_2_31_voxels(scan):
    """Two seeded Gaussian blocks in an otherwise zero volume: one across
    the 2^31 boundary (z 500..519), one in the far corner."""
    vs = np.asarray(scan["voxel_size"], dtype=np.float64)
    org = np.asarray(scan["origin"], dtype=np.float64)
    blocks = [((1000, 1000, 500), (40, 32, 20), 1), ((2016, 2016, 504), (32, 32, 16), 2)]
    vol = torch.zeros((CFG.nz, CFG.ny, CFG.nx), dtype=torch.float32, device="cuda")
    W, H = CFG.det_w, CFG.det_h
    ref = np.zeros((CFG.n_views, H, W), dtype=np.float64)
    for (x0, y0, z0), (bx, by, bz), seed in blocks:
        b = synth.gaussian_volume((bx, by, bz), seed=seed)
        vol[z0:z0 + bz, y0:y0 + by, x0:x0 + bx] = torch.from_numpy(b).cuda()
        bo = (org + vs * np.array([x0, y0, z0])).astype(np.float32)
        assert np.all(bo.astype(np.float64) == org.astype(np.float32).astype(np.float64)
                      + vs.astype(np.float32).astype(np.float64) * np.array([x0, y0, z0]))
        oracle.adjoint(b, scan["mats"], (bx, by, bz), scan["voxel_size"], bo, W, H, proj=ref, threads=NCPU)
        last = ((z0 + bz - 1) * CFG.ny + y0 + by - 1) * CFG.nx + x0 + bx - 1
        assert z0 * CFG.nx * CFG.ny < 2 ** 31 < last
    out = torch.zeros((CFG.n_views, H, W), dtype=torch.float32, device="cuda")
    fdk.fdk_forwardproject_adjoint(out, vol, scan["mats"], scan["voxel_size"], scan["origin"])
    fdk.fdk_device_status()
    assert float(np.abs(ref).max()) > 0
    rel, p = assert_parity(ref, out.cpu().numpy(), what="adjoint past 2^31")
    print(f"adjoint: max|diff|/max|q| {rel:.3e}, PSNR {p:.1f} dB")
