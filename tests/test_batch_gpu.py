"""The batched form: many scans of uneven size in one persistent launch.

A batch must equal the same scans back-projected one by one with
fdk_backproject, bit for bit (same per-voxel view order): on the staged path
for the scans the plan stages (FDK_FETCH_AUTO), on the LDG path with the
plan's tile variant for the others; the autotuner must leave the scans'
volumes untouched; the launch must survive CUDA-graph capture and replay;
and one batch is checked against the oracle.
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


def _small_batch(n=12, seed=77):
    rng = np.random.default_rng(seed)
    scans = []
    for i in range(n):
        nx, ny, nz = (int(v) for v in rng.integers(9, 41, size=3))
        views = int(rng.integers(6, 30))
        w, h = int(rng.integers(40, 97)), int(rng.integers(30, 73))
        if i % 2 == 0:
            w -= w % 4          # rows of a multiple of 16 bytes: the staged path applies
        cfg = synth.preset("small", nx=nx, ny=ny, nz=nz, voxel=240.0 / max(nx, ny, nz),
                           n_views=views, det_w=w, det_h=h, pixel=0.308 * 1248.0 / w,
                           seed=int(rng.integers(1, 1 << 30)))
        s = synth.make_scan(cfg, device="cuda")
        vol = torch.zeros((nz, ny, nx), device="cuda")
        vs, org = s["voxel_size"], s["origin"]
        if i % 3 == 1:   # anisotropic pitches and an origin off the isocentre
            vs = (vs * np.array([0.8, 1.0, 1.25], np.float32)).astype(np.float32)
            org = (-(np.array([nx, ny, nz], np.float64) - 1) / 2.0 * vs
                   + rng.uniform(-5.0, 5.0, size=3)).astype(np.float32)
        scans.append((vol, s["proj"], s["mats"], vs, org))
    return scans


def _sequential(scans, tile, init=0.0, plan=None):
    """Each scan by fdk_backproject on the path the plan takes for it (the
    LDG path with ``tile`` when no plan is given)."""
    out = []
    for i, (vol, proj, mats, vs, org) in enumerate(scans):
        v = torch.full_like(vol, init)
        if plan is not None and plan.scan_fetch(i) == fdk.FETCH_STAGE:
            fdk.fdk_backproject(v, proj, mats, vs, org, fetch=fdk.FETCH_STAGE)
        else:
            fdk.fdk_backproject(v, proj, mats, vs, org, fetch=fdk.FETCH_LDG, tile=tile)
        out.append(v)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("fetch", [fdk.FETCH_AUTO, fdk.FETCH_LDG])
@pytest.mark.parametrize("tile", [0, 2, 4, 5, 7])
def test_batch_equals_sequential_bitwise(tile, fetch):
    scans = _small_batch()
    plan = fdk.fdk_batch_plan_create(scans, tile=tile, fetch=fetch)
    assert plan.tile == tile
    staged = [plan.scan_fetch(i) == fdk.FETCH_STAGE for i in range(len(scans))]
    if fetch == fdk.FETCH_LDG or tile in (2, 4):
        assert not any(staged)        # LDG requested, or CTAs other than 16 x 16
    else:
        assert any(staged) and not all(staged)
    ref = _sequential(scans, tile, plan=plan)
    plan.execute()
    torch.cuda.synchronize()
    fdk.fdk_device_status()
    for (vol, *_), r in zip(scans, ref):
        assert torch.equal(vol, r)
    plan.close()


def test_batch_with_fine_voxel_scans_staged():
    """Scans at the pitch of the 512^3 workload (0.5 mm voxels on the 1248 x
    960 detector), where the staged path pays, among coarse ones: the staged
    scans equal fdk_backproject's default (staged) path bit for bit and the
    oracle within the accuracy bar."""
    scans = []
    for i, (n, views) in enumerate([(48, 40), (40, 24), (32, 30)]):
        cfg = synth.preset("fdk512", nx=n, ny=n + 8, nz=n - 8, n_views=views, seed=900 + i)
        s = synth.make_scan(cfg, device="cuda")
        scans.append((torch.zeros((cfg.nz, cfg.ny, cfg.nx), device="cuda"), s["proj"], s["mats"],
                      s["voxel_size"], s["origin"]))
    scans += _small_batch(n=3, seed=82)
    plan = fdk.fdk_batch_plan_create(scans)
    assert [plan.scan_fetch(i) for i in range(3)] == [fdk.FETCH_STAGE] * 3
    ref = _sequential(scans, plan.tile, plan=plan)
    plan.execute()
    torch.cuda.synchronize()
    fdk.fdk_device_status()
    for (vol, *_), r in zip(scans, ref):
        assert torch.equal(vol, r)
    vol, proj, mats, vs, org = scans[0]
    nz, ny, nx = vol.shape
    ref = oracle.backproject(proj.cpu().numpy(), mats, (nx, ny, nz), vs, org, threads=os.cpu_count() or 1)
    assert_parity(ref, vol.cpu().numpy(), what="staged scan of a batch vs oracle")
    plan.close()


def test_batch_with_a_scan_that_runs_alone():
    """A scan at the 512^3 workload's pitch with two waves of the staged
    kernel's tiles (192 x 192 x 128 voxels) runs as its own staged launches
    after the persistent kernel: it, and the small scans in the kernel, equal
    fdk_backproject bit for bit, also through CUDA-graph capture and replay;
    the autotuner leaves the volumes alone and its pick matches too."""
    cfg = synth.preset("fdk512", nx=192, ny=192, nz=128, n_views=24, seed=950)
    s = synth.make_scan(cfg, device="cuda")
    scans = [(torch.zeros((cfg.nz, cfg.ny, cfg.nx), device="cuda"), s["proj"], s["mats"],
              s["voxel_size"], s["origin"])]
    scans += _small_batch(n=4, seed=83)
    plan = fdk.fdk_batch_plan_create(scans)
    assert plan.scan_fetch(0) == fdk.FETCH_STAGE
    ref = _sequential(scans, plan.tile, plan=plan)
    plan.execute()
    torch.cuda.synchronize()
    fdk.fdk_device_status()
    for (vol, *_), r in zip(scans, ref):
        assert torch.equal(vol, r)
    # graph capture records the kernel and the scan's own launches
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        plan.execute(stream=st)
    for vol, *_ in scans:
        vol.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    for (vol, *_), r in zip(scans, ref):
        assert torch.equal(vol, r)
    plan.close()
    for vol, *_ in scans:
        vol.fill_(1.5)
    plan = fdk.fdk_batch_plan_create(scans, autotune=True)
    torch.cuda.synchronize()
    for vol, *_ in scans:
        assert torch.all(vol == 1.5)
    ref = _sequential(scans, plan.tile, init=1.5, plan=plan)
    plan.execute()
    torch.cuda.synchronize()
    for (vol, *_), r in zip(scans, ref):
        assert torch.equal(vol, r)
    plan.close()


def test_autotune_leaves_volumes_and_matches_its_tile():
    scans = _small_batch(seed=78)
    for vol, *_ in scans:
        vol.fill_(1.5)
    plan = fdk.fdk_batch_plan_create(scans, autotune=True)
    torch.cuda.synchronize()
    for vol, *_ in scans:
        assert torch.all(vol == 1.5)          # tuning wrote only to its scratch volume
    tile = plan.tile
    assert tile in (0, 2, 3, 4, 5, 7)
    ref = _sequential(scans, tile, init=1.5, plan=plan)
    plan.execute()
    torch.cuda.synchronize()
    for (vol, *_), r in zip(scans, ref):
        assert torch.equal(vol, r)


def test_batch_cuda_graph_replay():
    scans = _small_batch(n=6, seed=79)
    plan = fdk.fdk_batch_plan_create(scans, tile=0)
    assert any(plan.scan_fetch(i) == fdk.FETCH_STAGE for i in range(len(scans)))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.execute(stream=s)
    # capture recorded the work without running it
    for vol, *_ in scans:
        vol.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    ref = _sequential(scans, 0, plan=plan)
    for (vol, *_), r in zip(scans, ref):
        assert torch.equal(vol, r)
    g.replay()                                # replays accumulate like executions
    torch.cuda.synchronize()
    ref2 = [r.clone() for r in ref]
    for i, ((vol, proj, mats, vs, org), r) in enumerate(zip(scans, ref2)):
        if plan.scan_fetch(i) == fdk.FETCH_STAGE:
            fdk.fdk_backproject(r, proj, mats, vs, org, fetch=fdk.FETCH_STAGE)
        else:
            fdk.fdk_backproject(r, proj, mats, vs, org, fetch=fdk.FETCH_LDG, tile=0)
    torch.cuda.synchronize()
    for (vol, *_), r in zip(scans, ref2):
        assert torch.equal(vol, r)


def test_batch_against_oracle_and_one_shot():
    scans = _small_batch(n=4, seed=80)
    fdk.fdk_backproject_batched(scans, tile=0)
    for vol, proj, mats, vs, org in scans:
        nz, ny, nx = vol.shape
        ref = oracle.backproject(proj.cpu().numpy(), mats, (nx, ny, nz), vs, org,
                                 threads=os.cpu_count() or 1)
        if np.abs(ref).max() > 0:
            assert_parity(ref, vol.cpu().numpy(), what="batch vs oracle")


def test_batch_rejects_bad_scans():
    scans = _small_batch(n=2, seed=81)
    bad = list(scans[0])
    bad[2] = np.zeros((3, 12), np.float32)     # wrong matrix count
    with pytest.raises(ValueError):
        fdk.fdk_batch_plan_create([tuple(bad)])
    with pytest.raises(fdk.FdkError):
        fdk.fdk_batch_plan_create(scans, tile=6)
