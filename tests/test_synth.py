"""The synthetic scan generator against the geometry and phantom it states.

The generator stands in for the RabbitCT scan (496 views of 1248x960 pixels
from a C-arm short scan, Sec. IV and Sec. VIII): a circular 200-degree scan
with source-isocentre distance SID, source-detector distance SDD, square
pixels, seeded principal-point jitter and camera tilts, and a phantom of
seeded ellipsoids whose line integrals are computed analytically.  These
tests check those statements from the physical set-up, not from the
generator's own formulas:

* the source is the null space of every matrix and lies on the scan circle;
* a point on the physical detector plane (distance SDD from the source along
  the tilted principal axis, offset by whole pixel pitches) maps to its own
  pixel indices, with w = SDD / SID there and w close to 1 at the isocentre;
* a sphere's line integrals equal the chord length 2 sqrt(r^2 - d^2) times
  its density, d the distance from its centre to the ray;
* a rotated ellipsoid's line integrals equal a dense march along the ray;
* the named workloads and the batch have the sizes the benchmark quotes.
"""
import math

import numpy as np
import pytest
import torch

import synth


def _views(cfg):
    geo = synth.geometry(cfg)
    return geo, geo["mats64"], geo["source"], geo["rcam"]


@pytest.mark.parametrize("name", ["small", "fdk512"])
def test_source_is_null_space_on_the_scan_circle(name):
    cfg = synth.preset(name, n_views=37)
    geo, P, S, _ = _views(cfg)
    # P (S, 1) = 0: every ray of the camera starts at the source
    img = np.einsum("kij,kj->ki", P[:, :, :3], S) + P[:, :, 3]
    assert np.abs(img).max() < 1e-12 * np.abs(P).max() * cfg.sid
    # the source circle: radius SID in the plane z = 0, angles 0..200 degrees
    np.testing.assert_allclose(np.linalg.norm(S[:, :2], axis=1), cfg.sid, rtol=1e-12)
    np.testing.assert_allclose(S[:, 2], 0.0, atol=1e-9)
    ang = np.unwrap(np.arctan2(S[:, 1], S[:, 0]))
    np.testing.assert_allclose(np.rad2deg(ang), np.linspace(0.0, cfg.arc_deg, cfg.n_views), atol=1e-9)
    # the FP32 matrices handed to the library are the FP64 ones rounded
    np.testing.assert_array_equal(geo["mats"], P.astype(np.float32))


@pytest.mark.parametrize("name", ["small", "fdk512"])
def test_detector_plane_pixels_map_to_their_indices(name):
    """Pixel (m, n) sits SDD from the source along the camera's principal
    axis, (m - u0) and (n - v0) pixel pitches along the detector axes; the
    matrix must send that point to (u, v) = (m, n) with w = SDD / SID."""
    cfg = synth.preset(name, n_views=23)
    geo, P, S, R = _views(cfg)
    # the camera axes are orthonormal and within the stated tilts of the
    # ideal C-arm axes (three rotations of at most tilt_deg each)
    np.testing.assert_allclose(np.einsum("kij,klj->kil", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-12)
    lim = math.cos(math.radians(3 * cfg.tilt_deg))
    assert (np.einsum("kj,kj->k", R[:, 2], -S / cfg.sid) >= lim).all()        # principal axis to isocentre
    assert (R[:, 1, 2] >= lim).all()                                          # v along the rotation axis
    # the principal point is the detector centre within the stated jitter
    assert (np.abs(geo["u0"] - (cfg.det_w - 1) / 2) <= cfg.jitter_px).all()
    assert (np.abs(geo["v0"] - (cfg.det_h - 1) / 2) <= cfg.jitter_px).all()
    rng = np.random.default_rng(3)
    m = np.concatenate([[0, cfg.det_w - 1], rng.integers(0, cfg.det_w, 30)]).astype(np.float64)
    n = np.concatenate([[0, cfg.det_h - 1], rng.integers(0, cfg.det_h, 30)]).astype(np.float64)
    for k in range(cfg.n_views):
        D = (S[k] + cfg.sdd * R[k, 2] + np.outer(m - geo["u0"][k], cfg.pixel * R[k, 0])
             + np.outer(n - geo["v0"][k], cfg.pixel * R[k, 1]))
        uvw = D @ P[k, :, :3].T + P[k, :, 3]
        np.testing.assert_allclose(uvw[:, 2], cfg.sdd / cfg.sid, rtol=1e-12)
        np.testing.assert_allclose(uvw[:, 0] / uvw[:, 2], m, atol=1e-9)
        np.testing.assert_allclose(uvw[:, 1] / uvw[:, 2], n, atol=1e-9)
        # w at the isocentre is its depth over SID: 1 up to the tilt
        assert abs(P[k, 2, 3] - 1.0) <= 1.0 - lim


def _one_sphere(centre, r, density):
    return {"centres": np.array([centre], np.float64), "axes": np.full((1, 3), float(r)),
            "rots": np.eye(3)[None], "density": np.array([float(density)])}


def _pixel_rays(cfg, geo, k):
    """Unit ray directions from the source through every pixel centre of
    view k, from the physical detector plane, (H, W, 3)."""
    R, S = geo["rcam"][k], geo["source"][k]
    m = np.arange(cfg.det_w, dtype=np.float64)
    n = np.arange(cfg.det_h, dtype=np.float64)
    D = (S + cfg.sdd * R[2] + (m[None, :, None] - geo["u0"][k]) * cfg.pixel * R[0]
         + (n[:, None, None] - geo["v0"][k]) * cfg.pixel * R[1])
    d = D - S
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def test_sphere_line_integrals_are_chord_lengths():
    cfg = synth.preset("small", n_views=5)
    geo = synth.geometry(cfg)
    for centre, r, rho in (((0.0, 0.0, 0.0), 40.0, 0.7), ((25.0, -30.0, 15.0), 22.0, 0.3)):
        ph = _one_sphere(centre, r, rho)
        raw = synth.projections(cfg, geo, ph, filtered=False, dtype=torch.float64).numpy()
        assert (raw > 0).sum() > 50                     # the sphere covers many pixels
        for k in range(cfg.n_views):
            u = _pixel_rays(cfg, geo, k)
            cs = np.asarray(centre) - geo["source"][k]
            d2 = np.sum(np.cross(cs, u) ** 2, axis=-1)   # squared distance centre-ray
            half2 = np.maximum(r * r - d2, 0.0)           # (chord / 2)^2
            # compared as squares: at the rim the chord is the root of a
            # difference of two numbers near SID^2, so its rounding is large
            # in the chord and tiny in its square
            np.testing.assert_allclose((raw[k] / (2 * rho)) ** 2, half2, rtol=0, atol=1e-9 * r * r)
            deep = half2 > 0.01 * r * r
            np.testing.assert_allclose(raw[k][deep], rho * 2 * np.sqrt(half2[deep]), rtol=1e-9)


def test_rotated_ellipsoid_line_integrals_match_a_dense_march():
    """Brute force: step along each ray at 1e-3 mm and count the samples
    inside the ellipsoid (axes 35, 18, 9 mm, seeded rotation)."""
    cfg = synth.preset("small", n_views=3)
    geo = synth.geometry(cfg)
    q, rr = np.linalg.qr(np.random.default_rng(9).normal(size=(3, 3)))
    Q = q * np.sign(np.diag(rr))
    c = np.array([12.0, -7.0, 5.0])
    axes = np.array([35.0, 18.0, 9.0])
    ph = {"centres": c[None], "axes": axes[None], "rots": Q[None], "density": np.array([0.9])}
    raw = synth.projections(cfg, geo, ph, filtered=False, dtype=torch.float64).numpy()
    rng = np.random.default_rng(10)
    dt = 1e-3
    t_rel = np.arange(-axes.max(), axes.max(), dt) + dt / 2
    checked = 0
    for k in range(cfg.n_views):
        u = _pixel_rays(cfg, geo, k)
        hit = np.argwhere(raw[k] > 0)
        miss = np.argwhere(raw[k] == 0)
        picks = np.concatenate([hit[rng.choice(len(hit), 8, replace=False)],
                                miss[rng.choice(len(miss), 2, replace=False)]])
        S = geo["source"][k]
        for n, m in picks:
            d = u[n, m]
            tc = float(np.dot(c - S, d))                 # closest approach to the centre
            X = S + (tc + t_rel)[:, None] * d
            y = (X - c) @ Q / axes                       # ellipsoid frame, unit sphere
            inside = np.count_nonzero(np.sum(y * y, axis=1) <= 1.0)
            np.testing.assert_allclose(raw[k, n, m], 0.9 * inside * dt, rtol=0, atol=0.9 * 2 * dt)
            checked += 1
    assert checked == 30


def test_phantom_inside_the_field_of_view():
    for name in ("fdk128", "fdk512", "fdk1024", "fdk256", "small"):
        cfg = synth.PRESETS[name]
        ph = synth.phantom(cfg)
        assert ph["centres"].shape == (cfg.n_ellipsoids, 3)
        assert ((ph["density"] >= 0.1) & (ph["density"] <= 1.0)).all()
        reach = ph["axes"].max(axis=1)                 # bounding sphere of each ellipsoid
        assert (np.hypot(ph["centres"][:, 0], ph["centres"][:, 1]) + reach <= 90.0 + 1e-9).all()
        assert (np.abs(ph["centres"][:, 2]) + reach <= 70.0 + 1e-9).all()
        Q = ph["rots"]
        np.testing.assert_allclose(np.einsum("kji,kjl->kil", Q, Q),
                                   np.broadcast_to(np.eye(3), Q.shape), atol=1e-12)


def test_named_workloads_and_batch_sizes():
    expect = {"fdk128": (128, 2.0, 496, 1.04e9), "fdk512": (512, 0.5, 496, 6.66e10),
              "fdk1024": (1024, 0.25, 496, 5.33e11), "fdk256": (256, 1.0, 248, 4.16e9)}
    for name, (nvox, vox, views, upd) in expect.items():
        cfg = synth.PRESETS[name]
        assert (cfg.nx, cfg.ny, cfg.nz, cfg.voxel, cfg.n_views) == (nvox, nvox, nvox, vox, views)
        assert (cfg.det_w, cfg.det_h, cfg.pixel) == (1248, 960, 0.308)
        assert cfg.nx * cfg.voxel == 256.0                         # a 256 mm cube
        assert abs(cfg.updates / upd - 1) < 5e-3
        dims, vs, org = synth.volume_geometry(cfg)
        # the volume is centred: voxel centres symmetric about the isocentre
        np.testing.assert_allclose(org + (dims - 1) * vs, -org, rtol=1e-6)
    scans = synth.batch_scan_configs(32)
    assert len(scans) == 32
    for c in scans:
        assert all(64 <= d <= 384 for d in (c.nx, c.ny, c.nz))
        assert 120 <= c.n_views <= 496
        assert 640 <= c.det_w <= 1248 and 480 <= c.det_h <= 960
        assert abs(max(c.nx, c.ny, c.nz) * c.voxel - 256.0) < 1e-9
        assert abs(c.det_w * c.pixel - 1248 * 0.308) < 1e-9        # the same detector field
    assert len({(c.nx, c.ny, c.nz) for c in scans}) == 32
    assert any(len({c.nx, c.ny, c.nz}) > 1 for c in scans)          # non-cubic volumes present
    small = synth.small_batch_scan_configs(128)
    assert len(small) == 128
    for c in small:
        assert all(32 <= d <= 96 for d in (c.nx, c.ny, c.nz))
        assert 60 <= c.n_views <= 180
        assert 320 <= c.det_w <= 640 and 240 <= c.det_h <= 480
        assert abs(max(c.nx, c.ny, c.nz) * c.voxel - 256.0) < 1e-9
        assert abs(c.det_w * c.pixel - 1248 * 0.308) < 1e-9
    # each scan alone under-fills the GPU: fewer 16 x 16 x 8 tiles than 152 SMs x 4 CTAs
    assert max((c.nx + 15) // 16 * ((c.ny + 15) // 16) * ((c.nz + 7) // 8) for c in small) < 152 * 4


def test_same_seed_same_scan():
    cfg = synth.preset("tiny")
    a = synth.make_scan(cfg)
    b = synth.make_scan(cfg)
    np.testing.assert_array_equal(a["mats"], b["mats"])
    assert torch.equal(a["proj"], b["proj"])
    c = synth.make_scan(synth.preset("tiny", seed=8))
    assert not np.array_equal(a["mats"], c["mats"])
