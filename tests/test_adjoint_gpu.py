"""GPU parity of the transpose (fdk_forwardproject_adjoint) and of autograd.

The adjoint is checked elementwise against the FP64 oracle's transpose, by
the dot-product identity <B y, x> = <y, B^T x>, by central finite
differences of a loss through the autograd wrapper, and by 20 steps of
least-squares reconstruction whose loss must fall.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import assert_parity
from paper_1401_3615_gb300 import autograd, fdk

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1


def _gpu_adj(scan, vol):
    n = scan["mats"].shape[0]
    cfg = scan["cfg"]
    proj = torch.zeros((n, cfg.det_h, cfg.det_w), device="cuda")
    fdk.fdk_forwardproject_adjoint(proj, vol, scan["mats"], scan["voxel_size"], scan["origin"])
    torch.cuda.synchronize()
    return proj


def _oracle_adj(scan, vol_np, mats=None):
    cfg = scan["cfg"]
    m = scan["mats"] if mats is None else mats
    return oracle.adjoint(vol_np, m, scan["dims"], scan["voxel_size"], scan["origin"],
                          cfg.det_w, cfg.det_h, threads=NCPU)


@pytest.fixture(scope="module")
def ragged():
    return synth.make_scan(synth.preset("small", nx=37, ny=29, nz=21), device="cuda")


def test_adjoint_parity_ragged(ragged):
    x = synth.gaussian_volume(ragged["dims"], seed=31)
    got = _gpu_adj(ragged, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = _oracle_adj(ragged, x)
    assert_parity(ref, got, what="adjoint")


def test_adjoint_anisotropic_voxels_offset_origin():
    """Voxel pitches of 9, 11 and 13 mm along x, y and z and an origin off
    the isocentre."""
    s = synth.make_scan(synth.preset("small", nx=37, ny=29, nz=21), device="cuda")
    vs = np.array([9.0, 11.0, 13.0], np.float32)
    s["voxel_size"] = vs
    s["origin"] = (-(s["dims"].astype(np.float64) - 1) / 2.0 * vs + np.array([6.0, -4.0, 9.0])).astype(np.float32)
    x = synth.gaussian_volume(s["dims"], seed=38)
    assert_parity(_oracle_adj(s, x), _gpu_adj(s, torch.from_numpy(x).cuda()).cpu().numpy(),
                  what="adjoint, anisotropic")


def test_adjoint_accumulates_and_multi_pass():
    s = synth.make_scan(synth.preset("small", n_views=600, det_w=40, det_h=32, nx=20, ny=18, nz=10),
                        device="cuda")
    x = synth.gaussian_volume(s["dims"], seed=32)
    proj = torch.full((600, 32, 40), 0.25, device="cuda")
    fdk.fdk_forwardproject_adjoint(proj, torch.from_numpy(x).cuda(), s["mats"], s["voxel_size"],
                                   s["origin"])
    torch.cuda.synchronize()
    ref = _oracle_adj(s, x) + 0.25
    assert_parity(ref, proj.cpu().numpy())


def test_adjoint_device_matrices_multi_pass():
    """Matrices in device memory, which the host cannot read to group the
    views by ray orientation: one launch per pass in view order, here 600
    views in two passes."""
    s = synth.make_scan(synth.preset("small", n_views=600, det_w=40, det_h=32, nx=20, ny=18, nz=10),
                        device="cuda")
    x = synth.gaussian_volume(s["dims"], seed=39)
    proj = torch.zeros((600, 32, 40), device="cuda")
    fdk.fdk_forwardproject_adjoint(proj, torch.from_numpy(x).cuda(), torch.from_numpy(s["mats"]).cuda(),
                                   s["voxel_size"], s["origin"])
    torch.cuda.synchronize()
    assert_parity(_oracle_adj(s, x), proj.cpu().numpy(), what="adjoint, device matrices")


@pytest.mark.parametrize("lift_mm", [0.0, 75.0])
def test_adjoint_source_inside_volume(lift_mm):
    """The source circle (radius 150 mm) lies within the 400 mm x-y extent
    of the volume, so tiles straddle the source's principal plane and hold
    w <= 0 voxels, which receive nothing.  Unlifted, the volume is centred
    on the plane of the source circle and voxels sit a few mm in front of
    the source; lifted 75 mm, a voxel that projects onto the detector is at
    least 83 mm deep."""
    s = synth.make_scan(synth.preset("small", nx=40, ny=40, nz=8, voxel=10.0, sid=150.0, sdd=300.0),
                        device="cuda")
    s["origin"] = s["origin"] + np.float32([0.0, 0.0, lift_mm])
    x = synth.gaussian_volume(s["dims"], seed=33)
    rel, p = assert_parity(_oracle_adj(s, x), _gpu_adj(s, torch.from_numpy(x).cuda()).cpu().numpy(),
                           what=f"source inside, lifted {lift_mm} mm")
    print(f"adjoint, source inside, lifted {lift_mm} mm: max|diff|/max|f| = {rel:.3e}, PSNR = {p:.1f} dB")


def test_adjoint_large_footprints():
    """Coarse voxels on a fine detector: per-view footprints larger than the
    shared-memory buffer take the direct-atomic path."""
    big = synth.make_scan(synth.preset("small", nx=24, ny=24, nz=8, voxel=8.0, n_views=6,
                                       det_w=400, det_h=300, pixel=0.308), device="cuda")
    xb = synth.gaussian_volume(big["dims"], seed=34)
    assert_parity(_oracle_adj(big, xb), _gpu_adj(big, torch.from_numpy(xb).cuda()).cpu().numpy(),
                  what="large footprints")


def test_adjoint_full_detector_sampled_views():
    """256^3 volume, 1248 x 960 detector: 8 of the 248 views of the
    differentiation workload, whole images, against the oracle."""
    cfg = synth.PRESETS["fdk256"]
    geo = synth.geometry(cfg)
    pick = np.linspace(0, cfg.n_views - 1, 8).astype(int)
    mats = geo["mats"][pick]
    dims, vs, org = synth.volume_geometry(cfg)
    s = {"cfg": cfg, "mats": mats, "dims": dims, "voxel_size": vs, "origin": org}
    x = synth.gaussian_volume(dims, seed=35)
    got = _gpu_adj(s, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = _oracle_adj(s, x)
    assert_parity(ref, got, what="adjoint 256^3")


def test_adjoint_512_cube_sampled_views():
    """The transpose on the 512^3 workload in the launch configuration the
    benchmark times (host matrices, one launch per ray orientation, the
    16-voxel z-run this geometry takes): a seeded Gaussian 512^3 volume onto
    4 of the 496 views, whole 1248 x 960 images, against the oracle."""
    cfg = synth.PRESETS["fdk512"]
    geo = synth.geometry(cfg)
    pick = np.linspace(0, cfg.n_views - 1, 4).astype(int)
    dims, vs, org = synth.volume_geometry(cfg)
    s = {"cfg": cfg, "mats": geo["mats"][pick], "dims": dims, "voxel_size": vs, "origin": org}
    x = synth.gaussian_volume(dims, seed=37)
    got = _gpu_adj(s, torch.from_numpy(x).cuda()).cpu().numpy()
    assert_parity(_oracle_adj(s, x), got, what="adjoint 512^3")


def test_adjoint_fine_voxels_16_voxel_run():
    """0.5 mm voxels on the 1248 x 960 detector (the 512^3 workload's pitch),
    a 96 x 96 x 40 centre block, 32 views spread over the scan: the volume
    stays far from the source and the footprints fit half the shared buffer,
    so the adjoint takes its 16-voxel z-run; 40 slices leave a ragged last
    run of 8."""
    cfg = synth.preset("fdk512", nx=96, ny=96, nz=40)
    geo = synth.geometry(cfg)
    pick = np.linspace(0, cfg.n_views - 1, 32).astype(int)
    dims, vs, org = synth.volume_geometry(cfg)
    s = {"cfg": cfg, "mats": geo["mats"][pick], "dims": dims, "voxel_size": vs, "origin": org}
    x = synth.gaussian_volume(dims, seed=36)
    got = _gpu_adj(s, torch.from_numpy(x).cuda()).cpu().numpy()
    assert_parity(_oracle_adj(s, x), got, what="adjoint 0.5 mm, 16-voxel run")


def test_dot_product_identity(ragged):
    n, H, W = ragged["proj"].shape
    y = torch.from_numpy(synth.gaussian_projections(n, H, W, seed=41)).cuda()
    x = torch.from_numpy(synth.gaussian_volume(ragged["dims"], seed=42)).cuda()
    by = torch.zeros_like(x)
    fdk.fdk_backproject(by, y, ragged["mats"], ragged["voxel_size"], ragged["origin"])
    btx = _gpu_adj(ragged, x)
    lhs = float((by.double() * x.double()).sum())
    rhs = float((y.double() * btx.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_autograd_gradients_finite_differences(ragged):
    """d/dy <c, B y> = B^T c checked by central differences (eps = 1e-3) on
    32 seeded projection pixels; the operator is linear, so the differences
    are exact up to rounding."""
    n, H, W = ragged["proj"].shape
    vol_shape = (int(ragged["dims"][2]), int(ragged["dims"][1]), int(ragged["dims"][0]))
    c = torch.from_numpy(synth.gaussian_volume(ragged["dims"], seed=43)).cuda().double()
    y = ragged["proj"].clone().requires_grad_(True)
    vol = autograd.backproject(y, ragged["mats"], ragged["voxel_size"], ragged["origin"], vol_shape)
    loss = (vol.double() * c).sum()
    loss.backward()
    grad = y.grad.detach().cpu().numpy()
    rng = np.random.default_rng(44)
    eps = 1e-3
    for _ in range(32):
        k, j, i = rng.integers(0, n), rng.integers(0, H), rng.integers(0, W)
        vals = []
        for sgn in (1.0, -1.0):
            yp = ragged["proj"].clone()
            yp[k, j, i] += sgn * eps
            vp = autograd.backproject(yp, ragged["mats"], ragged["voxel_size"], ragged["origin"], vol_shape)
            vals.append(float((vp.double() * c).sum()))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - grad[k, j, i]) <= 2e-3 * max(1.0, abs(grad[k, j, i])), (fd, grad[k, j, i])


def test_autograd_forwardproject_backward_is_backprojection(ragged):
    n, H, W = ragged["proj"].shape
    x = torch.from_numpy(synth.gaussian_volume(ragged["dims"], seed=45)).cuda().requires_grad_(True)
    q = autograd.forwardproject(x, ragged["mats"], ragged["voxel_size"], ragged["origin"], (n, H, W))
    g = torch.from_numpy(synth.gaussian_projections(n, H, W, seed=46)).cuda()
    (q * g).sum().backward()
    expect = torch.zeros_like(x)
    fdk.fdk_backproject(expect, g, ragged["mats"], ragged["voxel_size"], ragged["origin"])
    torch.cuda.synchronize()
    assert_parity(expect.detach().cpu().numpy(), x.grad.cpu().numpy())


def test_least_squares_reconstruction_20_steps():
    """min_x ||B^T x - y||^2 over x by gradient descent with the exact
    Lipschitz step; the loss falls monotonically over 20 steps."""
    cfg = synth.preset("small", nx=32, ny=32, nz=16, voxel=6.0, n_views=60, det_w=96, det_h=64,
                       pixel=0.308 * 13)
    s = synth.make_scan(cfg, device="cuda", filtered=False)
    shape = (cfg.nz, cfg.ny, cfg.nx)
    det = (cfg.n_views, cfg.det_h, cfg.det_w)
    A = lambda v: autograd.forwardproject(v, s["mats"], s["voxel_size"], s["origin"], det)
    # Lipschitz constant of the gradient: 2 * largest eigenvalue of B B^T (power iteration)
    v = torch.randn(shape, device="cuda")
    for _ in range(30):
        v = autograd.backproject(A(v), s["mats"], s["voxel_size"], s["origin"], shape)
        v = v / v.norm()
    lam = float((A(v) ** 2).sum())
    y = s["proj"]
    x = torch.zeros(shape, device="cuda", requires_grad=True)
    losses = []
    for _ in range(20):
        loss = ((A(x) - y) ** 2).sum()
        losses.append(float(loss.detach()))
        g, = torch.autograd.grad(loss, x)
        with torch.no_grad():
            x -= g / (2.0 * lam)
    assert all(b <= a * (1 + 1e-6) for a, b in zip(losses, losses[1:])), losses
    assert losses[-1] < 0.5 * losses[0], losses


# The differentiation workload: 256^3 volume (1 mm voxels), 248 views of
# 1248 x 960, the ellipsoid phantom's projections.

@pytest.fixture(scope="module")
def fdk256():
    return synth.make_scan(synth.PRESETS["fdk256"], device="cuda")


def _vol_shape(scan):
    return (int(scan["dims"][2]), int(scan["dims"][1]), int(scan["dims"][0]))


def test_dot_product_identity_256_cube_248_views(fdk256):
    """<B y, x> = <y, B^T x> for seeded Gaussian y (248 x 960 x 1248) and x
    (256^3), both inner products reduced in FP64."""
    n, H, W = fdk256["proj"].shape
    y = torch.from_numpy(synth.gaussian_projections(n, H, W, seed=401)).cuda()
    x = torch.from_numpy(synth.gaussian_volume(fdk256["dims"], seed=402)).cuda()
    by = torch.zeros_like(x)
    fdk.fdk_backproject(by, y, fdk256["mats"], fdk256["voxel_size"], fdk256["origin"])
    lhs = float((by.double() * x.double()).sum())
    del by
    btx = torch.zeros_like(y)
    fdk.fdk_forwardproject_adjoint(btx, x, fdk256["mats"], fdk256["voxel_size"], fdk256["origin"])
    rhs = float((y.double() * btx.double()).sum())
    rel = abs(lhs - rhs) / max(abs(lhs), abs(rhs))
    print(f"fdk256 dot product: <By,x> = {lhs:.9e}, <y,B^T x> = {rhs:.9e}, relative difference {rel:.2e}")
    assert rel <= 1e-5, (lhs, rhs)


def test_finite_differences_256_cube_248_views(fdk256):
    """The gradient of L(p) = <c, B p> with respect to the projections, from
    the autograd backward (the transpose kernel), against central
    differences with eps = 1e-3 on 32 seeded projection pixels, at the
    phantom's filtered projections.  B is linear, so the differences are
    exact up to the FP32 rounding of the perturbed voxel sums (about 1e-4 of
    the gradient here); the losses are reduced in FP64."""
    proj = fdk256["proj"]
    n, H, W = proj.shape
    shape = _vol_shape(fdk256)
    geo = (fdk256["mats"], fdk256["voxel_size"], fdk256["origin"], shape)
    c = torch.from_numpy(synth.gaussian_volume(fdk256["dims"], seed=403)).cuda().double()
    y = proj.clone().requires_grad_(True)
    loss = (autograd.backproject(y, *geo).double() * c).sum()
    loss.backward()
    grad = y.grad.detach()
    del y
    rng = np.random.default_rng(404)
    pix = np.stack([rng.integers(0, n, 32), rng.integers(0, H, 32), rng.integers(0, W, 32)], 1)
    g = np.array([float(grad[k, j, i]) for k, j, i in pix])
    scale = float(np.sqrt(np.mean(g ** 2)))
    assert scale > 0
    eps = 1e-3
    worst = 0.0
    for (k, j, i), gk in zip(pix, g):
        vals = []
        for sgn in (1.0, -1.0):
            old = float(proj[k, j, i])
            proj[k, j, i] = old + sgn * eps
            vals.append(float((autograd.backproject(proj, *geo).double() * c).sum()))
            proj[k, j, i] = old
        fd = (vals[0] - vals[1]) / (2 * eps)
        err = abs(fd - gk) / max(abs(gk), scale)
        worst = max(worst, err)
        assert err <= 2e-3, (k, j, i, fd, gk)
    print(f"fdk256 finite differences, 32 pixels: worst |fd - grad| / max(|grad|, rms grad) = {worst:.2e}")


def test_least_squares_256_cube_248_views_20_steps():
    """20 steps of gradient descent on min_x ||B^T x - y||^2 at the
    differentiation workload's size, y the phantom's line integrals (248 x
    960 x 1248), x a 256^3 volume, with the Lipschitz step 1 / (2 lambda_max
    (B B^T)) from a power iteration: the loss falls at every step."""
    cfg = synth.PRESETS["fdk256"]
    s = synth.make_scan(cfg, device="cuda", filtered=False)
    shape = (cfg.nz, cfg.ny, cfg.nx)
    det = (cfg.n_views, cfg.det_h, cfg.det_w)
    A = lambda v: autograd.forwardproject(v, s["mats"], s["voxel_size"], s["origin"], det)
    torch.manual_seed(405)
    v = torch.randn(shape, device="cuda")
    for _ in range(20):
        v = autograd.backproject(A(v), s["mats"], s["voxel_size"], s["origin"], shape)
        v = v / v.norm()
    lam = float((A(v).double() ** 2).sum())
    y = s["proj"]
    x = torch.zeros(shape, device="cuda", requires_grad=True)
    losses = []
    for _ in range(20):
        loss = ((A(x) - y).double() ** 2).sum()
        losses.append(float(loss.detach()))
        g, = torch.autograd.grad(loss, x)
        with torch.no_grad():
            x -= g.float() / (2.0 * lam)
    print("fdk256 least squares, loss / initial:", [round(l / losses[0], 4) for l in losses])
    assert all(b <= a * (1 + 1e-6) for a, b in zip(losses, losses[1:])), losses
    assert losses[-1] < 0.9 * losses[0], losses
