"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a value
derived by hand from Listing 1 (Sec. IV), a closed form, an exact special
case, a brute-force evaluation along a different route, or an invariant of
the operator.  Together they catch the plausible slips: a dropped or squared
weight, a swapped axis or tap, a transposed matrix, an off-by-one cell, a
wrong sign in the fraction, a bounds mistake.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scan(name="small", **kw):
    return synth.make_scan(synth.preset(name, **kw))


def _bp(s, proj=None, mats=None, **kw):
    p = s["proj"].numpy() if proj is None else proj
    m = s["mats"] if mats is None else mats
    return oracle.backproject(p, m, s["dims"], s["voxel_size"], s["origin"], **kw)


def test_golden_hand_example():
    """Two views into a 3x2x1 volume, computed by hand (tests/golden)."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "listing1_hand.txt"))
            if ln.strip() and not ln.startswith("#")]
    expect = np.array(rows, dtype=np.float64)
    img = np.array([[1, 2, 4], [8, 16, 32]], dtype=np.float32)
    proj = np.stack([img, img])
    mats = np.array([[[2, 0, 0, 1], [0, 2, 0, 0], [0, 0, 0, 2]],
                     [[2, 0, 0, -2], [0, 2, 0, -1], [0, 0, 0, 2]]], dtype=np.float32)
    f = oracle.backproject(proj, mats, (3, 2, 1), (1, 1, 1), (0.25, 0.5, 0.0))
    assert f.shape == (1, 2, 3)
    np.testing.assert_array_equal(f[0], expect)


def test_closed_form_constant_projections():
    """Constant projections c: the bilinear weights sum to one, so wherever
    every view covers the voxel f = c * sum_k 1/w_k^2, with w_k the depth of
    the voxel along view k's principal axis over SID (computed here from the
    source position and camera axes, not from the matrix)."""
    cfg = synth.preset("small")
    s = _scan("small")
    c = 0.75
    proj = np.full(s["proj"].shape, c, dtype=np.float32)
    f = _bp(s, proj=proj)
    geo = s["geo"]
    dims, vs, org = s["dims"], s["voxel_size"].astype(np.float64), s["origin"].astype(np.float64)
    z, y, x = np.meshgrid(*(org[a] + np.arange(dims[a]) * vs[a] for a in (2, 1, 0)), indexing="ij")
    X = np.stack([x, y, z], -1)
    inv_w2 = np.zeros(x.shape)
    covered = np.ones(x.shape, dtype=bool)
    for k in range(cfg.n_views):
        d = X - geo["source"][k]
        R = geo["rcam"][k]
        depth = d @ R[2]
        u = geo["focal_px"] * (d @ R[0]) / depth + geo["u0"][k]
        v = geo["focal_px"] * (d @ R[1]) / depth + geo["v0"][k]
        covered &= (u >= 0) & (u <= cfg.det_w - 1) & (v >= 0) & (v <= cfg.det_h - 1)
        inv_w2 += (cfg.sid / depth) ** 2
    assert covered.sum() > 100
    # the FP32 matrices differ from the FP64 camera by rounding only
    np.testing.assert_allclose(f[covered], c * inv_w2[covered], rtol=2e-6)
    # outside the covered set the value must not exceed the closed form
    assert np.all(f[~covered] <= c * inv_w2[~covered] * (1 + 2e-6))


def _ortho(s_mm, zaxis=False):
    """u = x/s, v = y/s (or z/s), w = 1."""
    P = np.zeros((3, 4), dtype=np.float32)
    P[0, 0] = 1.0 / s_mm
    if zaxis:
        P[1, 2] = 1.0 / s_mm
    else:
        P[1, 1] = 1.0 / s_mm
    P[2, 3] = 1.0
    return P[None]


def test_orthographic_identity_copies_image():
    """w = 1, u = x, v = y: one view copies the image into every z slice,
    with zeros where the voxel grid runs past the detector (Listing 1's
    zero-outside rule).  x indexes columns (u), y indexes rows (v)."""
    rng = np.random.default_rng(3)
    W, H = 7, 5
    img = rng.standard_normal((1, H, W)).astype(np.float32)
    f = oracle.backproject(img, _ortho(1.0), (9, 6, 3), (1, 1, 1), (0, 0, 0))
    for z in range(3):
        np.testing.assert_array_equal(f[z, :H, :W], img[0].astype(np.float64))
        assert np.all(f[z, H:, :] == 0) and np.all(f[z, :, W:] == 0)
    # z -> v instead: slice y is constant, f[z][y][x] = I[z][x]
    img2 = rng.standard_normal((1, 3, W)).astype(np.float32)
    g = oracle.backproject(img2, _ortho(2.0, zaxis=True), (W, 4, 3), (2, 2, 2), (0, 0, 0))
    for y in range(4):
        np.testing.assert_array_equal(g[:, y, :], img2[0].astype(np.float64))


def test_orthographic_half_offsets_average_taps():
    """Half-voxel offsets land halfway between pixel centres: exact two-tap
    and four-tap averages, and a zero tap past the last column/row."""
    img = np.array([[[1, 2, 4, 8], [16, 32, 64, 128], [256, 512, 1024, 2048]]], dtype=np.float32)
    # origin x = 0.5: u = x + 0.5 -> average of columns x, x+1 (zero past the end)
    f = oracle.backproject(img, _ortho(1.0), (4, 3, 1), (1, 1, 1), (0.5, 0.0, 0.0))
    I = img[0].astype(np.float64)
    Ipad = np.pad(I, ((0, 1), (0, 1)))
    np.testing.assert_array_equal(f[0], 0.5 * (Ipad[:3, :4] + Ipad[:3, 1:5]))
    # both offsets: four-tap average
    g = oracle.backproject(img, _ortho(1.0), (4, 3, 1), (1, 1, 1), (0.5, 0.5, 0.0))
    np.testing.assert_array_equal(
        g[0], 0.25 * (Ipad[:3, :4] + Ipad[:3, 1:5] + Ipad[1:4, :4] + Ipad[1:4, 1:5]))
    # negative offset -0.25: u = x - 0.25, cell floor(u) = x - 1, a = 0.75;
    # voxel 0 sits in (-1, 0) and still sees 0.75 * column 0 (floor reading)
    h = oracle.backproject(img, _ortho(1.0), (4, 3, 1), (1, 1, 1), (-0.25, 0.0, 0.0))
    Il = np.pad(I, ((0, 0), (1, 0)))
    np.testing.assert_array_equal(h[0], 0.25 * Il[:, :4] + 0.75 * Il[:, 1:5])


def test_bruteforce_tent_sum_tiny():
    """8^3 volume, 4 views, 24x16 detector: the floor/cell/bounds route and the
    tent sum over every pixel agree to rounding."""
    s = _scan("tiny")
    f = _bp(s)
    bf = oracle.bruteforce(s["proj"].numpy(), s["mats"], s["dims"], s["voxel_size"], s["origin"])
    assert np.abs(f).max() > 0
    np.testing.assert_allclose(f, bf, rtol=0, atol=1e-12 * np.abs(bf).max())
    # also with Gaussian data covering the whole detector
    g = synth.gaussian_projections(4, 16, 24, seed=5)
    f2 = _bp(s, proj=g)
    bf2 = oracle.bruteforce(g, s["mats"], s["dims"], s["voxel_size"], s["origin"])
    np.testing.assert_allclose(f2, bf2, rtol=0, atol=1e-12 * np.abs(bf2).max())


def test_bruteforce_anisotropic_voxels_offset_origin():
    """Voxel pitches of 24, 32 and 40 mm along x, y and z and an origin off
    the isocentre: the oracle's per-axis world positions agree with the tent
    sum, which computes them on its own."""
    s = _scan("tiny")
    vs = np.array([24.0, 32.0, 40.0], np.float32)
    org = (-(s["dims"].astype(np.float64) - 1) / 2.0 * vs + np.array([5.0, -3.0, 7.0])).astype(np.float32)
    g = synth.gaussian_projections(4, 16, 24, seed=6)
    f = oracle.backproject(g, s["mats"], s["dims"], vs, org)
    bf = oracle.bruteforce(g, s["mats"], s["dims"], vs, org)
    assert np.abs(f).max() > 0
    np.testing.assert_allclose(f, bf, rtol=0, atol=1e-12 * np.abs(bf).max())


def test_linearity():
    s = _scan("small")
    n, H, W = s["proj"].shape
    # dyadic data with few significant bits, so alpha*p + beta*q is exact in FP32
    p = np.round(synth.gaussian_projections(n, H, W, seed=1) * 64) / 64
    q = np.round(synth.gaussian_projections(n, H, W, seed=2) * 64) / 64
    p, q = p.astype(np.float32), q.astype(np.float32)
    alpha, beta = 0.5, -2.0
    lhs = _bp(s, proj=(alpha * p + beta * q).astype(np.float32))
    rhs = alpha * _bp(s, proj=p) + beta * _bp(s, proj=q)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12 * np.abs(rhs).max())


def test_matrix_scale_invariance():
    """u and v are unchanged by P -> sP; the weight 1/w^2 scales by 1/s^2.
    s = 2 is exact in binary, so the result is exactly f/4."""
    s = _scan("small")
    f = _bp(s)
    f2 = _bp(s, mats=(2.0 * s["mats"]).astype(np.float32))
    np.testing.assert_array_equal(f2, f / 4.0)
    f3 = _bp(s, mats=(3.0 * s["mats"].astype(np.float64)).astype(np.float32))
    np.testing.assert_allclose(f3, f / 9.0, rtol=0, atol=1e-5 * np.abs(f).max())


def test_view_chunking_and_accumulate():
    """Back-projection accumulates (VOL +=, called once per projection):
    views [0,a) then [a,N) into the same volume equals one call over [0,N)."""
    s = _scan("small")
    P = s["proj"].numpy()
    M = s["mats"]
    full = _bp(s)
    v = np.zeros_like(full)
    _bp(s, proj=P[:5], mats=M[:5], vol=v)
    _bp(s, proj=P[5:], mats=M[5:], vol=v)
    np.testing.assert_array_equal(v, full)


def test_view_permutation():
    s = _scan("small")
    perm = np.random.default_rng(9).permutation(s["proj"].shape[0])
    f = _bp(s)
    g = _bp(s, proj=s["proj"].numpy()[perm], mats=s["mats"][perm])
    np.testing.assert_allclose(g, f, rtol=0, atol=1e-13 * np.abs(f).max())


def test_thread_split_bitwise():
    s = _scan("small")
    f1 = _bp(s, threads=1)
    for t in (2, 3, 7, 64):
        np.testing.assert_array_equal(_bp(s, threads=t), f1)


def test_voxel_list_matches_volume():
    s = _scan("small")
    f = _bp(s)
    rng = np.random.default_rng(4)
    xyz = np.stack([rng.integers(0, d, 50) for d in s["dims"]], axis=1)
    got = oracle.backproject_voxels(s["proj"].numpy(), s["mats"], s["voxel_size"], s["origin"], xyz)
    np.testing.assert_array_equal(got, f[xyz[:, 2], xyz[:, 1], xyz[:, 0]])


def test_origin_shift_is_index_shift():
    """Moving the origin by one voxel along x shifts the volume by one index."""
    s = _scan("small")
    f = _bp(s)
    org2 = s["origin"].copy()
    org2[0] += s["voxel_size"][0]
    g = oracle.backproject(s["proj"].numpy(), s["mats"], s["dims"], s["voxel_size"], org2)
    np.testing.assert_allclose(g[:, :, :-1], f[:, :, 1:], rtol=0, atol=1e-12 * np.abs(f).max())


def test_column_major_helper():
    """The paper's listing stores A column-major (A[0], A[3], A[6], A[9] is the
    u row); converting that layout gives the identical result."""
    s = _scan("small")
    colmaj = np.ascontiguousarray(s["mats"].transpose(0, 2, 1)).reshape(-1, 12)
    np.testing.assert_array_equal(synth.from_column_major(colmaj), s["mats"])
    np.testing.assert_array_equal(_bp(s, mats=synth.from_column_major(colmaj)), _bp(s))


def test_adjoint_dot_product():
    """<BP(y), x> = <y, BP^T(x)> for seeded Gaussian x, y (FP64)."""
    s = _scan("small")
    n, H, W = s["proj"].shape
    y = synth.gaussian_projections(n, H, W, seed=21)
    x = synth.gaussian_volume(s["dims"], seed=22)
    bp = _bp(s, proj=y)
    at = oracle.adjoint(x, s["mats"], s["dims"], s["voxel_size"], s["origin"], W, H, threads=3)
    lhs = float(np.dot(bp.ravel(), x.astype(np.float64).ravel()))
    rhs = float(np.dot(y.astype(np.float64).ravel(), at.ravel()))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 100
    at1 = oracle.adjoint(x, s["mats"], s["dims"], s["voxel_size"], s["origin"], W, H, threads=1)
    np.testing.assert_array_equal(at, at1)


def test_adjoint_single_voxel_is_tap_weights():
    """The transpose of one voxel under the orthographic matrix puts the
    bilinear weights on the four pixels around (u, v)."""
    vol = np.zeros((1, 1, 1), dtype=np.float32)
    vol[0, 0, 0] = 8.0
    P = _ortho(1.0)
    q = oracle.adjoint(vol, P, (1, 1, 1), (1, 1, 1), (1.25, 2.5, 0.0), 4, 5)
    expect = np.zeros((1, 5, 4))
    expect[0, 2, 1] = 8 * 0.75 * 0.5
    expect[0, 2, 2] = 8 * 0.25 * 0.5
    expect[0, 3, 1] = 8 * 0.75 * 0.5
    expect[0, 3, 2] = 8 * 0.25 * 0.5
    np.testing.assert_array_equal(q, expect)


def test_behind_source_contributes_nothing():
    """w <= 0 (voxel behind the source plane) adds zero."""
    img = np.ones((1, 4, 4), dtype=np.float32)
    P = np.array([[[0, 0, 0, 1], [0, 0, 0, 1], [1, 0, 0, 0]]], dtype=np.float32)  # w = X
    f = oracle.backproject(img, P, (4, 1, 1), (1, 1, 1), (-1.5, 0, 0))
    # X = -1.5, -0.5 (w < 0: zero), 0.5, 1.5 (w > 0: u = v = 1/X inside)
    assert f[0, 0, 0] == 0 and f[0, 0, 1] == 0
    np.testing.assert_allclose(f[0, 0, 2:], [1 / 0.25, 1 / 2.25])


def test_literal_truncation_differs_only_in_first_band():
    """The listing's (int) cast differs from floor only where u or v lies in
    (-1, 0); elsewhere both readings give identical bits."""
    img = np.arange(1, 13, dtype=np.float32).reshape(1, 3, 4)
    P = _ortho(1.0)
    # voxel x sits at u = x - 0.75: voxel 0 in (-1, 0), others >= 0.25
    a = oracle.backproject(img, P, (4, 3, 1), (1, 1, 1), (-0.75, 0, 0))
    b = oracle.backproject(img, P, (4, 3, 1), (1, 1, 1), (-0.75, 0, 0), literal_trunc=True)
    np.testing.assert_array_equal(a[:, :, 1:], b[:, :, 1:])
    assert not np.array_equal(a[:, :, 0], b[:, :, 0])
    # floor: 0.25 * column 0; truncation extrapolates 1.75*c0 - 0.75*c1
    np.testing.assert_array_equal(a[0, :, 0], 0.25 * img[0, :, 0])
    np.testing.assert_array_equal(b[0, :, 0], 1.75 * img[0, :, 0] - 0.75 * img[0, :, 1])


def test_empty_and_degenerate():
    img = np.ones((0, 4, 4), dtype=np.float32)
    f = oracle.backproject(img, np.zeros((0, 3, 4), np.float32), (3, 2, 1), (1, 1, 1), (0, 0, 0))
    assert f.shape == (1, 2, 3) and not f.any()
    g = oracle.backproject(np.ones((1, 4, 4), np.float32), _ortho(1.0), (0, 2, 1), (1, 1, 1), (0, 0, 0))
    assert g.shape == (1, 2, 0)


# --- FDK pre-processing (cosine weight and Ram-Lak row filter) -------------

def test_camera_from_matrix_matches_geometry():
    """(f, u0, v0) read off the matrix equal the generator's camera."""
    cfg = synth.preset("small")
    geo = synth.geometry(cfg)
    cam = oracle.camera(geo["mats"])
    np.testing.assert_allclose(cam[:, 0], geo["focal_px"], rtol=1e-5)
    np.testing.assert_allclose(cam[:, 1], geo["u0"], atol=1e-3)
    np.testing.assert_allclose(cam[:, 2], geo["v0"], atol=1e-3)


def test_filter_of_a_delta_is_the_kernel():
    """An orthographic camera at infinite focal length has cosine weight 1;
    filtering a unit impulse gives the Ram-Lak taps h(0)=1/4,
    h(odd d)=-1/(pi^2 d^2), h(even d)=0, shifted to the impulse."""
    W, H = 33, 2
    img = np.zeros((1, H, W), np.float32)
    img[0, 0, 10] = 1.0
    P = np.array([[[1e7, 0, 0, 16.0], [0, 1e7, 0, 0.5], [0, 0, 1.0, 1.0]]], np.float32)
    q = oracle.preweight_filter(img, P)
    d = np.abs(np.arange(W) - 10)
    h = np.where(d == 0, 0.25, np.where(d % 2 == 1, -1.0 / (np.pi ** 2 * np.maximum(d, 1) ** 2), 0.0))
    np.testing.assert_allclose(q[0, 0], h, rtol=1e-12, atol=1e-15)
    assert np.all(q[0, 1] == 0)


def test_filter_matches_fft_route_of_generator():
    """The direct FP64 convolution equals the generator's zero-padded FFT
    filtering (a different route to the same linear convolution)."""
    cfg = synth.preset("small", n_views=3)
    geo = synth.geometry(cfg)
    ph = synth.phantom(cfg)
    raw = synth.projections(cfg, geo, ph, filtered=False, dtype=torch.float64)
    filt = synth.projections(cfg, geo, ph, filtered=True, dtype=torch.float64).numpy()
    tau = cfg.pixel * cfg.sid / cfg.sdd
    dbeta = np.deg2rad(cfg.arc_deg) / (cfg.n_views - 1)
    # the generator scales by d_beta * tau and its kernel carries 1/tau^2
    q = oracle.preweight_filter(raw.float().numpy(), geo["mats"], scale=dbeta / tau)
    np.testing.assert_allclose(q, filt, rtol=0, atol=2e-6 * np.abs(filt).max())


def test_count_orthographic_closed_form():
    """w = 1, u = x/s + o_x/s, v = y/s + o_y/s: the pairs with -1 < u < W and
    -1 < v < H are counted in closed form.  Half-voxel offsets keep every
    pair 0.5 px from a decision (empty band); integer offsets put the column
    u = W exactly on one, where the strict bound excludes it and the band
    holds it."""
    P = np.stack([_ortho(2.0), _ortho(2.0)]).reshape(2, 12)
    dims, W, H = (10, 5, 3), 6, 8
    # u = x - 0.5: x in 0..6 (7 columns); v = y - 0.5: y in 0..4 (all 5 rows)
    c, b = oracle.count_updates(P, dims, (2, 2, 2), (-1.0, -1.0, 0.0), W, H)
    assert (c, b) == (2 * 7 * 5 * 3, 0)
    # u = x: x in 0..5 counted, x = 6 (u = W) in the band only
    c, b = oracle.count_updates(P, dims, (2, 2, 2), (0.0, 0.0, 0.0), W, H)
    assert (c, b) == (2 * 6 * 5 * 3, 2 * 1 * 5 * 3)


def test_count_matches_numpy_brute_force():
    """The threaded C count against a vectorised numpy evaluation of the same
    definition, on the tiny scan and on a volume that holds the source
    circle (w <= 0 pairs), for count and band alike, with any thread split."""
    for s in (_scan("tiny"), _scan("small", nx=40, ny=40, nz=8, voxel=10.0, sid=150.0, sdd=300.0)):
        d, vs, org = s["dims"], s["voxel_size"].astype(np.float64), s["origin"].astype(np.float64)
        W, H = s["cfg"].det_w, s["cfg"].det_h
        zz, yy, xx = np.meshgrid(*(np.arange(int(d[a])) for a in (2, 1, 0)), indexing="ij")
        X = np.stack([org[0] + xx * vs[0], org[1] + yy * vs[1], org[2] + zz * vs[2],
                      np.ones(xx.shape)], -1).reshape(-1, 4)
        cnt = band = 0
        for P in s["mats"].astype(np.float64):
            q = X @ P.T
            w = q[:, 2]
            near_w = np.abs(w) <= 1e-5
            front = (w > 0) & ~near_w
            u = np.where(front, q[:, 0] / np.where(front, w, 1.0), 0.0)
            v = np.where(front, q[:, 1] / np.where(front, w, 1.0), 0.0)
            cnt += int(np.sum(front & (u > -1) & (u < W) & (v > -1) & (v < H)))
            edge = (np.abs(u + 1) <= 1e-3) | (np.abs(u - W) <= 1e-3) | (np.abs(v + 1) <= 1e-3) | (np.abs(v - H) <= 1e-3)
            band += int(np.sum(near_w)) + int(np.sum(front & edge))
        for threads in (1, 3):
            assert oracle.count_updates(s["mats"], d, s["voxel_size"], s["origin"], W, H,
                                        threads=threads) == (cnt, band)


def test_count_scale_and_behind_source():
    """P -> 2P leaves u and v and the sign of w, so the count; P -> -P puts
    every voxel behind the source, so nothing is counted."""
    s = _scan("small")
    args = (s["dims"], s["voxel_size"], s["origin"], s["cfg"].det_w, s["cfg"].det_h)
    c, _ = oracle.count_updates(s["mats"], *args)
    assert c > 0
    assert oracle.count_updates((2.0 * s["mats"]).astype(np.float32), *args)[0] == c
    assert oracle.count_updates((-s["mats"]).astype(np.float32), *args)[0] == 0

