"""Seeded synthetic cone-beam scans shaped like the paper's workload.

The paper benchmarks on the RabbitCT rabbit scan: 496 filtered projections of
1248x960 FP32 pixels from a C-arm short scan, each with a 3x4 projection
matrix, reconstructed into a 512^3 (or 1024^3) FP32 volume (Sec. IV,
Sec. VIII).  That data set is not available here, so this module builds a
stand-in with the same shapes:

* geometry: circular short scan over 200 degrees at uniform angles, source to
  isocentre 600 mm, source to detector 1200 mm, 0.308 mm pixels, principal
  point at the detector centre plus a seeded +-2 px jitter and seeded +-0.5
  degree tilts of the camera axes, all folded into row-major 3x4 FP32
  matrices scaled so that w is the depth along the principal axis divided
  by the source-isocentre distance (w = 1 at the isocentre; the listing's
  1/w^2 is then exactly the FDK distance weight (SID/U)^2);
* phantom: seeded ellipsoids with densities in [0.1, 1.0];
* projections: analytic FP64 line integrals through the phantom,
  cosine-weighted and Ram-Lak filtered along detector rows, stored as FP32
  (or BF16/FP16 for the storage-precision form).

This module is shared by the oracle tests and the GPU path and holds none of
the back-projection arithmetic: it only makes inputs.  Every random draw comes
from ``numpy.random.default_rng(seed)``; the heavy loops run in torch float64
on whichever device is given, so the same seed gives the same scan (to FP64
rounding) on the CPU and on the GPU.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import torch

__all__ = [
    "ScanConfig", "PRESETS", "preset", "geometry", "phantom", "projections",
    "volume_geometry", "make_scan", "gaussian_volume", "gaussian_projections",
    "batch_scan_configs", "small_batch_scan_configs", "from_column_major",
]


@dataclasses.dataclass(frozen=True)
class ScanConfig:
    """One synthetic scan.  Lengths in mm, angles in degrees."""
    nx: int = 128
    ny: int = 128
    nz: int = 128
    voxel: float = 2.0            # isotropic voxel pitch (the paper's MM)
    n_views: int = 496
    det_w: int = 1248             # detector columns (u)
    det_h: int = 960              # detector rows (v)
    pixel: float = 0.308          # detector pixel pitch
    sid: float = 600.0            # source to isocentre
    sdd: float = 1200.0           # source to detector
    arc_deg: float = 200.0        # short-scan arc
    jitter_px: float = 2.0        # principal-point jitter amplitude
    tilt_deg: float = 0.5         # camera-axis tilt amplitude
    n_ellipsoids: int = 10
    seed: int = 1234

    @property
    def updates(self) -> int:
        """Voxel/view pairs: the update count of one full back-projection."""
        return self.nx * self.ny * self.nz * self.n_views


# Named workloads.  All volumes are a 256 mm cube centred at the isocentre.
PRESETS = {
    # 128^3, 2 mm voxels, 496 views of 1248x960: about 1.04e9 updates.
    "fdk128": ScanConfig(nx=128, ny=128, nz=128, voxel=2.0, seed=101),
    # 512^3, 0.5 mm voxels, 496 views: the headline 6.66e10-update run.
    "fdk512": ScanConfig(nx=512, ny=512, nz=512, voxel=0.5, seed=202),
    # 1024^3, 0.25 mm voxels, 496 views (the storage-precision form).
    "fdk1024": ScanConfig(nx=1024, ny=1024, nz=1024, voxel=0.25, seed=303),
    # 256^3, 1 mm voxels, 248 views (the differentiation form).
    "fdk256": ScanConfig(nx=256, ny=256, nz=256, voxel=1.0, n_views=248, seed=404),
    # Small cases for CPU tests and quick GPU parity runs.
    "tiny": ScanConfig(nx=8, ny=8, nz=8, voxel=32.0, n_views=4, det_w=24, det_h=16,
                       pixel=0.308 * 52, seed=7),
    "small": ScanConfig(nx=24, ny=20, nz=18, voxel=10.0, n_views=12, det_w=64, det_h=48,
                        pixel=0.308 * 19.5, seed=11),
}


def preset(name: str, **overrides) -> ScanConfig:
    return dataclasses.replace(PRESETS[name], **overrides)


def _rot(axis: np.ndarray, ang: float) -> np.ndarray:
    """Rodrigues rotation matrix about a unit axis (radians)."""
    a = axis / np.linalg.norm(axis)
    k = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * k + (1 - math.cos(ang)) * (k @ k)


def geometry(cfg: ScanConfig) -> dict:
    """Per-view projection matrices of a perturbed circular short scan.

    Returns ``mats`` (n_views, 3, 4) float32 row-major and, in float64, the
    source positions, the world-to-camera rotations, focal length and
    principal points needed to trace the detector rays.  Pixel (m, n) has its
    centre at detector coordinate (u, v) = (m, n); the matrix maps a world
    point X (mm) to (u', v', w) = P (X, 1) with u = u'/w, v = v'/w and w the
    depth of X along the principal axis divided by SID.
    """
    rng = np.random.default_rng(cfg.seed)
    n = cfg.n_views
    theta = np.deg2rad(np.linspace(0.0, cfg.arc_deg, n) if n > 1 else np.zeros(1))
    jit = rng.uniform(-cfg.jitter_px, cfg.jitter_px, size=(n, 2))
    tilt = np.deg2rad(rng.uniform(-cfg.tilt_deg, cfg.tilt_deg, size=(n, 3)))
    f = cfg.sdd / cfg.pixel
    u0 = (cfg.det_w - 1) / 2.0 + jit[:, 0]
    v0 = (cfg.det_h - 1) / 2.0 + jit[:, 1]
    mats = np.zeros((n, 3, 4))
    src = np.zeros((n, 3))
    rcam = np.zeros((n, 3, 3))
    for k in range(n):
        c, s = math.cos(theta[k]), math.sin(theta[k])
        S = cfg.sid * np.array([c, s, 0.0])
        e_w = -S / cfg.sid                      # principal axis, source -> isocentre
        e_u = np.array([-s, c, 0.0])            # tangential detector axis
        e_v = np.array([0.0, 0.0, 1.0])         # rotation axis
        R = np.stack([e_u, e_v, e_w])           # rows: camera axes in world frame
        T = _rot(e_u, tilt[k, 0]) @ _rot(e_v, tilt[k, 1]) @ _rot(e_w, tilt[k, 2])
        R = R @ T.T
        Kc = np.array([[f, 0.0, u0[k]], [0.0, f, v0[k]], [0.0, 0.0, 1.0]])
        P = Kc @ np.concatenate([R, (-R @ S)[:, None]], axis=1)
        P /= np.linalg.norm(P[2, :3]) * cfg.sid
        mats[k] = P
        src[k] = S
        rcam[k] = R
    return {
        "mats": mats.astype(np.float32),
        "mats64": mats,
        "source": src,
        "rcam": rcam,
        "focal_px": f,
        "u0": u0,
        "v0": v0,
    }


def phantom(cfg: ScanConfig) -> dict:
    """Seeded ellipsoids inside the field of view (radius <= 90 mm, |z| <= 70 mm).

    Returns centres (E,3), semi-axes (E,3), rotations (E,3,3, columns are the
    ellipsoid axes in world coordinates) and densities (E,), float64.
    """
    rng = np.random.default_rng(cfg.seed + 7919)
    e = cfg.n_ellipsoids
    axes = rng.uniform(8.0, 40.0, size=(e, 3))
    centres = np.zeros((e, 3))
    for i in range(e):
        rmax = 90.0 - axes[i].max()
        r = rmax * math.sqrt(rng.uniform(0.0, 1.0))
        phi = rng.uniform(0.0, 2 * math.pi)
        zmax = 70.0 - axes[i].max()
        centres[i] = [r * math.cos(phi), r * math.sin(phi), rng.uniform(-zmax, zmax)]
    rots = np.zeros((e, 3, 3))
    for i in range(e):
        q, rr = np.linalg.qr(rng.normal(size=(3, 3)))
        rots[i] = q * np.sign(np.diag(rr))
    dens = rng.uniform(0.1, 1.0, size=e)
    return {"centres": centres, "axes": axes, "rots": rots, "density": dens}


def _ramlak_kernel(n_fft: int, tau: float, device) -> torch.Tensor:
    """FFT of the discrete Ram-Lak kernel (Kak & Slaney): h(0)=1/(4 tau^2),
    h(odd n) = -1/(n^2 pi^2 tau^2), h(even n != 0) = 0, laid out for circular
    convolution of length n_fft (negative lags wrapped to the end)."""
    idx = torch.arange(n_fft, dtype=torch.float64, device=device)
    lag = torch.where(idx <= n_fft // 2, idx, idx - n_fft)
    h = torch.zeros(n_fft, dtype=torch.float64, device=device)
    odd = (lag.abs() % 2) == 1
    h[odd] = -1.0 / (lag[odd] ** 2 * math.pi ** 2 * tau ** 2)
    h[0] = 1.0 / (4.0 * tau ** 2)
    return torch.fft.rfft(h)


def projections(cfg: ScanConfig, geo: Optional[dict] = None, ph: Optional[dict] = None,
                device="cpu", dtype=torch.float32, filtered: bool = True,
                chunk: int = 8) -> torch.Tensor:
    """Filtered projections (n_views, det_h, det_w) on ``device`` in ``dtype``.

    Each pixel holds the FP64 line integral of the phantom along the ray from
    the source through the pixel centre, times the cosine pre-weight
    SDD / sqrt(SDD^2 + u_mm^2 + v_mm^2), Ram-Lak filtered along rows (spacing
    scaled to the isocentre) and scaled by d_beta, so that with w = depth/SID
    the back-projection is an FDK reconstruction up to short-scan redundancy.
    With ``filtered=False`` the raw line integrals are returned.
    """
    geo = geometry(cfg) if geo is None else geo
    ph = phantom(cfg) if ph is None else ph
    dev = torch.device(device)
    W, H, n = cfg.det_w, cfg.det_h, cfg.n_views
    out = torch.empty((n, H, W), dtype=dtype, device=dev)
    f = geo["focal_px"]
    mm = torch.arange(W, dtype=torch.float64, device=dev)
    nn = torch.arange(H, dtype=torch.float64, device=dev)
    cen = torch.tensor(ph["centres"], device=dev)
    ax = torch.tensor(ph["axes"], device=dev)
    rot = torch.tensor(ph["rots"], device=dev)
    dens = torch.tensor(ph["density"], device=dev)
    tau = cfg.pixel * cfg.sid / cfg.sdd
    n_fft = 1 << int(math.ceil(math.log2(2 * W - 1)))
    Hk = _ramlak_kernel(n_fft, tau, dev)
    dbeta = math.radians(cfg.arc_deg) / max(n - 1, 1)
    scale = dbeta * tau
    for k0 in range(0, n, chunk):
        ks = list(range(k0, min(n, k0 + chunk)))
        b = len(ks)
        u0 = torch.tensor(geo["u0"][ks], device=dev).view(b, 1, 1)
        v0 = torch.tensor(geo["v0"][ks], device=dev).view(b, 1, 1)
        R = torch.tensor(geo["rcam"][ks], device=dev)             # (b,3,3)
        S = torch.tensor(geo["source"][ks], device=dev)           # (b,3)
        cu = ((mm.view(1, 1, W) - u0) / f).expand(b, H, W)
        cv = ((nn.view(1, H, 1) - v0) / f).expand(b, H, W)
        # ray direction in camera frame (cu, cv, 1) -> world: R^T d_cam
        dwx = R[:, 0, 0].view(b, 1, 1) * cu + R[:, 1, 0].view(b, 1, 1) * cv + R[:, 2, 0].view(b, 1, 1)
        dwy = R[:, 0, 1].view(b, 1, 1) * cu + R[:, 1, 1].view(b, 1, 1) * cv + R[:, 2, 1].view(b, 1, 1)
        dwz = R[:, 0, 2].view(b, 1, 1) * cu + R[:, 1, 2].view(b, 1, 1) * cv + R[:, 2, 2].view(b, 1, 1)
        norm = torch.sqrt(dwx * dwx + dwy * dwy + dwz * dwz)
        dwx, dwy, dwz = dwx / norm, dwy / norm, dwz / norm
        line = torch.zeros((b, H, W), dtype=torch.float64, device=dev)
        for e in range(cen.shape[0]):
            Q = rot[e]                                            # columns: axes
            p = (S - cen[e]) @ Q / ax[e]                          # (b,3) source in unit-sphere frame
            qx = (dwx * Q[0, 0] + dwy * Q[1, 0] + dwz * Q[2, 0]) / ax[e, 0]
            qy = (dwx * Q[0, 1] + dwy * Q[1, 1] + dwz * Q[2, 1]) / ax[e, 1]
            qz = (dwx * Q[0, 2] + dwy * Q[1, 2] + dwz * Q[2, 2]) / ax[e, 2]
            A = qx * qx + qy * qy + qz * qz
            B = p[:, 0].view(b, 1, 1) * qx + p[:, 1].view(b, 1, 1) * qy + p[:, 2].view(b, 1, 1) * qz
            C = (p * p).sum(dim=1).view(b, 1, 1) - 1.0
            disc = torch.clamp(B * B - A * C, min=0.0)
            line += dens[e] * 2.0 * torch.sqrt(disc) / A
        if filtered:
            # cosine pre-weight: cos of the angle between ray and principal axis
            cosw = 1.0 / torch.sqrt(1.0 + cu * cu + cv * cv)
            g = line * cosw
            G = torch.fft.rfft(g, n=n_fft, dim=-1)
            q = torch.fft.irfft(G * Hk, n=n_fft, dim=-1)[..., :W]
            line = q * scale
        out[k0:k0 + b] = line.to(dtype)
    return out


def volume_geometry(cfg: ScanConfig):
    """(dims, voxel_size, origin) of a volume centred at the isocentre.

    dims = (nx, ny, nz); origin is the world position (mm) of the centre of
    voxel (0,0,0): -(n-1)/2 * voxel per axis.  Both float arrays are float32,
    the precision the library takes them in.
    """
    dims = np.array([cfg.nx, cfg.ny, cfg.nz], dtype=np.int32)
    vs = np.full(3, cfg.voxel, dtype=np.float32)
    org = (-(dims.astype(np.float64) - 1) / 2.0 * cfg.voxel).astype(np.float32)
    return dims, vs, org


def make_scan(cfg: ScanConfig, device="cpu", dtype=torch.float32, filtered=True) -> dict:
    """Everything one back-projection needs, generated from ``cfg.seed``."""
    geo = geometry(cfg)
    ph = phantom(cfg)
    proj = projections(cfg, geo, ph, device=device, dtype=dtype, filtered=filtered)
    dims, vs, org = volume_geometry(cfg)
    return {"cfg": cfg, "proj": proj, "mats": geo["mats"], "dims": dims,
            "voxel_size": vs, "origin": org, "geo": geo, "phantom": ph}


def gaussian_volume(dims, seed: int) -> np.ndarray:
    """Seeded N(0,1) FP32 volume (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = (int(d) for d in dims)
    return rng.standard_normal((nz, ny, nx)).astype(np.float32)


def gaussian_projections(n_views: int, det_h: int, det_w: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) FP32 projection stack (n_views, det_h, det_w)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_views, det_h, det_w)).astype(np.float32)


def batch_scan_configs(n_scans: int = 32, seed: int = 505) -> list:
    """Seeded uneven scans for the batched form: volumes 64..384 per axis
    (non-cubic), 120..496 views, detectors from 640x480 to 1248x960.  The
    pixel pitch is scaled so each detector spans the same field as the
    1248x960 / 0.308 mm panel; the volume stays a 256 mm cube."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scans):
        nx, ny, nz = (int(v) for v in rng.integers(64, 385, size=3))
        views = int(rng.integers(120, 497))
        w = int(rng.integers(640, 1249))
        h = int(rng.integers(480, 961))
        pix = 0.308 * 1248.0 / w
        out.append(ScanConfig(nx=nx, ny=ny, nz=nz, voxel=256.0 / max(nx, ny, nz),
                              n_views=views, det_w=w, det_h=h, pixel=pix,
                              seed=int(rng.integers(1, 2 ** 31))))
    return out


def small_batch_scan_configs(n_scans: int = 128, seed: int = 606) -> list:
    """Seeded small scans for the batched form, each too small to fill the GPU
    on its own: volumes 32..96 voxels per axis (non-cubic), 60..180 views,
    detectors from 320x240 to 640x480 with the pixel pitch scaled so each
    spans the field of the 1248x960 / 0.308 mm panel; the volume stays a
    256 mm cube."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scans):
        nx, ny, nz = (int(v) for v in rng.integers(32, 97, size=3))
        views = int(rng.integers(60, 181))
        w = int(rng.integers(320, 641))
        h = int(rng.integers(240, 481))
        pix = 0.308 * 1248.0 / w
        out.append(ScanConfig(nx=nx, ny=ny, nz=nz, voxel=256.0 / max(nx, ny, nz),
                              n_views=views, det_w=w, det_h=h, pixel=pix,
                              seed=int(rng.integers(1, 2 ** 31))))
    return out


def from_column_major(a: np.ndarray) -> np.ndarray:
    """Convert matrices stored column-major as in the paper's listing
    (A[0], A[3], A[6], A[9] form the u row) to row-major (n, 3, 4)."""
    a = np.asarray(a, dtype=np.float32).reshape(-1, 12)
    return np.ascontiguousarray(a.reshape(-1, 4, 3).transpose(0, 2, 1))
