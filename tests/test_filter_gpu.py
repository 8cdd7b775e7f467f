"""GPU parity of the FDK pre-processing (cosine pre-weight + Ram-Lak row
filter, fdk_preweight_filter) against the FP64 oracle's direct convolution.

The device computes the row convolution by FFT in FP32; the bar is
max|diff| <= 3e-5 max|q| with PSNR >= 100 dB.  An independent FP32 route --
the same weights and zero-padded circular convolution through a
single-precision (complex64) FFT library on the host -- measures 1.4e-5 of
max|q| on the 2048 x 2 case below and 8e-6 on 1248 x 5, so the bar is about
twice what FP32 FFT arithmetic itself reaches on full 2048-pixel rows.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import assert_parity
from paper_1401_3615_gb300 import fdk

pytestmark = pytest.mark.gpu
TOL = 3e-5


def _raw(cfg):
    geo = synth.geometry(cfg)
    raw = synth.projections(cfg, geo, synth.phantom(cfg), device="cuda", filtered=False)
    return raw, geo["mats"]


@pytest.mark.parametrize("W,H", [(64, 48), (1, 5), (33, 7), (128, 3), (1000, 4),
                                 (1025, 3), (1248, 5), (1280, 3), (1281, 2), (2048, 2),
                                 (2049, 2), (3072, 2), (4096, 2)])
def test_filter_parity_shapes(W, H):
    cfg = synth.preset("small", n_views=3, det_w=W, det_h=H, pixel=0.308 * 1248.0 / W)
    raw, mats = _raw(cfg)
    out = torch.empty_like(raw)
    fdk.fdk_preweight_filter(out, raw, mats, scale=0.7)
    torch.cuda.synchronize()
    ref = oracle.preweight_filter(raw.cpu().numpy(), mats, scale=0.7)
    if np.abs(ref).max() == 0:
        assert torch.all(out == 0)
    else:
        assert_parity(ref, out.cpu().numpy(), rel_tol=TOL, psnr_min=100, what=f"filter {W}x{H}")


def test_filter_in_place_multi_pass_and_device_matrices():
    cfg = synth.preset("small", n_views=600, det_w=40, det_h=9, pixel=0.308 * 31.2)
    raw, mats = _raw(cfg)
    ref = oracle.preweight_filter(raw.cpu().numpy(), mats, scale=1.0)
    x = raw.clone()
    fdk.fdk_preweight_filter(x, x, mats)                     # in place, two passes of views
    y = torch.empty_like(raw)
    fdk.fdk_preweight_filter(y, raw, torch.from_numpy(mats).cuda())
    torch.cuda.synchronize()
    assert_parity(ref, x.cpu().numpy(), rel_tol=TOL, psnr_min=100)
    assert torch.equal(x, y)


@pytest.mark.parametrize("W", [1028, 1540])
def test_filter_register_fft_in_place_two_passes_device_matrices(W):
    """Rows of 1028 pixels (the N = 2560 register-FFT kernel) and 1540 (N =
    4096): 520 views in two passes of views, in place, and with device
    matrices."""
    cfg = synth.preset("small", n_views=520, det_w=W, det_h=3, pixel=0.308 * 1248.0 / W)
    raw, mats = _raw(cfg)
    ref = oracle.preweight_filter(raw.cpu().numpy(), mats, scale=1.0)
    x = raw.clone()
    fdk.fdk_preweight_filter(x, x, mats)
    y = torch.empty_like(raw)
    fdk.fdk_preweight_filter(y, raw, torch.from_numpy(mats).cuda())
    fdk.fdk_device_status()      # no bounded wait of the staged rows gave up
    assert_parity(ref, x.cpu().numpy(), rel_tol=TOL, psnr_min=100)
    assert torch.equal(x, y)


@pytest.mark.parametrize("W", [1248, 1604])
def test_filter_register_fft_staged_equals_unstaged_rows(W):
    """Rows of 1248 (N = 2560) and 1604 pixels (N = 4096) are copied into
    shared memory by bulk copies (16-byte aligned rows); the same images
    starting 4 bytes later take the direct-load variant.  Both give the same
    bits."""
    cfg = synth.preset("small", n_views=5, det_w=W, det_h=7, pixel=0.308 * 1248.0 / W)
    raw, mats = _raw(cfg)
    a = torch.empty_like(raw)
    fdk.fdk_preweight_filter(a, raw, mats, scale=0.5)
    flat = torch.zeros(raw.numel() + 1, device="cuda")
    shifted = flat[1:].view(raw.shape)
    shifted.copy_(raw)
    b = torch.empty_like(raw)
    fdk.fdk_preweight_filter(b, shifted, mats, scale=0.5)
    fdk.fdk_device_status()
    assert torch.equal(a, b)


def test_filter_full_detector():
    """1248 x 960 images of the benchmark geometry (3 views) against the
    oracle, and 8 views against the generator's own zero-padded FFT route
    (FP64), which computes the same linear convolution."""
    cfg = synth.preset("fdk512", n_views=8)
    geo = synth.geometry(cfg)
    ph = synth.phantom(cfg)
    raw = synth.projections(cfg, geo, ph, device="cuda", filtered=False)
    dbeta = np.deg2rad(cfg.arc_deg) / (cfg.n_views - 1)
    tau = cfg.pixel * cfg.sid / cfg.sdd        # detector pitch at the isocentre (mm)
    out = torch.empty_like(raw)
    fdk.fdk_preweight_filter(out, raw, geo["mats"], scale=dbeta / tau)
    fdk.fdk_device_status()
    got = out.cpu().numpy()
    ref3 = oracle.preweight_filter(raw[:3].cpu().numpy(), geo["mats"][:3], scale=dbeta / tau)
    assert_parity(ref3, got[:3], rel_tol=TOL, psnr_min=100, what="filter vs oracle")
    filt = synth.projections(cfg, geo, ph, device="cuda", filtered=True, dtype=torch.float64)
    assert_parity(filt.cpu().numpy(), got, rel_tol=TOL, psnr_min=100, what="filter vs generator")
