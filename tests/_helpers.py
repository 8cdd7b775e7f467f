"""Shared helpers for the parity tests (no method arithmetic here)."""
import numpy as np

# Accuracy bar for FP32 GPU results against the FP64 oracle: the maximum
# absolute difference at most 1e-4 of the oracle's maximum magnitude, and a
# PSNR (peak = max |f_oracle|) of at least 80 dB.
REL_TOL = 1e-4
PSNR_MIN = 80.0


def psnr(ref: np.ndarray, got: np.ndarray) -> float:
    ref = np.asarray(ref, dtype=np.float64)
    got = np.asarray(got, dtype=np.float64)
    mse = float(np.mean((ref - got) ** 2))
    peak = float(np.abs(ref).max())
    if mse == 0.0:
        return float("inf")
    return 10.0 * np.log10(peak * peak / mse)


def assert_parity(ref, got, rel_tol=REL_TOL, psnr_min=PSNR_MIN, what=""):
    ref = np.asarray(ref, dtype=np.float64)
    got = np.asarray(got, dtype=np.float64)
    assert ref.shape == got.shape, (ref.shape, got.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite values"
    peak = float(np.abs(ref).max())
    err = float(np.abs(ref - got).max())
    p = psnr(ref, got)
    assert err <= rel_tol * peak, f"{what}: max|diff| {err:.3e} > {rel_tol:g} * {peak:.3e} (psnr {p:.1f})"
    assert p >= psnr_min, f"{what}: PSNR {p:.1f} dB < {psnr_min}"
    return err / peak if peak > 0 else 0.0, p
