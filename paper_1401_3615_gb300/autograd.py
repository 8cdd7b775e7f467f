"""torch.autograd wrappers around the library's back-projection and its transpose.

``backproject(proj, ...)`` is the linear map B of Listing 1 (projections ->
volume); its backward is the transpose B^T, computed by the library's
voxel-driven splat (``fdk_forwardproject_adjoint``).  ``forwardproject(vol,
...)`` is B^T (volume -> projections, the forward projector matched to B);
its backward is B.  Both run entirely in the library's kernels; the classes
here only route tensors.  Gradients flow to whichever inputs require them.
"""
from __future__ import annotations

import torch

from . import fdk as _fdk


class _Geometry:
    """Scan geometry shared by both operators."""

    def __init__(self, mats, voxel_size, origin, vol_shape, det_shape):
        self.mats = mats                      # host (n,12) array or CUDA tensor
        self.voxel_size = voxel_size
        self.origin = origin
        self.vol_shape = tuple(int(s) for s in vol_shape)    # (nz, ny, nx)
        self.det_shape = tuple(int(s) for s in det_shape)    # (n_views, H, W)


def _bp(g: _Geometry, proj: torch.Tensor) -> torch.Tensor:
    vol = torch.zeros(g.vol_shape, dtype=torch.float32, device=proj.device)
    _fdk.fdk_backproject(vol, proj.contiguous(), g.mats, g.voxel_size, g.origin)
    return vol


def _bpt(g: _Geometry, vol: torch.Tensor) -> torch.Tensor:
    proj = torch.zeros(g.det_shape, dtype=torch.float32, device=vol.device)
    _fdk.fdk_forwardproject_adjoint(proj, vol.contiguous(), g.mats, g.voxel_size, g.origin)
    return proj


class BackprojectFn(torch.autograd.Function):
    """volume = B(projections); d projections = B^T(d volume)."""

    @staticmethod
    def forward(ctx, proj: torch.Tensor, geom: _Geometry) -> torch.Tensor:
        ctx.geom = geom
        return _bp(geom, proj.float())

    @staticmethod
    def backward(ctx, grad_vol: torch.Tensor):
        grad_proj = _bpt(ctx.geom, grad_vol.float()) if ctx.needs_input_grad[0] else None
        return grad_proj, None


class ForwardProjectFn(torch.autograd.Function):
    """projections = B^T(volume); d volume = B(d projections)."""

    @staticmethod
    def forward(ctx, vol: torch.Tensor, geom: _Geometry) -> torch.Tensor:
        ctx.geom = geom
        return _bpt(geom, vol.float())

    @staticmethod
    def backward(ctx, grad_proj: torch.Tensor):
        grad_vol = _bp(ctx.geom, grad_proj.float()) if ctx.needs_input_grad[0] else None
        return grad_vol, None


def backproject(proj: torch.Tensor, mats, voxel_size, origin, vol_shape) -> torch.Tensor:
    """Differentiable back-projection of proj (n_views, H, W) into a new
    (nz, ny, nx) volume."""
    g = _Geometry(mats, voxel_size, origin, vol_shape, proj.shape)
    return BackprojectFn.apply(proj, g)


def forwardproject(vol: torch.Tensor, mats, voxel_size, origin, det_shape) -> torch.Tensor:
    """Differentiable transpose: volume (nz, ny, nx) -> projections
    (n_views, H, W) = det_shape."""
    g = _Geometry(mats, voxel_size, origin, vol.shape, det_shape)
    return ForwardProjectFn.apply(vol, g)
