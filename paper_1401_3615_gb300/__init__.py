"""GB300-native voxel-driven cone-beam back-projection (FDK hot path).

The compute lives in ``libfdk.so`` (hand-written sm_103a CUDA behind the C
ABI in ``include/fdk.h``); this package only marshals tensors into that ABI.
Importing the package does not load the library; the first call does, and it
raises if the library cannot be built or loaded -- there is no CPU fallback.
"""
from .fdk import (  # noqa: F401
    FdkError, FETCH_AUTO, FETCH_LDG, FETCH_TEX, FETCH_QUAD, FETCH_STAGE, fdk_backproject, fdk_backproject_host, fdk_backproject_static, fdk_forwardproject_adjoint,
    fdk_count_updates, fdk_last_error, fdk_release, fdk_version, library_path, BatchPlan,
    fdk_batch_plan_create, fdk_backproject_batched, fdk_preweight_filter, fdk_device_status, fdk_microbench,
)

__all__ = [
    "FdkError", "FETCH_AUTO", "FETCH_LDG", "FETCH_TEX", "FETCH_QUAD", "FETCH_STAGE", "fdk_backproject", "fdk_backproject_host", "fdk_backproject_static",
    "fdk_forwardproject_adjoint", "fdk_count_updates", "fdk_last_error", "fdk_release",
    "fdk_version", "library_path", "BatchPlan", "fdk_batch_plan_create", "fdk_backproject_batched",
    "fdk_preweight_filter", "fdk_device_status", "fdk_microbench",
]
