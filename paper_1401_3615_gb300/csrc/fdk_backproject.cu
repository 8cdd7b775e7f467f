// Dispatch of a back-projection pass to the fetch path and storage type.
#include "fdk_internal.cuh"

namespace fdk {

fdk_status launch_bp_ldg_f32(const BpArgs &a, int tile, cudaStream_t s);
fdk_status launch_bp_ldg_f16(const BpArgs &a, int tile, cudaStream_t s);
fdk_status launch_bp_ldg_bf16(const BpArgs &a, int tile, cudaStream_t s);
fdk_status launch_bp_tex_f32(const BpArgs &a, int tile, cudaStream_t s);
fdk_status launch_bp_tex_f16(const BpArgs &a, int tile, cudaStream_t s);
fdk_status launch_bp_tex_bf16(const BpArgs &a, int tile, cudaStream_t s);
fdk_status launch_bp_quad_f32(const BpArgs &a, int tile, cudaStream_t s);
fdk_status launch_bp_quad_f16(const BpArgs &a, int tile, cudaStream_t s);
fdk_status launch_bp_quad_bf16(const BpArgs &a, int tile, cudaStream_t s);
fdk_status launch_bp_stage(const BpArgs &a, int dtype, cudaStream_t s);

fdk_status launch_backproject(const BpArgs &a, int fetch, int dtype, int tile, cudaStream_t s)
{
    if (dtype != FDK_F32 && dtype != FDK_F16 && dtype != FDK_BF16) {
        set_error("unsupported projection dtype %d", dtype);
        return FDK_ERR_INVALID_ARG;
    }
    switch (fetch) {
    case FDK_FETCH_STAGE:
        return launch_bp_stage(a, dtype, s);
    case FDK_FETCH_TEX:
        return dtype == FDK_F32 ? launch_bp_tex_f32(a, tile, s)
             : dtype == FDK_F16 ? launch_bp_tex_f16(a, tile, s) : launch_bp_tex_bf16(a, tile, s);
    case FDK_FETCH_QUAD:
        return dtype == FDK_F32 ? launch_bp_quad_f32(a, tile, s)
             : dtype == FDK_F16 ? launch_bp_quad_f16(a, tile, s) : launch_bp_quad_bf16(a, tile, s);
    default:
        return dtype == FDK_F32 ? launch_bp_ldg_f32(a, tile, s)
             : dtype == FDK_F16 ? launch_bp_ldg_f16(a, tile, s) : launch_bp_ldg_bf16(a, tile, s);
    }
}

}  // namespace fdk
