// Instantiations of the back-projection kernel: QUAD fetch, float/half/bfloat16 storage.
#include "fdk_bp_kernel.cuh"

namespace fdk {

fdk_status launch_bp_quad_f32(const BpArgs &a, int tile, cudaStream_t s)
{
    return launch_tiles<kQuad, float, false>(a, tile, s);
}

fdk_status launch_bp_quad_f16(const BpArgs &a, int tile, cudaStream_t s)
{
    return launch_tiles<kQuad, __half, false>(a, tile, s);
}

fdk_status launch_bp_quad_bf16(const BpArgs &a, int tile, cudaStream_t s)
{
    return launch_tiles<kQuad, __nv_bfloat16, false>(a, tile, s);
}

}  // namespace fdk
