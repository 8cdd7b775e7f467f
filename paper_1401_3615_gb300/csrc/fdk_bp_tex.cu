// Instantiations of the back-projection kernel: TEX fetch, float/half/bfloat16 storage.
#include "fdk_bp_kernel.cuh"

namespace fdk {

fdk_status launch_bp_tex_f32(const BpArgs &a, int tile, cudaStream_t s)
{
    return launch_tiles<kTex, float, false>(a, tile, s);
}

fdk_status launch_bp_tex_f16(const BpArgs &a, int tile, cudaStream_t s)
{
    return launch_tiles<kTex, __half, false>(a, tile, s);
}

fdk_status launch_bp_tex_bf16(const BpArgs &a, int tile, cudaStream_t s)
{
    return launch_tiles<kTex, __nv_bfloat16, false>(a, tile, s);
}

}  // namespace fdk
