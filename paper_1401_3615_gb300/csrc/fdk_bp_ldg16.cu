// Instantiations of the back-projection kernel: LDG fetch, half/bfloat16 storage.
#include "fdk_bp_kernel.cuh"

namespace fdk {

fdk_status launch_bp_ldg_f16(const BpArgs &a, int tile, cudaStream_t s)
{
    // the float flat index is exact while every tap index is below 2^23
    if ((long long)a.g.W * (a.g.H + 1) < (1LL << 23)) return launch_tiles<kLdg, __half, true>(a, tile, s);
    return launch_tiles<kLdg, __half, false>(a, tile, s);
}

fdk_status launch_bp_ldg_bf16(const BpArgs &a, int tile, cudaStream_t s)
{
    // the float flat index is exact while every tap index is below 2^23
    if ((long long)a.g.W * (a.g.H + 1) < (1LL << 23)) return launch_tiles<kLdg, __nv_bfloat16, true>(a, tile, s);
    return launch_tiles<kLdg, __nv_bfloat16, false>(a, tile, s);
}

}  // namespace fdk
