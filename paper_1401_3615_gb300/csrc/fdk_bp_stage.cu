// The plain staged back-projection: one CTA per 16 x 16 x 16 tile (the
// pipeline itself is in fdk_stage.cuh).
#include "fdk_stage.cuh"

namespace fdk {

template <int BX, int BY, int WX, int R, int MINB, bool FIDX, typename T>
__global__ void __launch_bounds__(BX * BY, MINB)
fdk_bp_stage_kernel(const __grid_constant__ BpArgs a)
{
    __shared__ StageTables t;
    __shared__ __align__(8) StageBarriers sb;
    extern __shared__ __align__(1024) float stages[];
    // CTAs are scheduled in blockIdx.x order: walking along the rays keeps
    // the resident CTAs' footprints overlapping, so their boxes hit in L2
    const int tx = a.walk_y ? blockIdx.y : blockIdx.x, ty = a.walk_y ? blockIdx.x : blockIdx.y;
    stage_init(sb);
    stage_tile<BX, BY, WX, R, FIDX, kNumBoxH, BpArgs, T>(a, a.tmap, a.err, a.wait_limit, tx * BX, ty * BY,
                                                         blockIdx.z * R, t, sb, stages);
}

template <int WX, bool FIDX, typename T>
static fdk_status launch_stage_shape(const BpArgs &a, cudaStream_t s)
{
    constexpr int BX = 16, BY = 16, R = 16, MINB = 3;
    auto k = fdk_bp_stage_kernel<BX, BY, WX, R, MINB, FIDX, T>;
    const int smem = kStages * kStageFloats * (int)sizeof(float);
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) {
        set_error("staged back-projection: cudaFuncSetAttribute failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    const unsigned gx = (a.g.nx + BX - 1) / BX, gy = (a.g.ny + BY - 1) / BY;
    dim3 grid(a.walk_y ? gy : gx, a.walk_y ? gx : gy, (a.g.nz + R - 1) / R);
    k<<<grid, BX * BY, smem, s>>>(a);
    err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("staged back-projection launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

// 16 x 16 x 16 tiles; a.tmap holds the pass's tensor maps (of T pixels).
template <typename T>
static fdk_status launch_stage_typed(const BpArgs &a, cudaStream_t s)
{
    const bool fidx = (long long)a.g.W * (a.g.H + 1) < (1LL << 23);
    if (a.warp_x == 4) return fidx ? launch_stage_shape<4, true, T>(a, s) : launch_stage_shape<4, false, T>(a, s);
    return fidx ? launch_stage_shape<8, true, T>(a, s) : launch_stage_shape<8, false, T>(a, s);
}

fdk_status launch_bp_stage(const BpArgs &a, int dtype, cudaStream_t s)
{
    if (dtype == FDK_F16) return launch_stage_typed<__half>(a, s);
    if (dtype == FDK_BF16) return launch_stage_typed<__nv_bfloat16>(a, s);
    return launch_stage_typed<float>(a, s);
}

}  // namespace fdk
