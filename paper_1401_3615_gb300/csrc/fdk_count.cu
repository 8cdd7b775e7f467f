// Clipped update count: voxel/view pairs whose footprint can touch the
// detector (w > 0, -1 < u < W, -1 < v < H), the count behind the paper's
// GUp/s figures (Sec. VII).  Reporting aid only; it shares the per-tile view
// table and the FP32 detector arithmetic of the back-projection kernel.
#include "fdk_tile.cuh"

namespace fdk {

template <int BX, int BY, int R>
__global__ void __launch_bounds__(BX * BY)
fdk_count_kernel(const __grid_constant__ BpArgs a, unsigned long long *count)
{
    constexpr int KC = 128;
    __shared__ ViewEntry tab[KC];
    __shared__ unsigned char cls[KC];
    __shared__ unsigned short act[KC];
    __shared__ int n_act;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * R;
    const int lx = threadIdx.x % BX, ly = threadIdx.x / BX;
    const int x = x0 + lx, y = y0 + ly;
    const float dxf = (float)(lx - BX / 2), dyf = (float)(ly - BY / 2);
    unsigned long long c = 0;
    for (int v0 = 0; v0 < a.n_views; v0 += KC) {
        const int nv = min(KC, a.n_views - v0);
        build_view_table<BX, BY, R>(a, v0, nv, x0, y0, z0, tab, cls, act, &n_act);
        if (x < a.g.nx && y < a.g.ny) {
            for (int q = 0; q < n_act; ++q) {
                const ViewEntry e = tab[act[q] & 1023];
                const float bu = fmaf(dyf, e.b.x, fmaf(dxf, e.a.z, e.a.x));
                const float bv = fmaf(dyf, e.b.y, fmaf(dxf, e.a.w, e.a.y));
                const float bw = fmaf(dyf, e.w.z, fmaf(dxf, e.w.y, e.w.x));
                for (int r = 0; r < R && z0 + r < a.g.nz; ++r) {
                    const float rf = (float)(r - R / 2);
                    const float wl = fmaf(rf, e.w.w, bw);
                    if (!(wl > 0.0f)) continue;
                    const float iw = rcp_approx(wl);
                    const float u = fmaf(fmaf(rf, e.b.z, bu), iw, e.o.x);
                    const float v = fmaf(fmaf(rf, e.b.w, bv), iw, e.o.y);
                    c += (u > -1.0f && u < (float)a.g.W && v > -1.0f && v < (float)a.g.H) ? 1 : 0;
                }
            }
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

fdk_status launch_count(const BpArgs &a, unsigned long long *count_dev, cudaStream_t s)
{
    constexpr int BX = 32, BY = 8, R = 8;
    dim3 grid((a.g.nx + BX - 1) / BX, (a.g.ny + BY - 1) / BY, (a.g.nz + R - 1) / R);
    fdk_count_kernel<BX, BY, R><<<grid, BX * BY, 0, s>>>(a, count_dev);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("count launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

}  // namespace fdk
