// Adjoint (transpose) of the back-projection: a voxel-driven bilinear splat.
//
// For every view k and voxel, with the same FP32 detector arithmetic as the
// back-projection kernel (the per-tile view table of fdk_tile.cuh), the
// voxel's value times 1/w^2 is spread over the four pixels around (u, v)
// with the bilinear weights (1-a)(1-b), a(1-b), (1-a)b, ab; pixels outside
// the image receive nothing.  This is exactly the transpose of the listing's
// gather (Listing 1), so <BP(y), x> = <y, BP^T(x)> up to FP32 rounding.
//
// Scatter strategy: per (tile, view) the CTA first accumulates into a
// shared-memory copy of the tile's detector footprint (its corner-derived
// pixel box) with shared atomics, then adds the non-zero cells to the
// projections with one global atomic each.  Footprints too large for the
// shared buffer fall back to direct global atomics.
#include "fdk_tile.cuh"

namespace fdk {

constexpr int kAdjBX = 16, kAdjBY = 16, kAdjR = 8, kAdjChunk = 64;
constexpr int kAdjCap = 6144;   // floats of shared footprint buffer (24 KB)

__device__ __forceinline__ void adj_tap(float *acc_s, float *proj, const int4 &bb, int W, int H,
                                        int ti, int tj, float val)
{
    if ((unsigned)ti >= (unsigned)W || (unsigned)tj >= (unsigned)H || val == 0.0f) return;
    const int li = ti - bb.x, lj = tj - bb.y;
    if ((unsigned)li < (unsigned)bb.z && (unsigned)lj < (unsigned)bb.w && bb.z * bb.w <= kAdjCap)
        atomicAdd(acc_s + lj * bb.z + li, val);
    else
        atomicAdd(proj + (long long)tj * W + ti, val);
}

template <int BX, int BY, int R>
__global__ void __launch_bounds__(BX * BY, 3)
fdk_adj_kernel(const __grid_constant__ BpArgs a, float *__restrict__ proj_out)
{
    constexpr int NT = BX * BY;
    __shared__ ViewEntry tab[kAdjChunk];
    __shared__ unsigned char cls[kAdjChunk];
    __shared__ unsigned short act[kAdjChunk];
    __shared__ int4 bbox[kAdjChunk];
    __shared__ int n_act;
    __shared__ float acc_s[kAdjCap];

    const int tid = threadIdx.x;
    for (int p = tid; p < kAdjCap; p += NT) acc_s[p] = 0.0f;

    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * R;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int WX = 8, WY = 4, WPX = BX / WX;
    const int lx = (warp % WPX) * WX + (lane % WX);
    const int ly = (warp / WPX) * WY + (lane / WX);
    const float dxf = (float)(lx - BX / 2), dyf = (float)(ly - BY / 2);
    const int W = a.g.W, H = a.g.H;

    // this thread's voxel values (zero past the volume edge)
    float f[R];
    const int x = x0 + lx, y = y0 + ly;
    const bool inxy = x < a.g.nx && y < a.g.ny;
    const long long sxy = (long long)a.g.nx * a.g.ny;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int z = z0 + r;
        f[r] = (inxy && z < a.g.nz) ? __ldg(a.vol + (long long)z * sxy + (long long)y * a.g.nx + x) : 0.0f;
    }

    for (int v0 = 0; v0 < a.n_views; v0 += kAdjChunk) {
        const int nv = min(kAdjChunk, a.n_views - v0);
        build_view_table<BX, BY, R>(a, v0, nv, x0, y0, z0, tab, cls, act, &n_act, bbox);
        const int n = n_act;
        for (int q = 0; q < n; ++q) {
            const int ev = act[q];
            const int lv = ev & 1023, c = ev >> 10;
            const ViewEntry e = tab[lv];
            const int4 bb = bbox[lv];
            float *proj = proj_out + (long long)(v0 + lv) * a.plane;
            const float bu = fmaf(dyf, e.b.x, fmaf(dxf, e.a.z, e.a.x));
            const float bv = fmaf(dyf, e.b.y, fmaf(dxf, e.a.w, e.a.y));
            const float bw = fmaf(dyf, e.w.z, fmaf(dxf, e.w.y, e.w.x));
            const int U = (int)e.o.x, V = (int)e.o.y;
            const float lou = -2.0f - e.o.x, lov = -2.0f - e.o.y;
            const float hiu = (float)(W + 1) - e.o.x, hiv = (float)(H + 1) - e.o.y;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float rf = (float)(r - R / 2);
                const float wl = fmaf(rf, e.w.w, bw);
                const float iw = rcp_approx(wl);
                float us = fmaf(rf, e.b.z, bu) * iw, vs = fmaf(rf, e.b.w, bv) * iw;
                us = fminf(fmaxf(us, lou), hiu);
                vs = fminf(fmaxf(vs, lov), hiv);
                const float tu = __fadd_rd(us, kFloorMagic), tv = __fadd_rd(vs, kFloorMagic);
                const float au = us - (tu - kFloorMagic), bvv = vs - (tv - kFloorMagic);
                const int i = __float_as_int(tu) - kFloorBits + U;
                const int j = __float_as_int(tv) - kFloorBits + V;
                float g = f[r] * iw * iw;
                if (c == kGeneral && !(wl > 0.0f)) g = 0.0f;
                const float gl = g * (1.0f - bvv), gh = g * bvv;
                adj_tap(acc_s, proj, bb, W, H, i, j, gl * (1.0f - au));
                adj_tap(acc_s, proj, bb, W, H, i + 1, j, gl * au);
                adj_tap(acc_s, proj, bb, W, H, i, j + 1, gh * (1.0f - au));
                adj_tap(acc_s, proj, bb, W, H, i + 1, j + 1, gh * au);
            }
            const int npx = bb.z * bb.w;
            if (npx > 0 && npx <= kAdjCap) {
                __syncthreads();
                for (int p = tid; p < npx; p += NT) {
                    const float s = acc_s[p];
                    if (s != 0.0f) {
                        atomicAdd(proj + (long long)(bb.y + p / bb.z) * W + bb.x + p % bb.z, s);
                        acc_s[p] = 0.0f;
                    }
                }
                __syncthreads();
            }
        }
        __syncthreads();   // the next chunk overwrites the table
    }
}

fdk_status launch_adjoint(const BpArgs &a, float *proj_out, cudaStream_t s)
{
    dim3 grid((a.g.nx + kAdjBX - 1) / kAdjBX, (a.g.ny + kAdjBY - 1) / kAdjBY, (a.g.nz + kAdjR - 1) / kAdjR);
    fdk_adj_kernel<kAdjBX, kAdjBY, kAdjR><<<grid, kAdjBX * kAdjBY, 0, s>>>(a, proj_out);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("adjoint launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

}  // namespace fdk
