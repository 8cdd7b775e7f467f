// Voxel-driven cone-beam back-projection kernels (Listing 1, Sec. IV).
//
// Work decomposition: a CTA owns a BX x BY x R box of voxels; each thread
// owns one (x, y) column of R consecutive z voxels and keeps their sums in
// registers across every view of the pass, so the volume is read once and
// written once per pass (up to 512 views) instead of once per view.  Views
// are visited in index order, so each voxel sums its views in the same
// order as the definition.
//
// Per view and voxel the hot loop does, in FP32:
//   u'_l, v'_l, w   = three FMAs from per-(tile, view) coefficients
//   r = 1/w (MUFU), u = u'_l r, v = v'_l r (cell-relative detector position)
//   floor, fractions a, b
//   four taps: a 2x2 texture gather with zero border (TEX path), or four
//   read-only loads (LDG path, bounds-checked only on boundary tiles)
//   three lerps, acc += val * r * r
#include "fdk_tile.cuh"

namespace fdk {

template <typename T> struct Elem;
template <> struct Elem<float> {
    static __device__ __forceinline__ float load(const float *p) { return __ldg(p); }
};
template <> struct Elem<__half> {
    static __device__ __forceinline__ float load(const __half *p) { return __half2float(__ldg(p)); }
};
template <> struct Elem<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16 *p)
    {
        const unsigned short b = __ldg(reinterpret_cast<const unsigned short *>(p));
        return __uint_as_float((unsigned)b << 16);
    }
};

// 2x2 gather of texels (i, j), (i+1, j), (i, j+1), (i+1, j+1) returned as
// (p00, p10, p01, p11).  (x, y) = (i + 1, j + 1) sits exactly on the corner
// shared by the four texel centres, so the hardware footprint selection
// agrees with floor() in FP32.
template <typename T> struct Gather;
template <> struct Gather<float> {
    static __device__ __forceinline__ float4 fetch(cudaTextureObject_t t, float x, float y)
    {
        const float4 g = tex2Dgather<float4>(t, x, y, 0);
        return make_float4(g.w, g.z, g.x, g.y);
    }
};
template <> struct Gather<__half> {
    static __device__ __forceinline__ float4 fetch(cudaTextureObject_t t, float x, float y)
    {
        const float4 g = tex2Dgather<float4>(t, x, y, 0);
        return make_float4(g.w, g.z, g.x, g.y);
    }
};
template <> struct Gather<__nv_bfloat16> {
    static __device__ __forceinline__ float4 fetch(cudaTextureObject_t t, float x, float y)
    {
        const ushort4 g = tex2Dgather<ushort4>(t, x, y, 0);
        return make_float4(__uint_as_float((unsigned)g.w << 16), __uint_as_float((unsigned)g.z << 16),
                           __uint_as_float((unsigned)g.x << 16), __uint_as_float((unsigned)g.y << 16));
    }
};

enum Fetch : int { kLdg = 1, kTex = 2 };

// One view against this thread's R voxels.  MODE: kInterior (no checks),
// kBoundary (tap bounds checks), kGeneral (bounds and per-voxel w > 0).
template <int R, int FETCH, int MODE, typename T>
__device__ __forceinline__ void bp_view(float (&acc)[R], const ViewEntry &e, float dxf, float dyf,
                                        const T *img, int W, int H, cudaTextureObject_t tex)
{
    const float bu = fmaf(dyf, e.ru.z, fmaf(dxf, e.ru.y, e.ru.x));
    const float bv = fmaf(dyf, e.rv.z, fmaf(dxf, e.rv.y, e.rv.x));
    const float bw = fmaf(dyf, e.rw.z, fmaf(dxf, e.rw.y, e.rw.x));
    const int U = __float_as_int(e.off.z), V = __float_as_int(e.off.w);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float rf = (float)(r - R / 2);
        const float ul = fmaf(rf, e.ru.w, bu);
        const float vl = fmaf(rf, e.rv.w, bv);
        const float wl = fmaf(rf, e.rw.w, bw);
        const float iw = rcp_approx(wl);
        float us = ul * iw, vs = vl * iw;
        if (MODE != kInterior) {
            // keep far-off rays in a range where the int conversions are exact;
            // every tap there is outside the image either way
            us = fminf(fmaxf(us, -4.0f - (float)U), (float)(W + 4 - U));
            vs = fminf(fmaxf(vs, -4.0f - (float)V), (float)(H + 4 - V));
        }
        const float fu = floorf(us), fv = floorf(vs);
        const float a = us - fu, b = vs - fv;
        float p00, p10, p01, p11;
        if (FETCH == kTex) {
            const float4 g = Gather<T>::fetch(tex, fu + e.off.x, fv + e.off.y);
            p00 = g.x; p10 = g.y; p01 = g.z; p11 = g.w;
        } else if (MODE == kInterior) {
            const T *p = img + ((int)fv + V) * W + ((int)fu + U);
            p00 = Elem<T>::load(p);
            p10 = Elem<T>::load(p + 1);
            p01 = Elem<T>::load(p + W);
            p11 = Elem<T>::load(p + W + 1);
        } else {
            const int i = (int)fu + U, j = (int)fv + V;
            const bool c0 = (unsigned)i < (unsigned)W, c1 = (unsigned)(i + 1) < (unsigned)W;
            const bool r0 = (unsigned)j < (unsigned)H, r1 = (unsigned)(j + 1) < (unsigned)H;
            // clamp the address into the image, zero the tap if it was outside
            const int ic0 = min(max(i, 0), W - 1), ic1 = min(max(i + 1, 0), W - 1);
            const int jc0 = min(max(j, 0), H - 1), jc1 = min(max(j + 1, 0), H - 1);
            p00 = Elem<T>::load(img + jc0 * W + ic0);
            p10 = Elem<T>::load(img + jc0 * W + ic1);
            p01 = Elem<T>::load(img + jc1 * W + ic0);
            p11 = Elem<T>::load(img + jc1 * W + ic1);
            p00 = (c0 && r0) ? p00 : 0.0f;
            p10 = (c1 && r0) ? p10 : 0.0f;
            p01 = (c0 && r1) ? p01 : 0.0f;
            p11 = (c1 && r1) ? p11 : 0.0f;
        }
        const float lo = fmaf(a, p10 - p00, p00);
        const float hi = fmaf(a, p11 - p01, p01);
        float val = fmaf(b, hi - lo, lo);
        float iw2 = iw * iw;
        if (MODE == kGeneral) {
            const bool front = wl > 0.0f;
            val = front ? val : 0.0f;
            iw2 = front ? iw2 : 0.0f;
        }
        acc[r] = fmaf(val, iw2, acc[r]);
    }
}

// CTA tile BX x BY x R; warps cover WX x (32/WX) voxel patches in (x, y).
template <int BX, int BY, int WX, int R, int FETCH, typename T>
__global__ void __launch_bounds__(BX * BY)
fdk_bp_kernel(const __grid_constant__ BpArgs a)
{
    static_assert(32 % WX == 0 && BX % WX == 0 && BY % (32 / WX) == 0, "warp tiling");
    constexpr int WY = 32 / WX;
    constexpr int WPX = BX / WX;
    __shared__ ViewEntry tab[KMAX];
    __shared__ unsigned char cls[KMAX];
    __shared__ unsigned short act[KMAX];
    __shared__ int n_act;

    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * R;
    build_view_table<BX, BY, R>(a, x0, y0, z0, tab, cls, act, &n_act);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lx = (warp % WPX) * WX + (lane % WX);
    const int ly = (warp / WPX) * WY + (lane / WX);
    const float dxf = (float)(lx - BX / 2), dyf = (float)(ly - BY / 2);
    const int W = a.g.W, H = a.g.H;
    const T *proj = static_cast<const T *>(a.proj);

    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0f;

    const int n = n_act;
    for (int q = 0; q < n; ++q) {
        const int ev = act[q];
        const int v = ev & 1023, c = ev >> 10;
        const ViewEntry e = tab[v];
        const T *img = proj + (long long)v * a.plane;
        const cudaTextureObject_t tex = (FETCH == kTex) ? (cudaTextureObject_t)a.tex[v] : 0;
        if (c == kInterior) {
            bp_view<R, FETCH, kInterior, T>(acc, e, dxf, dyf, img, W, H, tex);
        } else if (c == kBoundary) {
            bp_view<R, FETCH, kBoundary, T>(acc, e, dxf, dyf, img, W, H, tex);
        } else {
            bp_view<R, FETCH, kGeneral, T>(acc, e, dxf, dyf, img, W, H, tex);
        }
    }

    const int x = x0 + lx, y = y0 + ly;
    if (x < a.g.nx && y < a.g.ny) {
        const long long sxy = (long long)a.g.nx * a.g.ny;
        float *col = a.vol + (long long)y * a.g.nx + x;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int z = z0 + r;
            if (z < a.g.nz) col[z * sxy] += acc[r];
        }
    }
}

template <int BX, int BY, int WX, int R, int FETCH, typename T>
static fdk_status launch_one(const BpArgs &a, cudaStream_t s)
{
    dim3 grid((a.g.nx + BX - 1) / BX, (a.g.ny + BY - 1) / BY, (a.g.nz + R - 1) / R);
    fdk_bp_kernel<BX, BY, WX, R, FETCH, T><<<grid, BX * BY, 0, s>>>(a);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("back-projection launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

template <int FETCH, typename T>
static fdk_status launch_zrun(const BpArgs &a, int zrun, cudaStream_t s)
{
    switch (zrun) {
    case 4: return launch_one<32, 8, 8, 4, FETCH, T>(a, s);
    case 16: return launch_one<32, 8, 8, 16, FETCH, T>(a, s);
    default: return launch_one<32, 8, 8, 8, FETCH, T>(a, s);
    }
}

fdk_status launch_backproject(const BpArgs &a, int fetch, int dtype, int zrun, cudaStream_t s)
{
    if (fetch == kTex) {
        switch (dtype) {
        case FDK_F32: return launch_zrun<kTex, float>(a, zrun, s);
        case FDK_F16: return launch_zrun<kTex, __half>(a, zrun, s);
        case FDK_BF16: return launch_zrun<kTex, __nv_bfloat16>(a, zrun, s);
        }
    } else {
        switch (dtype) {
        case FDK_F32: return launch_zrun<kLdg, float>(a, zrun, s);
        case FDK_F16: return launch_zrun<kLdg, __half>(a, zrun, s);
        case FDK_BF16: return launch_zrun<kLdg, __nv_bfloat16>(a, zrun, s);
        }
    }
    set_error("unsupported projection dtype %d", dtype);
    return FDK_ERR_INVALID_ARG;
}

}  // namespace fdk
