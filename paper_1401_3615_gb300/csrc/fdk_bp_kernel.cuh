// Voxel-driven cone-beam back-projection kernels (Listing 1, Sec. IV),
// templated over the CTA tile, fetch path and storage type; instantiated in
// fdk_bp_*.cu.
//
// Work decomposition: a CTA owns a BX x BY x R box of voxels; each thread
// owns one (x, y) column of R consecutive z voxels and keeps their sums in
// registers across every view of the pass, so the volume is read once and
// written once per pass (up to 512 views) instead of once per view.  Views
// are visited in index order, so each voxel sums its views in the same
// order as the definition.
//
// Per view and voxel the hot loop does, in FP32:
//   (u'_l, v'_l), w = FMAs from per-(tile, view) coefficients
//   r = 1/w (MUFU), (u, v) = (u'_l, v'_l) r, cell-relative detector position
//   floor and fractions (a, b) by a round-down magic add
//   four taps: read-only loads (LDG path: bounds-free on interior tiles) or
//   a 2x2 texture gather with zero border (TEX path)
//   three lerps, acc += val r^2
// The u/v pair of one voxel and the w, weight and accumulator of two z
// neighbours are processed as packed f32x2 operations (FFMA2/FADD2/FMUL2),
// which halves the issue slots of the FP32 work.
#pragma once

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
// agrees with the FP32 floor.
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

enum Fetch : int { kLdg = 1, kTex = 2, kQuad = 3 };

template <typename T> struct QuadType { using type = uint2; };
template <> struct QuadType<float> { using type = float4; };

// One quad cell (p00, p10, p01, p11) as FP32.
template <typename T> struct QuadLoad;
template <> struct QuadLoad<float> {
    static __device__ __forceinline__ float4 load(const void *base, unsigned long long off)
    {
        return __ldg(reinterpret_cast<const float4 *>(reinterpret_cast<const char *>(base) + off * 16));
    }
};
template <> struct QuadLoad<__half> {
    static __device__ __forceinline__ float4 load(const void *base, unsigned long long off)
    {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(base) + off * 8));
        const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
        const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
};
template <> struct QuadLoad<__nv_bfloat16> {
    static __device__ __forceinline__ float4 load(const void *base, unsigned long long off)
    {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(base) + off * 8));
        return make_float4(__uint_as_float(q.x << 16), __uint_as_float(q.x & 0xffff0000u),
                           __uint_as_float(q.y << 16), __uint_as_float(q.y & 0xffff0000u));
    }
};

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// Bilinear value from the four taps and the fractions (a, b):
// lo = p00 + a (p10 - p00), hi = p01 + a (p11 - p01), val = lo + b (hi - lo).
__device__ __forceinline__ float bilerp(float p00, float p10, float p01, float p11, float2 ab)
{
    const float2 d = __ffma2_rn(f2(p00, p01), f2(-1.0f), f2(p10, p11));
    const float2 lh = __ffma2_rn(f2(ab.x), d, f2(p00, p01));
    return fmaf(ab.y, lh.y - lh.x, lh.x);
}

// Per-thread values of one view: (u'_l, v'_l) and w at z offset 0.
struct ViewBase {
    float2 uv;
    float w;
};

__device__ __forceinline__ ViewBase view_base(const ViewEntry &e, float dxf, float dyf)
{
    ViewBase b;
    b.uv = __ffma2_rn(f2(dyf), f2(e.b.x, e.b.y), __ffma2_rn(f2(dxf), f2(e.a.z, e.a.w), f2(e.a.x, e.a.y)));
    b.w = fmaf(dyf, e.w.z, fmaf(dxf, e.w.y, e.w.x));
    return b;
}

// Interior tiles: all four taps of every voxel lie inside the image.
// FIDX: the flat tap index is formed in FP32 (exact while W*H < 2^23) and its
// bit pattern used as the address offset; otherwise integer arithmetic.
// Each f32x2 pair holds one quantity for two z neighbours, so every packed
// operation finds its operands in place.
template <int R, typename T, bool FIDX>
__device__ __forceinline__ void view_interior_ldg(float (&acc)[R], const ViewEntry &e, float dxf,
                                                  float dyf, const T *img, int W)
{
    const float2 BU = f2(fmaf(dyf, e.b.x, fmaf(dxf, e.a.z, e.a.x)));
    const float2 BV = f2(fmaf(dyf, e.b.y, fmaf(dxf, e.a.w, e.a.y)));
    const float2 BW = f2(fmaf(dyf, e.w.z, fmaf(dxf, e.w.y, e.w.x)));
    const float2 GU = f2(e.b.z), GV = f2(e.b.w), GW = f2(e.w.w);
    const float2 M = f2(kFloorMagic), NM = f2(-kFloorMagic), NEG = f2(-1.0f);
    const float2 PITCH = f2((float)W), OZ = f2(e.o.z);
    const int U = (int)e.o.x, V = (int)e.o.y;
    // row pointers biased so the index bits address the tap directly
    const unsigned long long row0 =
        FIDX ? (unsigned long long)img - (unsigned long long)kIndexBits * sizeof(T)
             : (unsigned long long)img;
    const unsigned long long row1 = row0 + (unsigned long long)W * sizeof(T);
    // (u', v', w) of the run's first two voxels, then stepped two voxels at a
    // time (the steps 2 g are exact)
    const float2 RF0 = f2((float)(-R / 2), (float)(1 - R / 2));
    float2 wl = __ffma2_rn(RF0, GW, BW), uq = __ffma2_rn(RF0, GU, BU), vq = __ffma2_rn(RF0, GV, BV);
    const float2 G2W = __fadd2_rn(GW, GW), G2U = __fadd2_rn(GU, GU), G2V = __fadd2_rn(GV, GV);
#pragma unroll
    for (int r = 0; r < R; r += 2) {
        if (r > 0) {
            wl = __fadd2_rn(wl, G2W);
            uq = __fadd2_rn(uq, G2U);
            vq = __fadd2_rn(vq, G2V);
        }
        const float2 iw = f2(rcp_approx(wl.x), rcp_approx(wl.y));
        const float2 u = __fmul2_rn(uq, iw);
        const float2 v = __fmul2_rn(vq, iw);
        const float2 tu = __fadd2_rd(u, M), tv = __fadd2_rd(v, M);
        const float2 flu = __fadd2_rn(tu, NM), flv = __fadd2_rn(tv, NM);
        const float2 au = __ffma2_rn(flu, NEG, u), bv = __ffma2_rn(flv, NEG, v);
        unsigned long long o0, o1;
        if (FIDX) {
            const float2 k = __fadd2_rn(__ffma2_rn(flv, PITCH, flu), OZ);
            o0 = (unsigned long long)__float_as_uint(k.x) * sizeof(T);
            o1 = (unsigned long long)__float_as_uint(k.y) * sizeof(T);
        } else {
            const int i0 = __float_as_int(tu.x) - kFloorBits + U, j0 = __float_as_int(tv.x) - kFloorBits + V;
            const int i1 = __float_as_int(tu.y) - kFloorBits + U, j1 = __float_as_int(tv.y) - kFloorBits + V;
            o0 = (unsigned long long)(j0 * W + i0) * sizeof(T);
            o1 = (unsigned long long)(j1 * W + i1) * sizeof(T);
        }
        const T *q00 = reinterpret_cast<const T *>(row0 + o0);
        const T *q01 = reinterpret_cast<const T *>(row1 + o0);
        const T *q10 = reinterpret_cast<const T *>(row0 + o1);
        const T *q11 = reinterpret_cast<const T *>(row1 + o1);
        const float2 p00 = f2(Elem<T>::load(q00), Elem<T>::load(q10));
        const float2 p10 = f2(Elem<T>::load(q00 + 1), Elem<T>::load(q10 + 1));
        const float2 p01 = f2(Elem<T>::load(q01), Elem<T>::load(q11));
        const float2 p11 = f2(Elem<T>::load(q01 + 1), Elem<T>::load(q11 + 1));
        const float2 lo = __ffma2_rn(au, __ffma2_rn(p00, NEG, p10), p00);
        const float2 hi = __ffma2_rn(au, __ffma2_rn(p01, NEG, p11), p01);
        const float2 val = __ffma2_rn(bv, __ffma2_rn(lo, NEG, hi), lo);
        const float2 s2 = __ffma2_rn(val, __fmul2_rn(iw, iw), f2(acc[r], acc[r + 1]));
        acc[r] = s2.x;
        acc[r + 1] = s2.y;
    }
}

// Boundary (and, with GENERAL, source-plane-crossing) tiles on the LDG path:
// per-tap bounds checks, loads only for taps inside the image.
template <int R, typename T, bool GENERAL>
__device__ __forceinline__ void view_checked_ldg(float (&acc)[R], const ViewEntry &e, float dxf,
                                                 float dyf, const T *img, int W, int H)
{
    const ViewBase vb = view_base(e, dxf, dyf);
    const float2 gz = f2(e.b.z, e.b.w);
    const int U = (int)e.o.x, V = (int)e.o.y;
    // cell-relative clamp range keeping every int exact; taps there read 0
    const float2 lo = f2(-2.0f - e.o.x, -2.0f - e.o.y);
    const float2 hi = f2((float)(W + 1) - e.o.x, (float)(H + 1) - e.o.y);
    // (u', v', w) stepped along the run as in the packed paths: one chain for
    // the even voxels and one for the odd, two voxels per step
    float w0 = fmaf((float)(-R / 2), e.w.w, vb.w), w1 = fmaf((float)(1 - R / 2), e.w.w, vb.w);
    float2 q0 = __ffma2_rn(f2((float)(-R / 2)), gz, vb.uv), q1 = __ffma2_rn(f2((float)(1 - R / 2)), gz, vb.uv);
    const float g2w = e.w.w + e.w.w;
    const float2 g2 = __fadd2_rn(gz, gz);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r >= 2) {
            if (r & 1) { w1 += g2w; q1 = __fadd2_rn(q1, g2); }
            else { w0 += g2w; q0 = __fadd2_rn(q0, g2); }
        }
        const float wl = (r & 1) ? w1 : w0;
        const float iw = rcp_approx(wl);
        float2 uv = __fmul2_rn((r & 1) ? q1 : q0, f2(iw));
        uv = f2(fminf(fmaxf(uv.x, lo.x), hi.x), fminf(fmaxf(uv.y, lo.y), hi.y));
        const float2 t = __fadd2_rd(uv, f2(kFloorMagic));
        const float2 fl = __fadd2_rn(t, f2(-kFloorMagic));
        const float2 ab = __ffma2_rn(fl, f2(-1.0f), uv);
        const int i = __float_as_int(t.x) - kFloorBits + U;
        const int j = __float_as_int(t.y) - kFloorBits + V;
        const bool c0 = (unsigned)i < (unsigned)W, c1 = (unsigned)(i + 1) < (unsigned)W;
        const bool r0 = (unsigned)j < (unsigned)H, r1 = (unsigned)(j + 1) < (unsigned)H;
        const T *q = img + (j * W + i);
        float p00 = 0.0f, p10 = 0.0f, p01 = 0.0f, p11 = 0.0f;
        if (c0 && r0) p00 = Elem<T>::load(q);
        if (c1 && r0) p10 = Elem<T>::load(q + 1);
        if (c0 && r1) p01 = Elem<T>::load(q + W);
        if (c1 && r1) p11 = Elem<T>::load(q + W + 1);
        float val = bilerp(p00, p10, p01, p11, ab);
        float iw2 = iw * iw;
        if (GENERAL) {
            const bool front = wl > 0.0f;
            val = front ? val : 0.0f;
            iw2 = front ? iw2 : 0.0f;
        }
        acc[r] = fmaf(val, iw2, acc[r]);
    }
}

// Quad path: one load per voxel from the zero-bordered quad image.  Interior
// tiles need no clamp; boundary tiles clamp the detector position into the
// bordered range [-2, W] x [-2, H], whose outer cells are all zero, so the
// clamp never changes a result.
template <int R, typename T, bool CLAMP>
__device__ __forceinline__ void view_quad(float (&acc)[R], const ViewEntry &e, float dxf, float dyf,
                                          const void *qimg, int W, int H, int QP)
{
    const ViewBase vb = view_base(e, dxf, dyf);
    const float2 gz = f2(e.b.z, e.b.w);
    const float2 M = f2(kFloorMagic);
    const float QPf = (float)QP;
    const float2 lo = f2(-2.0f - e.o.x, -2.0f - e.o.y);
    const float2 hi = f2((float)W - e.o.x, (float)H - e.o.y);
    // bias so that the index bits address the cell directly
    const unsigned long long bias = (unsigned long long)kIndexBits;
#pragma unroll
    for (int r = 0; r < R; r += 2) {
        const float rf0 = (float)(r - R / 2), rf1 = rf0 + 1.0f;
        const float2 wl = __ffma2_rn(f2(rf0, rf1), f2(e.w.w), f2(vb.w));
        const float iw0 = rcp_approx(wl.x), iw1 = rcp_approx(wl.y);
        float2 uv0 = __fmul2_rn(__ffma2_rn(f2(rf0), gz, vb.uv), f2(iw0));
        float2 uv1 = __fmul2_rn(__ffma2_rn(f2(rf1), gz, vb.uv), f2(iw1));
        if (CLAMP) {
            uv0 = f2(fminf(fmaxf(uv0.x, lo.x), hi.x), fminf(fmaxf(uv0.y, lo.y), hi.y));
            uv1 = f2(fminf(fmaxf(uv1.x, lo.x), hi.x), fminf(fmaxf(uv1.y, lo.y), hi.y));
        }
        const float2 fl0 = __fadd2_rn(__fadd2_rd(uv0, M), f2(-kFloorMagic));
        const float2 fl1 = __fadd2_rn(__fadd2_rd(uv1, M), f2(-kFloorMagic));
        const float2 ab0 = __ffma2_rn(fl0, f2(-1.0f), uv0), ab1 = __ffma2_rn(fl1, f2(-1.0f), uv1);
        const float2 s = __ffma2_rn(f2(fl0.y, fl1.y), f2(QPf), f2(fl0.x, fl1.x));
        const float2 k = __fadd2_rn(s, f2(e.o.w));
        const float4 q0 = QuadLoad<T>::load(qimg, (unsigned long long)__float_as_uint(k.x) - bias);
        const float4 q1 = QuadLoad<T>::load(qimg, (unsigned long long)__float_as_uint(k.y) - bias);
        const float v0 = bilerp(q0.x, q0.y, q0.z, q0.w, ab0);
        const float v1 = bilerp(q1.x, q1.y, q1.z, q1.w, ab1);
        const float2 w2 = __fmul2_rn(f2(iw0, iw1), f2(iw0, iw1));
        const float2 s2 = __ffma2_rn(f2(v0, v1), w2, f2(acc[r], acc[r + 1]));
        acc[r] = s2.x;
        acc[r + 1] = s2.y;
    }
}

// Texture path: the gather's zero border covers every off-image tap, so one
// code path serves interior and boundary tiles.
template <int R, typename T, bool GENERAL>
__device__ __forceinline__ void view_tex(float (&acc)[R], const ViewEntry &e, float dxf, float dyf,
                                         cudaTextureObject_t tex, int W, int H)
{
    const ViewBase vb = view_base(e, dxf, dyf);
    const float2 gz = f2(e.b.z, e.b.w);
    const float2 cell = f2(e.o.x + 1.0f, e.o.y + 1.0f);
    const float2 lo = f2(-4.0f - e.o.x, -4.0f - e.o.y);
    const float2 hi = f2((float)(W + 4) - e.o.x, (float)(H + 4) - e.o.y);
#pragma unroll
    for (int r = 0; r < R; r += 2) {
        const float rf0 = (float)(r - R / 2), rf1 = rf0 + 1.0f;
        const float2 wl = __ffma2_rn(f2(rf0, rf1), f2(e.w.w), f2(vb.w));
        const float iw0 = rcp_approx(wl.x), iw1 = rcp_approx(wl.y);
        float2 uv0 = __fmul2_rn(__ffma2_rn(f2(rf0), gz, vb.uv), f2(iw0));
        float2 uv1 = __fmul2_rn(__ffma2_rn(f2(rf1), gz, vb.uv), f2(iw1));
        if (GENERAL) {
            // keep texel coordinates finite behind the source plane
            uv0 = f2(fminf(fmaxf(uv0.x, lo.x), hi.x), fminf(fmaxf(uv0.y, lo.y), hi.y));
            uv1 = f2(fminf(fmaxf(uv1.x, lo.x), hi.x), fminf(fmaxf(uv1.y, lo.y), hi.y));
        }
        const float2 fl0 = __fadd2_rn(__fadd2_rd(uv0, f2(kFloorMagic)), f2(-kFloorMagic));
        const float2 fl1 = __fadd2_rn(__fadd2_rd(uv1, f2(kFloorMagic)), f2(-kFloorMagic));
        const float2 ab0 = __ffma2_rn(fl0, f2(-1.0f), uv0), ab1 = __ffma2_rn(fl1, f2(-1.0f), uv1);
        const float2 x0 = __fadd2_rn(fl0, cell), x1 = __fadd2_rn(fl1, cell);
        const float4 g0 = Gather<T>::fetch(tex, x0.x, x0.y);
        const float4 g1 = Gather<T>::fetch(tex, x1.x, x1.y);
        float v0 = bilerp(g0.x, g0.y, g0.z, g0.w, ab0);
        float v1 = bilerp(g1.x, g1.y, g1.z, g1.w, ab1);
        float2 w2 = __fmul2_rn(f2(iw0, iw1), f2(iw0, iw1));
        if (GENERAL) {
            const bool f0 = wl.x > 0.0f, f1 = wl.y > 0.0f;
            v0 = f0 ? v0 : 0.0f;
            v1 = f1 ? v1 : 0.0f;
            w2 = f2(f0 ? w2.x : 0.0f, f1 ? w2.y : 0.0f);
        }
        const float2 s2 = __ffma2_rn(f2(v0, v1), w2, f2(acc[r], acc[r + 1]));
        acc[r] = s2.x;
        acc[r + 1] = s2.y;
    }
}

// Back-project every view of `a` into the BX x BY x R box at (x0, y0, z0):
// per-thread register sums over all views, then one read-modify-write of the
// box.  A is the launch's argument block (the kernel parameters of a plain
// launch, or a scan descriptor of a batch); the shared tables are the
// caller's.  Warps cover WX x (32/WX) voxel patches in (x, y).
template <int BX, int BY, int WX, int R, int KCHUNK, int FETCH, typename T, bool FIDX, class A>
__device__ __forceinline__ void bp_tile(const A &a, int x0, int y0, int z0, ViewEntry *tab,
                                        unsigned char *cls, unsigned short *act, int *n_act_s)
{
    static_assert(32 % WX == 0 && BX % WX == 0 && BY % (32 / WX) == 0, "warp tiling");
    static_assert(R % 2 == 0, "z-run must be even (voxel pairs)");
    constexpr int WY = 32 / WX;
    constexpr int WPX = BX / WX;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lx = (warp % WPX) * WX + (lane % WX);
    const int ly = (warp / WPX) * WY + (lane / WX);
    const float dxf = (float)(lx - BX / 2), dyf = (float)(ly - BY / 2);
    const int W = a.g.W, H = a.g.H;
    const T *proj = static_cast<const T *>(a.proj);

    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0f;

    for (int v0 = 0; v0 < a.n_views; v0 += KCHUNK) {
        const int nv = min(KCHUNK, a.n_views - v0);
        build_view_table<BX, BY, R>(a, v0, nv, x0, y0, z0, tab, cls, act, n_act_s);
        const int n = *n_act_s;
        for (int q = 0; q < n; ++q) {
            const int ev = act[q];
            const int lv = ev & 1023, c = ev >> 10;
            const int v = v0 + lv;
            const ViewEntry e = tab[lv];
            if constexpr (FETCH == kTex) {
                const cudaTextureObject_t tex = (cudaTextureObject_t)a.tex[v];
                if (c != kGeneral) view_tex<R, T, false>(acc, e, dxf, dyf, tex, W, H);
                else view_tex<R, T, true>(acc, e, dxf, dyf, tex, W, H);
                continue;
            }
            if constexpr (FETCH == kQuad) {
                if (c != kGeneral) {
                    const void *qimg = static_cast<const char *>(a.quads) +
                                       (long long)a.vidx[v] * a.qplane * (long long)sizeof(typename QuadType<T>::type);
                    if (c == kInterior) view_quad<R, T, false>(acc, e, dxf, dyf, qimg, W, H, a.qpitch);
                    else view_quad<R, T, true>(acc, e, dxf, dyf, qimg, W, H, a.qpitch);
                    continue;
                }
            }
            const T *img = proj + (long long)a.vidx[v] * a.plane;
            if (c == kInterior) view_interior_ldg<R, T, FIDX>(acc, e, dxf, dyf, img, W);
            else if (c == kBoundary) view_checked_ldg<R, T, false>(acc, e, dxf, dyf, img, W, H);
            else view_checked_ldg<R, T, true>(acc, e, dxf, dyf, img, W, H);
        }
        __syncthreads();   // the next chunk overwrites the table
    }

    const int x = x0 + lx, y = y0 + ly;
    if (x < a.g.nx && y < a.g.ny) {
        const long long sxy = (long long)a.g.nx * a.g.ny;
        add_to_column<R>(a.vol + (long long)y * a.g.nx + x, sxy, z0, a.g.nz, acc);
    }
}

// One CTA per BX x BY x R tile of the volume (plain launch).
template <int BX, int BY, int WX, int R, int MINB, int KCHUNK, int FETCH, typename T, bool FIDX>
__global__ void __launch_bounds__(BX * BY, MINB)
fdk_bp_kernel(const __grid_constant__ BpArgs a)
{
    __shared__ ViewEntry tab[KCHUNK];
    __shared__ unsigned char cls[KCHUNK];
    __shared__ unsigned short act[KCHUNK];
    __shared__ int n_act;
    bp_tile<BX, BY, WX, R, KCHUNK, FETCH, T, FIDX>(a, blockIdx.x * BX, blockIdx.y * BY, blockIdx.z * R,
                                                    tab, cls, act, &n_act);
}

// CTA tile variants (BX x BY voxels in x, y; R voxels per thread along z;
// minimum resident CTAs per SM for the register budget).  Warps cover 8 x 4
// or 4 x 8 voxel patches (BpArgs::warp_x): views whose rays run mostly along
// x project a 4 x 8 patch onto fewer L1 banks, views along y an 8 x 4 patch.
// Index 0 is the default (the fastest at 512^3 x 496 views, 1248 x 960) and
// shares its kernel with index 1.
struct TileCfg { int bx, by, r, minb; };
constexpr int kNumTiles = 8;
constexpr TileCfg kTiles[kNumTiles] = {
    {16, 16, 8, 4}, {16, 16, 8, 4}, {32, 16, 4, 2}, {32, 16, 8, 2},
    {32, 8, 4, 4}, {16, 16, 4, 4}, {32, 8, 16, 3}, {16, 16, 16, 3},
};

template <int BX, int BY, int R, int MINB, int FETCH, typename T, bool FIDX>
fdk_status launch_one(const BpArgs &a, cudaStream_t s)
{
    constexpr int KCHUNK = 128;
    dim3 grid((a.g.nx + BX - 1) / BX, (a.g.ny + BY - 1) / BY, (a.g.nz + R - 1) / R);
    if (a.warp_x == 4)
        fdk_bp_kernel<BX, BY, 4, R, MINB, KCHUNK, FETCH, T, FIDX><<<grid, BX * BY, 0, s>>>(a);
    else
        fdk_bp_kernel<BX, BY, 8, R, MINB, KCHUNK, FETCH, T, FIDX><<<grid, BX * BY, 0, s>>>(a);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("back-projection launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

template <int TILE, int FETCH, typename T, bool FIDX>
fdk_status launch_tile(const BpArgs &a, cudaStream_t s)
{
    constexpr TileCfg c = kTiles[TILE];
    return launch_one<c.bx, c.by, c.r, c.minb, FETCH, T, FIDX>(a, s);
}

// Dispatch over the tile variants for one fetch path and storage type.
template <int FETCH, typename T, bool FIDX>
fdk_status launch_tiles(const BpArgs &a, int tile, cudaStream_t s)
{
    switch (tile) {
    case 2: return launch_tile<2, FETCH, T, FIDX>(a, s);
    case 3: return launch_tile<3, FETCH, T, FIDX>(a, s);
    case 4: return launch_tile<4, FETCH, T, FIDX>(a, s);
    case 5: return launch_tile<5, FETCH, T, FIDX>(a, s);
    case 6: return launch_tile<6, FETCH, T, FIDX>(a, s);
    case 7: return launch_tile<7, FETCH, T, FIDX>(a, s);
    default: return launch_tile<0, FETCH, T, FIDX>(a, s);
    }
}

}  // namespace fdk
