// Per-CTA view table: the geometry of one volume tile against every view of
// a pass, built once in shared memory before the hot loop.
//
// For the tile centre voxel c and view k the forward projection
// (u', v', w) = P_k (X_c, 1) (Listing 1, the "forward projection" lines) is
// evaluated in FP64, an integer detector cell (U, V) near u'/w, v'/w is
// chosen, and the rows are shifted to that cell:
//     u'_local(d) = (P_0 - U P_2) . (X_c + d*s, 1)
// so that u = U + u'_local / w.  In the hot loop every voxel is a small
// integer offset d from the centre and the FP32 values stay small, which
// keeps the detector coordinate accurate to ~1e-5 px instead of the ~1e-4 px
// that a direct FP32 evaluation of P (X, 1) gives for 256 mm volumes.  Only
// the reference values and the two cancelling differences u' - U w and
// v' - V w need FP64; the per-step coefficients are FP32 FMAs.
//
// The same prologue classifies the tile for the view from its eight corner
// voxels (u and v of a box are extreme at its corners when w > 0): a tile
// whose footprint misses (-1, W) x (-1, H) is skipped -- the paper's clipping
// mask, Sec. VI -- and a tile whose taps all lie inside the image needs no
// bounds checks (the effect of the paper's zero padding, Sec. VI).
#pragma once

#include "fdk_internal.cuh"

namespace fdk {

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// floor() by a round-down add: for |x| < 2^22, x + 1.5*2^23 rounded toward
// -inf is floor(x) + 1.5*2^23 exactly; its bit pattern is 0x4B400000 + floor(x).
constexpr float kFloorMagic = 12582912.0f;
constexpr int kFloorBits = 0x4B400000;
// Flat tap index by float: for 0 <= n < 2^23, n + 2^23 is exact and its bit
// pattern is 0x4B000000 + n.
constexpr float kIndexMagic = 8388608.0f;
constexpr unsigned kIndexBits = 0x4B000000u;

// Add a thread's sums to its z-run of voxels (volume +=) with fire-and-forget
// global reductions instead of a load, an add and a store: the load's latency
// otherwise ends every tile (about 5 us per tile and launch at 512^3).  Each
// voxel has one writer per launch, so the result is the plain
// read-add-write's; the reduction flushes subnormal sums to zero.
template <int R>
__device__ __forceinline__ void add_to_column(float *col, long long sxy, int z0, int nz, const float (&acc)[R])
{
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (z0 + r < nz) atomicAdd(col + (long long)(z0 + r) * sxy, acc[r]);
}

// Fill tab[0..nv) for views v0..v0+nv of the pass and the compacted list
// act[0..*n_act) of those whose class is not kSkip; act[q] = (v - v0) |
// class << 10.  All threads of the CTA call this; it ends with
// __syncthreads().  Tables are built in chunks of views so that the shared
// memory they take stays small and the rest of the SM's L1 holds image data.
// With STAGE, interior and boundary views whose tap box fits a shared-memory
// stage become kStaged: sbox[lv] = (x0, j0, m, rows8) describes the TMA copy
// (columns x0.. of box width m, 8-row boxes from row j0; x0 is a multiple of
// 16 / ESZ, ESZ the pixel's bytes, so the first column is 16-byte aligned)
// and e.o.z, e.o.w address taps in that box.  The box spans the corner footprint widened by one pixel on each
// side against FP32 rounding; it may extend past the image, where the copy
// reads zeros -- exactly the zero-outside rule of the interpolation.
// With bbox != nullptr it also stores, per view, the pixel box that holds
// every in-image tap of the tile, (i0, j0, width, height), widened by 1/64
// pixel against FP32 rounding (the per-voxel positions agree with the corners'
// to about 1e-5 pixel) and clipped to the image, and in wrange the
// smallest and largest w of the tile's corners (of the whole tile, since w
// is linear in the voxel position).
template <int BX, int BY, int R, class A, bool STAGE = false, int ESZ = 4>
__device__ void build_view_table(const A &a, int v0, int nv, int x0, int y0, int z0,
                                 ViewEntry *tab, unsigned char *cls, unsigned short *act,
                                 int *n_act, int4 *bbox = nullptr, float2 *wrange = nullptr,
                                 int4 *sbox = nullptr)
{
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;
    const Geom &g = a.g;
    const float sx = g.vs[0], sy = g.vs[1], sz = g.vs[2];
    const double Xc = (double)g.org[0] + (double)(x0 + BX / 2) * (double)sx;
    const double Yc = (double)g.org[1] + (double)(y0 + BY / 2) * (double)sy;
    const double Zc = (double)g.org[2] + (double)(z0 + R / 2) * (double)sz;
    // corner offsets of the full tile box (every computed voxel, including
    // those past the volume edge that are computed but not stored)
    const float dx0 = (float)(-(BX / 2)), dx1 = (float)(BX - 1 - BX / 2);
    const float dy0 = (float)(-(BY / 2)), dy1 = (float)(BY - 1 - BY / 2);
    const float dz0 = (float)(-(R / 2)), dz1 = (float)(R - 1 - R / 2);
    const float eps = 1.0f / 64.0f;
    const float Wf = (float)g.W;

    for (int lv = tid; lv < nv; lv += nthreads) {
        const int v = v0 + lv;
        float P[12];
        if (a.mats_dev) {
#pragma unroll
            for (int q = 0; q < 12; ++q) P[q] = __ldg(a.mats_dev + 12 * v + q);
        } else {
#pragma unroll
            for (int q = 0; q < 12; ++q) P[q] = a.mats[12 * v + q];
        }
        const double up = fma((double)P[0], Xc, fma((double)P[1], Yc, fma((double)P[2], Zc, (double)P[3])));
        const double vp = fma((double)P[4], Xc, fma((double)P[5], Yc, fma((double)P[6], Zc, (double)P[7])));
        const double wp = fma((double)P[8], Xc, fma((double)P[9], Yc, fma((double)P[10], Zc, (double)P[11])));
        float Uf = 0.0f, Vf = 0.0f;
        if (wp > 0.0) {
            const float iw = 1.0f / (float)wp;
            Uf = rintf(fminf(fmaxf((float)up * iw, -1048576.0f), 1048576.0f));
            Vf = rintf(fminf(fmaxf((float)vp * iw, -1048576.0f), 1048576.0f));
        }
        ViewEntry e;
        e.a = make_float4((float)fma(-(double)Uf, wp, up), (float)fma(-(double)Vf, wp, vp),
                          fmaf(-Uf, P[8], P[0]) * sx, fmaf(-Vf, P[8], P[4]) * sx);
        e.b = make_float4(fmaf(-Uf, P[9], P[1]) * sy, fmaf(-Vf, P[9], P[5]) * sy,
                          fmaf(-Uf, P[10], P[2]) * sz, fmaf(-Vf, P[10], P[6]) * sz);
        e.w = make_float4((float)wp, P[8] * sx, P[9] * sy, P[10] * sz);
        // flat index offsets of the cell (U, V) in the image and in the quad
        // image, plus the index magic (exact while the images are below 2^23
        // cells and the cell lies in or near them)
        e.o = make_float4(Uf, Vf, fmaf(Vf, Wf, Uf) + kIndexMagic,
                          fmaf(Vf + 2.0f, Wf + 3.0f, Uf + 2.0f) + kIndexMagic);

        // classify from the 8 corners
        float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
        float wlo = 3.0e38f, whi = -3.0e38f;
        int npos = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float dx = (c & 1) ? dx1 : dx0;
            const float dy = (c & 2) ? dy1 : dy0;
            const float dz = (c & 4) ? dz1 : dz0;
            const float wl = fmaf(dz, e.w.w, fmaf(dy, e.w.z, fmaf(dx, e.w.y, e.w.x)));
            const float ul = fmaf(dz, e.b.z, fmaf(dy, e.b.x, fmaf(dx, e.a.z, e.a.x)));
            const float vl = fmaf(dz, e.b.w, fmaf(dy, e.b.y, fmaf(dx, e.a.w, e.a.y)));
            wlo = fminf(wlo, wl);
            whi = fmaxf(whi, wl);
            if (wl > 0.0f) {
                ++npos;
                const float r = rcp_approx(wl);
                const float uu = fmaf(ul, r, Uf), vv = fmaf(vl, r, Vf);
                umin = fminf(umin, uu); umax = fmaxf(umax, uu);
                vmin = fminf(vmin, vv); vmax = fmaxf(vmax, vv);
            }
        }
        int c;
        if (npos == 0) {
            c = kSkip;                      // w <= 0 on the whole tile (w is linear)
        } else if (npos < 8) {
            c = kGeneral;                   // tile crosses the source plane: per-voxel w test
        } else if (umax < -1.0f - eps || umin > Wf + eps ||
                   vmax < -1.0f - eps || vmin > (float)g.H + eps) {
            c = kSkip;                      // every tap of every voxel is off the detector
        } else if (umin >= eps && umax <= Wf - 1.0f - eps &&
                   vmin >= eps && vmax <= (float)(g.H - 1) - eps) {
            c = kInterior;                  // all four taps inside for every voxel
        } else {
            c = kBoundary;
        }
        // boundary tiles whose reference cell lies far off the image (only
        // near the source plane) take the fully checked path, so the quad
        // index offset in e.o.w stays an exact FP32 integer
        if (c == kBoundary && (Uf < -64.0f || Uf > Wf + 64.0f || Vf < -64.0f || Vf > (float)g.H + 64.0f))
            c = kGeneral;
        if (STAGE && (c == kInterior || c == kBoundary)) {
            const float lim = 1048576.0f;
            const int i0 = (int)floorf(fmaxf(umin, -lim)) - 1, i1 = (int)floorf(fminf(umax, lim)) + 2;
            const int j0 = (int)floorf(fmaxf(vmin, -lim)) - 1, j1 = (int)floorf(fminf(vmax, lim)) + 2;
            const int bx0 = i0 & ~(16 / ESZ - 1);
            const int wpx = i1 - bx0 + 1;
            const int m = wpx <= 32 ? 0 : (wpx - 32 + 15) / 16;
            const int rows8 = (j1 - j0 + kBoxRows) / kBoxRows;
            if (m < kNumBoxW && rows8 * kBoxRows * box_width(m) <= kStageFloats * 4 / ESZ) {
                const int BW = box_width(m);
                e.o.z = (float)(((int)Vf - j0) * BW + ((int)Uf - bx0)) + kIndexMagic;
                e.o.w = (float)BW;
                sbox[lv] = make_int4(bx0, j0, m, rows8);
                c = kStaged;
            }
        }
        tab[lv] = e;
        cls[lv] = (unsigned char)c;
        if (bbox) {
            int4 bb = make_int4(0, 0, 0, 0);
            if (c == kInterior || c == kBoundary) {
                const float Hf = (float)g.H;
                const int i0 = max(0, (int)floorf(fmaxf(umin - eps, -4.0f)));
                const int i1 = min(g.W - 1, (int)floorf(fminf(umax + eps, Wf + 4.0f)) + 1);
                const int j0 = max(0, (int)floorf(fmaxf(vmin - eps, -4.0f)));
                const int j1 = min(g.H - 1, (int)floorf(fminf(vmax + eps, Hf + 4.0f)) + 1);
                if (i1 >= i0 && j1 >= j0) bb = make_int4(i0, j0, i1 - i0 + 1, j1 - j0 + 1);
            }
            bbox[lv] = bb;
            wrange[lv] = make_float2(wlo, whi);
        }
    }
    __syncthreads();
    if (tid < 32) {
        int count = 0;
        for (int base = 0; base < nv; base += 32) {
            const int v = base + tid;
            const int c = (v < nv) ? (int)cls[v] : 0;
            const unsigned m = __ballot_sync(0xffffffffu, c != kSkip);
            if (c != kSkip) {
                const int pos = count + __popc(m & ((1u << tid) - 1u));
                act[pos] = (unsigned short)(v | (c << 10));
            }
            count += __popc(m);
        }
        if (tid == 0) *n_act = count;
    }
    __syncthreads();
}

}  // namespace fdk
