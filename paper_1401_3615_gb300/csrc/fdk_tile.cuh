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
// that a direct FP32 evaluation of P (X, 1) gives for 256 mm volumes.
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

// Fill tab[0..n_views) and the compacted list act[0..*n_act) of views whose
// class is not kSkip; act[q] = view | class << 10.  All threads of the CTA
// call this; it ends with __syncthreads().
template <int BX, int BY, int R>
__device__ void build_view_table(const BpArgs &a, int x0, int y0, int z0, ViewEntry *tab,
                                 unsigned char *cls, unsigned short *act, int *n_act)
{
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;
    const Geom &g = a.g;
    const double sx = g.vs[0], sy = g.vs[1], sz = g.vs[2];
    const double Xc = (double)g.org[0] + (double)(x0 + BX / 2) * sx;
    const double Yc = (double)g.org[1] + (double)(y0 + BY / 2) * sy;
    const double Zc = (double)g.org[2] + (double)(z0 + R / 2) * sz;
    // corner offsets of the full tile box (every computed voxel, including
    // those past the volume edge that are computed but not stored)
    const float dx0 = (float)(-(BX / 2)), dx1 = (float)(BX - 1 - BX / 2);
    const float dy0 = (float)(-(BY / 2)), dy1 = (float)(BY - 1 - BY / 2);
    const float dz0 = (float)(-(R / 2)), dz1 = (float)(R - 1 - R / 2);
    const float eps = 1.0f / 64.0f;

    for (int v = tid; v < a.n_views; v += nthreads) {
        double P[12];
        if (a.mats_dev) {
#pragma unroll
            for (int q = 0; q < 12; ++q) P[q] = (double)__ldg(a.mats_dev + 12 * v + q);
        } else {
#pragma unroll
            for (int q = 0; q < 12; ++q) P[q] = (double)a.mats[12 * v + q];
        }
        const double up = P[0] * Xc + P[1] * Yc + P[2] * Zc + P[3];
        const double vp = P[4] * Xc + P[5] * Yc + P[6] * Zc + P[7];
        const double wp = P[8] * Xc + P[9] * Yc + P[10] * Zc + P[11];
        int U = 0, V = 0;
        if (wp > 0.0) {
            float uf = (float)up / (float)wp, vf = (float)vp / (float)wp;
            uf = fminf(fmaxf(uf, -1048576.0f), 1048576.0f);
            vf = fminf(fmaxf(vf, -1048576.0f), 1048576.0f);
            U = __float2int_rn(uf);
            V = __float2int_rn(vf);
        }
        const double dU = (double)U, dV = (double)V;
        ViewEntry e;
        e.ru = make_float4((float)(up - dU * wp), (float)((P[0] - dU * P[8]) * sx),
                           (float)((P[1] - dU * P[9]) * sy), (float)((P[2] - dU * P[10]) * sz));
        e.rv = make_float4((float)(vp - dV * wp), (float)((P[4] - dV * P[8]) * sx),
                           (float)((P[5] - dV * P[9]) * sy), (float)((P[6] - dV * P[10]) * sz));
        e.rw = make_float4((float)wp, (float)(P[8] * sx), (float)(P[9] * sy), (float)(P[10] * sz));
        e.off = make_float4((float)U + 1.0f, (float)V + 1.0f, __int_as_float(U), __int_as_float(V));

        // classify from the 8 corners
        float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
        int npos = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float dx = (c & 1) ? dx1 : dx0;
            const float dy = (c & 2) ? dy1 : dy0;
            const float dz = (c & 4) ? dz1 : dz0;
            const float wl = fmaf(dz, e.rw.w, fmaf(dy, e.rw.z, fmaf(dx, e.rw.y, e.rw.x)));
            const float ul = fmaf(dz, e.ru.w, fmaf(dy, e.ru.z, fmaf(dx, e.ru.y, e.ru.x)));
            const float vl = fmaf(dz, e.rv.w, fmaf(dy, e.rv.z, fmaf(dx, e.rv.y, e.rv.x)));
            if (wl > 0.0f) {
                ++npos;
                const float uu = ul / wl + (float)U, vv = vl / wl + (float)V;
                umin = fminf(umin, uu); umax = fmaxf(umax, uu);
                vmin = fminf(vmin, vv); vmax = fmaxf(vmax, vv);
            }
        }
        int c;
        if (npos == 0) {
            c = kSkip;                      // w <= 0 on the whole tile (w is linear)
        } else if (npos < 8) {
            c = kGeneral;                   // tile crosses the source plane: per-voxel w test
        } else if (umax < -1.0f - eps || umin > (float)g.W + eps ||
                   vmax < -1.0f - eps || vmin > (float)g.H + eps) {
            c = kSkip;                      // every tap of every voxel is off the detector
        } else if (umin >= eps && umax <= (float)(g.W - 1) - eps &&
                   vmin >= eps && vmax <= (float)(g.H - 1) - eps) {
            c = kInterior;                  // all four taps inside for every voxel
        } else {
            c = kBoundary;
        }
        tab[v] = e;
        cls[v] = (unsigned char)c;
    }
    __syncthreads();
    if (tid < 32) {
        int count = 0;
        for (int base = 0; base < a.n_views; base += 32) {
            const int v = base + tid;
            const int c = (v < a.n_views) ? (int)cls[v] : 0;
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
