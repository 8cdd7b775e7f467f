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
// pixel box), then adds the non-zero cells to the projections with one
// global atomic per cell (one 16-byte vector atomic per 4 cells when rows are
// aligned).  The shared accumulation is fixed point with native 32-bit
// integer atomics (an FP32 add on shared memory is a compare-and-swap loop):
// contributions are scaled by s = (2^31 - 2^13) wmin^2 / sum|f|, with sum|f|
// over the tile's voxels and wmin the tile's smallest w for the view, so no
// cell can overflow whatever the geometry, and each contribution is
// rounded to 1/s, about 1e-6 of a typical contribution.  Footprints too
// large for the shared buffer fall back to direct FP32 global atomics.
//
// Tiles are 16 x 16 voxels in x, y with a z-run of 8 or 16 voxels per thread.
// The host picks the run per call: 16 where the volume stays far from every
// source and the footprints fit half the buffer, else 8.
#include "fdk_tile.cuh"

namespace fdk {

// Views per table chunk: as many as 3 CTAs per SM allow, 11 KB of tables
// beside the 64 KB footprint buffer, exactly the SM's 228 KB with the
// per-CTA reserve (91 views: three chunks per ray-orientation group at
// 512^3 x 496 instead of four or five, 0.5% less time than 64).
constexpr int kAdjBX = 16, kAdjBY = 16, kAdjChunk = 91;
constexpr int kAdjCap = 16384;  // cells of the shared footprint buffer (64 KB, dynamic)
// Tiles whose FP32 detector positions may be off by more than this many
// pixels (tiles close to the source) splat from FP64 positions instead.  The
// bound stays below 1.3e-5 px on the benchmark geometries (128^3..1024^3 on
// the 1248 x 960 detector), so they never take that path.
constexpr float kPreciseUV = 2.0e-5f;

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// One tap of a boundary or near-source voxel: pixels outside the image get
// nothing; pixels inside the tile's footprint box go to the shared buffer,
// any other (never expected) to the projections directly.
__device__ __forceinline__ void adj_tap_checked(int *acc_s, bool fixed, float scale, float *proj,
                                                const int4 &bb, bool fits, int W, int H, int ti,
                                                int tj, float val)
{
    if ((unsigned)ti >= (unsigned)W || (unsigned)tj >= (unsigned)H) return;
    const int li = ti - bb.x, lj = tj - bb.y;
    if (fits && (unsigned)li < (unsigned)bb.z && (unsigned)lj < (unsigned)bb.w) {
        if (fixed) atomicAdd(acc_s + lj * bb.z + li, __float2int_rn(val * scale));
        else atomicAdd(reinterpret_cast<float *>(acc_s) + lj * bb.z + li, val);
    } else {
        atomicAdd(proj + (long long)tj * W + ti, val);
    }
}

// Shared-memory integer reductions into the cell at a 32-bit shared address
// and the one after it (the offset in the instruction, not in a register).
__device__ __forceinline__ void red_shared_pair(uint32_t addr, int v0, int v1)
{
    asm volatile("red.shared.add.s32 [%0], %1;" :: "r"(addr), "r"(v0) : "memory");
    asm volatile("red.shared.add.s32 [%0+4], %1;" :: "r"(addr), "r"(v1) : "memory");
}

// The four taps of one voxel of a boundary tile: cells (i, j), (i + 1, j) at
// shared address q0 and the next, (i, j + 1), (i + 1, j + 1) at q1 and the
// next, each reduced only when it lies in the box of bz x bh cells (i, j
// box-relative).  The tests are predicates of the reductions, not branches.
__device__ __forceinline__ void red_shared_quad_in_box(uint32_t q0, uint32_t q1, int i, int j, unsigned bz,
                                                       unsigned bh, int v00, int v10, int v01, int v11)
{
    asm volatile("{\n\t.reg .pred b0, b1, p;\n\t"
                 "setp.lt.u32 b0, %2, %5;\n\t"
                 "setp.lt.u32 b1, %3, %5;\n\t"
                 "setp.lt.and.u32 p, %4, %6, b0;\n\t"
                 "@p red.shared.add.s32 [%0], %8;\n\t"
                 "setp.lt.and.u32 p, %7, %6, b0;\n\t"
                 "@p red.shared.add.s32 [%0+4], %9;\n\t"
                 "setp.lt.and.u32 p, %4, %6, b1;\n\t"
                 "@p red.shared.add.s32 [%1], %10;\n\t"
                 "setp.lt.and.u32 p, %7, %6, b1;\n\t"
                 "@p red.shared.add.s32 [%1+4], %11;\n\t}"
                 :: "r"(q0), "r"(q1), "r"(j), "r"(j + 1), "r"(i), "r"(bh), "r"(bz), "r"(i + 1),
                    "r"(v00), "r"(v10), "r"(v01), "r"(v11)
                 : "memory");
}

// The four weighted taps of a voxel: value g = f / w^2 and fractions (a, b).
struct Taps {
    float w00, w10, w01, w11;
};
__device__ __forceinline__ Taps tap_weights(float g, float a, float b)
{
    const float gh = g * b, gl = g - gh;
    Taps t;
    t.w10 = gl * a;
    t.w00 = gl - t.w10;
    t.w11 = gh * a;
    t.w01 = gh - t.w11;
    return t;
}

// Fixed-point splat of one view for an interior or boundary tile.  Interior:
// every tap lies in the image and, by the 1-pixel margin of the footprint box
// bb, inside bb; the clamp of the cell index only guards memory.  Each f32x2 pair holds one
// quantity of two z neighbours, as in the forward's hot loop.  The
// contribution f / w^2 is scaled to fixed point before it is split into the
// four tap weights, and the cell index (j - j0) * bw + (i - i0) is formed in
// FP32 (exact: below 2^14 plus the 2^23 index magic), whose bits then address
// the cell directly.
// CHECK (boundary tiles): taps outside the image are dropped.  The box is
// clipped to the image and holds every tap inside it, so each reduction is
// predicated on its pixel lying in the box, and its address is formed from
// the integer cell index.
template <int R, bool CHECK>
__device__ __forceinline__ void splat_fixed(const float (&f)[R], const ViewEntry &e, float2 buv, float bw,
                                            const int4 &bb, const int4 &sp, float scale, int *acc_v)
{
    const float2 BU = f2(buv.x), BV = f2(buv.y), BWW = f2(bw);
    const float2 GU = f2(e.b.z), GV = f2(e.b.w), GW = f2(e.w.w);
    const float2 M = f2(kFloorMagic), NM = f2(-kFloorMagic), NEG = f2(-1.0f);
    const float2 PITCH = f2((float)bb.z);
    const float2 OFF = f2(__int_as_float(sp.x));
    const float kmax = __int_as_float(sp.y);
    const float2 SC = f2(scale);
    const uint32_t cbase = (uint32_t)__cvta_generic_to_shared(acc_v);
    const uint32_t abase = cbase - (kIndexBits << 2);
    const uint32_t abase1 = abase + ((uint32_t)bb.z << 2);
    // (u', v', w) of the run's first two voxels, then stepped two voxels at a
    // time, exactly as the back-projection steps them (so the two operators
    // see the same detector positions)
    const float2 RF0 = f2((float)(-R / 2), (float)(1 - R / 2));
    float2 wl = __ffma2_rn(RF0, GW, BWW), uq = __ffma2_rn(RF0, GU, BU), vq = __ffma2_rn(RF0, GV, BV);
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
        const float2 flu = __fadd2_rn(tu, NM);
        const float2 flv = __fadd2_rn(tv, NM);
        const float2 au = __ffma2_rn(flu, NEG, u), bv = __ffma2_rn(flv, NEG, v);
        const float2 g = __fmul2_rn(__fmul2_rn(iw, iw), __fmul2_rn(f2(f[r], f[r + 1]), SC));
        const float2 gh = __fmul2_rn(g, bv), gl = __ffma2_rn(gh, NEG, g);
        const float2 w10 = __fmul2_rn(gl, au), w00 = __ffma2_rn(w10, NEG, gl);
        const float2 w11 = __fmul2_rn(gh, au), w01 = __ffma2_rn(w11, NEG, gh);
        if (!CHECK) {
            float2 k = __fadd2_rn(__ffma2_rn(flv, PITCH, flu), OFF);
            k = f2(fminf(fmaxf(k.x, kIndexMagic), kmax), fminf(fmaxf(k.y, kIndexMagic), kmax));
            const uint32_t o0 = (uint32_t)__float_as_int(k.x) << 2, o1 = (uint32_t)__float_as_int(k.y) << 2;
            red_shared_pair(abase + o0, __float2int_rn(w00.x), __float2int_rn(w10.x));
            red_shared_pair(abase1 + o0, __float2int_rn(w01.x), __float2int_rn(w11.x));
            red_shared_pair(abase + o1, __float2int_rn(w00.y), __float2int_rn(w10.y));
            red_shared_pair(abase1 + o1, __float2int_rn(w01.y), __float2int_rn(w11.y));
        } else {
            // box-relative pixel indices from the floor bits; the box is
            // clipped to the image and holds every tap inside it, so a tap
            // is kept exactly when it lies in the box (which also keeps
            // every access in the buffer)
            const int i0 = __float_as_int(tu.x) - kFloorBits + sp.z, j0 = __float_as_int(tv.x) - kFloorBits + sp.w;
            const int i1 = __float_as_int(tu.y) - kFloorBits + sp.z, j1 = __float_as_int(tv.y) - kFloorBits + sp.w;
            const unsigned bzu = (unsigned)bb.z, bwu = (unsigned)bb.w;
            // cell addresses in integers: a voxel one cell above or left of
            // the box still has taps inside it, at a negative base index
            const uint32_t q0 = cbase + (uint32_t)(j0 * bb.z + i0) * 4u;
            const uint32_t q1 = cbase + (uint32_t)(j1 * bb.z + i1) * 4u;
            const uint32_t rowb = (uint32_t)bb.z * 4u;
            red_shared_quad_in_box(q0, q0 + rowb, i0, j0, bzu, bwu, __float2int_rn(w00.x), __float2int_rn(w10.x),
                                   __float2int_rn(w01.x), __float2int_rn(w11.x));
            red_shared_quad_in_box(q1, q1 + rowb, i1, j1, bzu, bwu, __float2int_rn(w00.y), __float2int_rn(w10.y),
                                   __float2int_rn(w01.y), __float2int_rn(w11.y));
        }
    }
}

// VEC4: rows of the projections are 16-byte aligned (W % 4 == 0 and an
// aligned base), so footprint boxes are widened to 4-pixel groups and
// flushed with one vector atomic per group.
template <int BX, int BY, int R, int WX, bool VEC4>
__global__ void __launch_bounds__(BX * BY, 3)
fdk_adj_kernel(const __grid_constant__ BpArgs a, float *__restrict__ proj_out)
{
    constexpr int NT = BX * BY;
    __shared__ ViewEntry tab[kAdjChunk];
    __shared__ unsigned char cls[kAdjChunk];
    __shared__ unsigned short act[kAdjChunk];
    __shared__ int4 bbox[kAdjChunk];
    __shared__ float2 wrange[kAdjChunk];   // w range of the tile, then (scale, 1 / scale)
    __shared__ int4 vflags[kAdjChunk];     // (flags, row divisor, flush step, view index)
    __shared__ int4 vsplat[kAdjChunk];     // (cell offset, last base cell, column, row offsets)
    __shared__ int n_act;
    extern __shared__ __align__(16) int acc_s[];   // kAdjCap cells: fixed point, or FP32 bits
    __shared__ float red_s[NT / 32];

    const int tid = threadIdx.x;
    for (int p = tid; p < kAdjCap; p += NT) acc_s[p] = 0;

    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * R;
    const int lane = tid & 31, warp = tid >> 5;
    static_assert(32 % WX == 0 && BX % WX == 0 && BY % (32 / WX) == 0, "warp tiling");
    constexpr int WY = 32 / WX, WPX = BX / WX;
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
    // sum |f| over the tile: bounds every footprint cell's sum
    float sf = 0.0f;
#pragma unroll
    for (int r = 0; r < R; ++r) sf += fabsf(f[r]);
    for (int o = 16; o > 0; o >>= 1) sf += __shfl_xor_sync(0xffffffffu, sf, o);
    if (lane == 0) red_s[warp] = sf;
    __syncthreads();
    float ftile = 0.0f;
    for (int w = 0; w < NT / 32; ++w) ftile += red_s[w];
    if (!(ftile > 0.0f)) return;   // uniform: an all-zero tile adds nothing
    ftile *= 1.0009765625f;         // headroom for the FP32 rounding of the sum

    // The footprint buffer is used as two halves while boxes fit one: view q
    // accumulates in the half that view q-1 is not being flushed from, so
    // the flush of q-1 needs no barrier before the splat of q.  A box larger
    // than a half takes the whole buffer after a barrier.  [prev_lo, prev_hi)
    // is the cell range whose flush may still be in progress (uniform).
    int prev_lo = 0, prev_hi = 0;
    for (int v0 = 0; v0 < a.n_views; v0 += kAdjChunk) {
        const int nv = min(kAdjChunk, a.n_views - v0);
        build_view_table<BX, BY, R>(a, v0, nv, x0, y0, z0, tab, cls, act, &n_act, bbox, wrange);
        // what every thread needs of a view but depends on the view alone,
        // once per view: the box (widened to 4-cell groups for the vector
        // flush), the fixed-point scale, whether FP64 positions are needed,
        // and the flush's (row, group) stepping without a division
        for (int lv = tid; lv < nv; lv += NT) {
            const int c = cls[lv];
            if (c == kSkip) continue;
            const ViewEntry e = tab[lv];
            int4 bb = bbox[lv];
            if (VEC4 && bb.z > 0) {
                const int i0 = bb.x & ~3, i1 = ((bb.x + bb.z + 3) & ~3);
                bb.x = i0;
                bb.z = i1 - i0;
            }
            const int npx = bb.z * bb.w;
            const float2 wr = wrange[lv];
            const bool fits = npx > 0 && npx <= kAdjCap;
            // fixed point when w varies little over the tile, else FP32 cells
            const bool fixed = fits && wr.x > 0.0f && wr.y <= 1.5f * wr.x;
            // FP32 rounding of the table's detector positions, about
            // 2^-24 (|c| + extent |g|) / w pixels, bounded over the tile;
            // the splat's tap weights move by that much
            const float tu = fabsf(e.a.x) + (BX / 2) * fabsf(e.a.z) + (BY / 2) * fabsf(e.b.x) +
                             (R / 2) * fabsf(e.b.z);
            const float tv = fabsf(e.a.y) + (BX / 2) * fabsf(e.a.w) + (BY / 2) * fabsf(e.b.y) +
                             (R / 2) * fabsf(e.b.w);
            const bool precise = c == kGeneral || !(wr.x > 0.0f) ||
                                 fmaxf(tu, tv) * 5.9604645e-8f > kPreciseUV * wr.x;
            const float sc = fixed ? 2147475456.0f * (wr.x * wr.x) / ftile : 0.0f;
            const int gw = VEC4 ? bb.z >> 2 : bb.z;   // flush items per row
            const int rowdiv = gw > 0 ? (16777216 + gw - 1) / gw : 0;
            const int drow = gw > 0 ? NT / gw : 0;
            const int U = (int)e.o.x, V = (int)e.o.y;
            bbox[lv] = bb;
            wrange[lv] = make_float2(sc, fixed ? ftile / (2147475456.0f * (wr.x * wr.x)) : 0.0f);
            vflags[lv] = make_int4((fits ? 1 : 0) | (fixed ? 2 : 0) | (precise ? 4 : 0), rowdiv,
                                   drow | ((NT - drow * gw) << 16), a.vidx[v0 + lv]);
            vsplat[lv] = make_int4(__float_as_int((float)((V - bb.y) * bb.z + (U - bb.x)) + kIndexMagic),
                                   __float_as_int((float)(npx - bb.z - 2) + kIndexMagic), U - bb.x, V - bb.y);
        }
        __syncthreads();
        prev_lo = prev_hi = 0;
        const int n = n_act;
        for (int q = 0; q < n; ++q) {
            const int ev = act[q];
            const int lv = ev & 1023, c = ev >> 10;
            const ViewEntry e = tab[lv];
            const int4 bb = bbox[lv];
            const int4 vf = vflags[lv];
            const int npx = bb.z * bb.w;
            const bool fits = (vf.x & 1) != 0, fixed = (vf.x & 2) != 0, precise = (vf.x & 4) != 0;
            const float2 sc = wrange[lv];
            const float scale = sc.x, inv_scale = sc.y;
            int *acc_v = acc_s;
            if (fits) {
                const int lo = (npx <= kAdjCap / 2 && prev_lo == 0 && prev_hi > 0) ? kAdjCap / 2 : 0;
                if (lo < prev_hi && prev_lo < lo + npx) __syncthreads();   // that flush must be done
                acc_v = acc_s + lo;
                prev_lo = lo;
                prev_hi = lo + npx;
            }
            float *proj = proj_out + (long long)vf.w * a.plane;
            const float2 buv = __ffma2_rn(f2(dyf), f2(e.b.x, e.b.y), __ffma2_rn(f2(dxf), f2(e.a.z, e.a.w), f2(e.a.x, e.a.y)));
            const float bw = fmaf(dyf, e.w.z, fmaf(dxf, e.w.y, e.w.x));
            const float2 gz = f2(e.b.z, e.b.w);
            if (precise) {
                // close to the source (or across its plane): each voxel's
                // (u', v', w) from the matrix in FP64 and u = u'/w, v = v'/w
                // by division, as the definition reads
                const int v = v0 + lv;
                const float *Pm = a.mats_dev ? a.mats_dev + 12 * v : a.mats + 12 * v;
                const double X = (double)a.g.org[0] + (double)x * (double)a.g.vs[0];
                const double Y = (double)a.g.org[1] + (double)y * (double)a.g.vs[1];
                const double bu = fma((double)Pm[0], X, fma((double)Pm[1], Y, (double)Pm[3]));
                const double bvv = fma((double)Pm[4], X, fma((double)Pm[5], Y, (double)Pm[7]));
                const double bww = fma((double)Pm[8], X, fma((double)Pm[9], Y, (double)Pm[11]));
                const double pu = Pm[2], pv = Pm[6], pw = Pm[10];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (f[r] == 0.0f) continue;
                    const double Z = (double)a.g.org[2] + (double)(z0 + r) * (double)a.g.vs[2];
                    const double wd = fma(pw, Z, bww);
                    if (!(wd > 0.0)) continue;
                    const double ud = fmin(fmax(fma(pu, Z, bu) / wd, -2.0), (double)W + 1.0);
                    const double vd = fmin(fmax(fma(pv, Z, bvv) / wd, -2.0), (double)H + 1.0);
                    const double fu = floor(ud), fv = floor(vd);
                    const Taps k = tap_weights((float)((double)f[r] / (wd * wd)), (float)(ud - fu),
                                               (float)(vd - fv));
                    const int i = (int)fu, j = (int)fv;
                    adj_tap_checked(acc_v, fixed, scale, proj, bb, fits, W, H, i, j, k.w00);
                    adj_tap_checked(acc_v, fixed, scale, proj, bb, fits, W, H, i + 1, j, k.w10);
                    adj_tap_checked(acc_v, fixed, scale, proj, bb, fits, W, H, i, j + 1, k.w01);
                    adj_tap_checked(acc_v, fixed, scale, proj, bb, fits, W, H, i + 1, j + 1, k.w11);
                }
            } else if (fixed && c == kInterior) {
                splat_fixed<R, false>(f, e, buv, bw, bb, vsplat[lv], scale, acc_v);
            } else if (fixed && c == kBoundary) {
                splat_fixed<R, true>(f, e, buv, bw, bb, vsplat[lv], scale, acc_v);
            } else {
                const int U = (int)e.o.x, V = (int)e.o.y;
                const float lou = -2.0f - e.o.x, lov = -2.0f - e.o.y;
                const float hiu = (float)(W + 1) - e.o.x, hiv = (float)(H + 1) - e.o.y;
                // stepped as in the back-projection: a chain for the even
                // voxels of the run and one for the odd, two voxels per step
                float w0 = fmaf((float)(-R / 2), e.w.w, bw), w1 = fmaf((float)(1 - R / 2), e.w.w, bw);
                float2 q0 = __ffma2_rn(f2((float)(-R / 2)), gz, buv), q1 = __ffma2_rn(f2((float)(1 - R / 2)), gz, buv);
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
                    uv = f2(fminf(fmaxf(uv.x, lou), hiu), fminf(fmaxf(uv.y, lov), hiv));
                    const float2 t = __fadd2_rd(uv, f2(kFloorMagic));
                    const float au = uv.x - (t.x - kFloorMagic), bv = uv.y - (t.y - kFloorMagic);
                    const int i = __float_as_int(t.x) - kFloorBits + U;
                    const int j = __float_as_int(t.y) - kFloorBits + V;
                    float g = f[r] * iw * iw;
                    if (c == kGeneral && !(wl > 0.0f)) g = 0.0f;
                    if (g == 0.0f) continue;
                    const Taps k = tap_weights(g, au, bv);
                    adj_tap_checked(acc_v, fixed, scale, proj, bb, fits, W, H, i, j, k.w00);
                    adj_tap_checked(acc_v, fixed, scale, proj, bb, fits, W, H, i + 1, j, k.w10);
                    adj_tap_checked(acc_v, fixed, scale, proj, bb, fits, W, H, i, j + 1, k.w01);
                    adj_tap_checked(acc_v, fixed, scale, proj, bb, fits, W, H, i + 1, j + 1, k.w11);
                }
            }
            if (fits) {
                __syncthreads();
                if (VEC4) {
                    const int gw = bb.z >> 2;
                    int4 *acc4 = reinterpret_cast<int4 *>(acc_v);
                    // (row, group) of p, stepped along with p
                    int row = (int)(((unsigned)tid * (unsigned)vf.y) >> 24), grp = tid - row * gw;
                    const int drow = vf.z & 0xFFFF, dgrp = vf.z >> 16;
                    for (int p = tid; p < (npx >> 2); p += NT) {
                        const int4 s4 = acc4[p];
                        const int col = grp << 2, rw = row;
                        grp += dgrp;
                        row += drow;
                        if (grp >= gw) { grp -= gw; ++row; }
                        if ((s4.x | s4.y | s4.z | s4.w) != 0) {
                            const int row = rw;
                            const float4 v = fixed
                                ? make_float4((float)s4.x * inv_scale, (float)s4.y * inv_scale,
                                              (float)s4.z * inv_scale, (float)s4.w * inv_scale)
                                : make_float4(__int_as_float(s4.x), __int_as_float(s4.y),
                                              __int_as_float(s4.z), __int_as_float(s4.w));
                            atomicAdd(reinterpret_cast<float4 *>(proj + (long long)(bb.y + row) * W + bb.x + col), v);
                            acc4[p] = make_int4(0, 0, 0, 0);
                        }
                    }
                } else {
                    for (int p = tid; p < npx; p += NT) {
                        const int s1 = acc_v[p];
                        if (s1 != 0) {
                            const float v = fixed ? (float)s1 * inv_scale : __int_as_float(s1);
                            atomicAdd(proj + (long long)(bb.y + p / bb.z) * W + bb.x + p % bb.z, v);
                            acc_v[p] = 0;
                        }
                    }
                }
            }
        }
        __syncthreads();   // the next chunk overwrites the table
    }
}

template <int R, int WX>
static fdk_status launch_adjoint_wx(const BpArgs &a, float *proj_out, cudaStream_t s)
{
    dim3 grid((a.g.nx + kAdjBX - 1) / kAdjBX, (a.g.ny + kAdjBY - 1) / kAdjBY, (a.g.nz + R - 1) / R);
    const bool vec4 = (a.g.W % 4) == 0 && ((uintptr_t)proj_out % 16) == 0;
    const size_t smem = (size_t)kAdjCap * sizeof(int);
    auto k = vec4 ? fdk_adj_kernel<kAdjBX, kAdjBY, R, WX, true> : fdk_adj_kernel<kAdjBX, kAdjBY, R, WX, false>;
    // opt in to more than 48 KB of dynamic shared memory (idempotent)
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) {
        cudaGetLastError();
        set_error("adjoint: shared-memory opt-in failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    k<<<grid, kAdjBX * kAdjBY, smem, s>>>(a, proj_out);
    err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("adjoint launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

template <int R>
static fdk_status launch_adjoint_r(const BpArgs &a, float *proj_out, cudaStream_t s)
{
    switch (a.warp_x) {
    case 2: return launch_adjoint_wx<R, 2>(a, proj_out, s);
    case 4: return launch_adjoint_wx<R, 4>(a, proj_out, s);
    case 16: return launch_adjoint_wx<R, 16>(a, proj_out, s);
    default: return launch_adjoint_wx<R, 8>(a, proj_out, s);
    }
}

// Warp patches of a.warp_x voxels along x by 32 / a.warp_x along y; tiles of
// 16 x 16 x z_run voxels, z_run 8 or 16.
fdk_status launch_adjoint(const BpArgs &a, float *proj_out, int z_run, cudaStream_t s)
{
    return z_run == 16 ? launch_adjoint_r<16>(a, proj_out, s) : launch_adjoint_r<8>(a, proj_out, s);
}

}  // namespace fdk
