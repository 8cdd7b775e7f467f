// Staged fetch path of the back-projection (Listing 1, Sec. IV): for every
// (tile, view) whose footprint fits, the pixel box holding all of the tile's
// taps is copied from global memory into shared memory by the tensor-memory
// accelerator (cp.async.bulk.tensor, completion on an mbarrier) and the four
// taps of each voxel are read from there.  The copy reads zeros outside the
// image, so boundary tiles need no bounds checks (the effect of the paper's
// zero-padded projection copy, Sec. VI, without a copy in global memory).
//
// Why: on the global-load path the L1 data pipe is the binding unit, and
// about a third of its cycles are sector fills of the footprints from L2.
// A bulk copy moves the same footprint in full 128-byte lines.
//
// Pipeline per CTA: kStages shared-memory stages.  Every thread waits on the
// stage's mbarrier and computes the view; after a CTA barrier (the stage is
// then free) thread 0 issues the copy of the staged view kStages further on
// into it, so the next view's copy is in flight while the CTA computes.  The
// copy goes in as few TMA boxes as the map heights allow (8 to 64 rows on a
// plain launch), because the issuing warp lags the next barrier by the
// issue's length.
// Each thread owns a z-run of 16 voxels, so the per-view barrier is shared
// by 16 updates per thread (8 per thread measured 10% slower, 24 slower
// still).  (A barrier-free variant, in which the last warp done with a stage
// refills it, measured 12% slower: its warps spin on the mbarriers instead.)
// Every wait is bounded; a thread whose wait gives up raises a shared flag
// that all read after the barrier: *err is set, thread 0 drains the copies
// still in flight (again bounded) and the CTA stops without writing its
// tile.  The taps are read with 32-bit shared addresses.
#pragma once

#include "fdk_bp_kernel.cuh"

namespace fdk {

constexpr int kStages = 2;
// Views per table chunk on this path.  Each chunk ends the CTA's copy
// pipeline (the next chunk's boxes are known only after its table is built),
// so chunks are as long as 3 CTAs per SM allow: 96 views took 1.3% less time
// than 64 at 512^3 x 496 (three chunks per ray-orientation group instead of
// four or five); 9 KB of tables per CTA beside the 64 KB of stages.
constexpr int kStageChunk = 96;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Bounded wait for the phase with the given parity of the mbarrier at bar:
// at most `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit)
{
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Copy the box of table entry lv (view v0 + lv of the pass) into stage st.
// Called by one thread.  tmaps holds NH maps per box width, of boxes 8, 16,
// .., 8 * 2^(NH-1) rows high: the box's rows8 8-row blocks go in as few copies
// as those heights allow (one copy per set bit of rows8, tallest first).
// ESZ: bytes per pixel (4 for FP32 images, 2 for FP16 / BF16).
template <int NH, class A, int ESZ = 4>
__device__ __forceinline__ void stage_issue(const A &a, const CUtensorMap *tmaps, int v0, int lv,
                                            const int4 *sbox, float *stages, uint32_t full0, unsigned st)
{
    // order the CTA's reads of this stage (before the caller's barrier)
    // before the asynchronous copy that overwrites it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const int4 b = sbox[lv];                       // (x0, j0, m, rows8)
    const int BW = box_width(b.z);
    const uint32_t bar = full0 + 8u * st;
    const uint32_t bytes = (uint32_t)(b.w * kBoxRows * BW) * (uint32_t)ESZ;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"(bytes) : "memory");
    const uint32_t dst = smem_addr(stages + (size_t)st * kStageFloats);
    const int img = a.vidx[v0 + lv];
    int r = 0, left = b.w;
#pragma unroll
    for (int h = NH - 1; h >= 0; --h) {
        const CUtensorMap *map = tmaps + b.z * NH + h;
        while (left >= (1 << h)) {
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4}], [%5];"
                :: "r"(dst + (uint32_t)(r * kBoxRows * BW) * (uint32_t)ESZ), "l"(map), "r"(b.x),
                   "r"(b.y + r * kBoxRows), "r"(img), "r"(bar)
                : "memory");
            r += 1 << h;
            left -= 1 << h;
        }
    }
}

// Shared-memory loads of the words at a 32-bit shared address and the one
// after it (the offset in the instruction, not in a register).  Volatile, so
// they stay after the (volatile) mbarrier wait that makes the stage's data
// visible.
__device__ __forceinline__ float lds(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ float lds_next(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1+4];" : "=f"(v) : "r"(addr));
    return v;
}

// The same for each pixel type: the pixel at a 32-bit shared address and the
// one after it, widened to FP32 exactly.
template <typename T> struct StagedPixel;
template <> struct StagedPixel<float> {
    static constexpr int kShift = 2;   // log2 of the pixel's bytes
    static __device__ __forceinline__ float at(uint32_t addr) { return lds(addr); }
    static __device__ __forceinline__ float next(uint32_t addr) { return lds_next(addr); }
};
template <> struct StagedPixel<__nv_bfloat16> {
    static constexpr int kShift = 1;
    static __device__ __forceinline__ float at(uint32_t addr)
    {
        unsigned v;
        asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(addr));
        return __uint_as_float(v << 16);
    }
    static __device__ __forceinline__ float next(uint32_t addr)
    {
        unsigned v;
        asm volatile("ld.shared.u16 %0, [%1+2];" : "=r"(v) : "r"(addr));
        return __uint_as_float(v << 16);
    }
};
template <> struct StagedPixel<__half> {
    static constexpr int kShift = 1;
    static __device__ __forceinline__ float at(uint32_t addr)
    {
        unsigned short v;
        asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
        return __half2float(__ushort_as_half(v));
    }
    static __device__ __forceinline__ float next(uint32_t addr)
    {
        unsigned short v;
        asm volatile("ld.shared.u16 %0, [%1+2];" : "=h"(v) : "r"(addr));
        return __half2float(__ushort_as_half(v));
    }
};

// Staged view: the taps come from the stage's box, BW = e.o.w pixels wide,
// whose cell (U, V) sits at index e.o.z - 2^23.  No bounds checks: the box
// holds every tap of the tile, with zeros where it extends past the image.
// Each f32x2 pair holds one quantity for two z neighbours, so every packed
// operation finds its operands in place.
template <int R, typename T = float>
__device__ __forceinline__ void view_staged(float (&acc)[R], const ViewEntry &e, float dxf, float dyf,
                                            const float *stage)
{
    using P = StagedPixel<T>;
    const float2 BU = f2(fmaf(dyf, e.b.x, fmaf(dxf, e.a.z, e.a.x)));
    const float2 BV = f2(fmaf(dyf, e.b.y, fmaf(dxf, e.a.w, e.a.y)));
    const float2 BW = f2(fmaf(dyf, e.w.z, fmaf(dxf, e.w.y, e.w.x)));
    const float2 GU = f2(e.b.z), GV = f2(e.b.w), GW = f2(e.w.w);
    const float2 M = f2(kFloorMagic), NM = f2(-kFloorMagic), NEG = f2(-1.0f);
    const float2 PITCH = f2(e.o.w), OZ = f2(e.o.z);
    // 32-bit shared addresses of the tap rows j and j + 1, with the index
    // magic folded into the bases
    const uint32_t sbase = smem_addr(stage) - (kIndexBits << P::kShift);
    const uint32_t sbase1 = sbase + ((uint32_t)(int)e.o.w << P::kShift);
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
        const float2 flu = __fadd2_rn(__fadd2_rd(u, M), NM);
        const float2 flv = __fadd2_rn(__fadd2_rd(v, M), NM);
        const float2 au = __ffma2_rn(flu, NEG, u), bv = __ffma2_rn(flv, NEG, v);
        const float2 k = __fadd2_rn(__ffma2_rn(flv, PITCH, flu), OZ);
        const uint32_t o0 = (uint32_t)__float_as_int(k.x) << P::kShift, o1 = (uint32_t)__float_as_int(k.y) << P::kShift;
        const uint32_t a0 = sbase + o0, a1 = sbase + o1, b0 = sbase1 + o0, b1 = sbase1 + o1;
        const float2 p00 = f2(P::at(a0), P::at(a1)), p10 = f2(P::next(a0), P::next(a1));
        const float2 p01 = f2(P::at(b0), P::at(b1)), p11 = f2(P::next(b0), P::next(b1));
        const float2 lo = __ffma2_rn(au, __ffma2_rn(p00, NEG, p10), p00);
        const float2 hi = __ffma2_rn(au, __ffma2_rn(p01, NEG, p11), p01);
        const float2 val = __ffma2_rn(bv, __ffma2_rn(lo, NEG, hi), lo);
        const float2 s2 = __ffma2_rn(val, __fmul2_rn(iw, iw), f2(acc[r], acc[r + 1]));
        acc[r] = s2.x;
        acc[r + 1] = s2.y;
    }
}

// Shared state of the staged pipeline.  The mbarriers and the issued-copy
// counts live for the whole CTA (a persistent CTA keeps them across tiles);
// the table arrays are rebuilt per chunk of views.
struct StageTables {
    ViewEntry tab[kStageChunk];
    int4 sbox[kStageChunk];
    unsigned char cls[kStageChunk];
    unsigned short act[kStageChunk];
    unsigned short stg[kStageChunk];       // table entries of the staged views, in order
    int n_act, n_stg;
};
struct StageBarriers {
    unsigned long long full[kStages];
    unsigned nissue[kStages];              // copies issued into each stage so far
    unsigned consumed;                     // staged views consumed so far (uniform)
    unsigned failed;                       // set by a thread whose bounded wait gave up
};

// Called once per CTA by all threads before the first stage_tile.
__device__ __forceinline__ void stage_init(StageBarriers &sb)
{
    if (threadIdx.x == 0) {
        const uint32_t full0 = smem_addr(sb.full);
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(full0 + 8u * s) : "memory");
            sb.nissue[s] = 0;
        }
        sb.consumed = 0;
        sb.failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
}

// Back-project every view of `a` into the BX x BY x R tile at (x0, y0, z0)
// (volume +=), staging the views whose box fits through the CTA's stages
// and reading the others with global loads.  All threads of the CTA call
// this.  Returns false, with the tile unwritten, when a bounded wait gave up
// (the CTA must then stop using the stages); *err is set and the copies in
// flight are drained.
template <int BX, int BY, int WX, int R, bool FIDX, int NH, class A, typename T = float>
__device__ __forceinline__ bool stage_tile(const A &a, const CUtensorMap *tmaps, unsigned *err, long long wait_limit,
                                           int x0, int y0, int z0, StageTables &t, StageBarriers &sb,
                                           float *stages)
{
    static_assert(32 % WX == 0 && BX % WX == 0 && BY % (32 / WX) == 0, "warp tiling");
    static_assert(R % 2 == 0, "z-run must be even (voxel pairs)");
    constexpr int KCHUNK = kStageChunk;
    constexpr int WY = 32 / WX;
    constexpr int WPX = BX / WX;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int lx = (warp % WPX) * WX + (lane % WX);
    const int ly = (warp / WPX) * WY + (lane / WX);
    const float dxf = (float)(lx - BX / 2), dyf = (float)(ly - BY / 2);
    const int W = a.g.W, H = a.g.H;
    const T *proj = static_cast<const T *>(a.proj);
    const uint32_t full0 = smem_addr(sb.full);

    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0f;

    unsigned base = sb.consumed;   // staged views of earlier chunks and tiles (uniform)
    for (int v0 = 0; v0 < a.n_views; v0 += KCHUNK) {
        const int nv = min(KCHUNK, a.n_views - v0);
        build_view_table<BX, BY, R, A, true, (int)sizeof(T)>(a, v0, nv, x0, y0, z0, t.tab, t.cls, t.act, &t.n_act,
                                             nullptr, nullptr, t.sbox);
        const int n = t.n_act;
        if (warp == 0) {
            // compact the staged views, in view order
            int count = 0;
            for (int q0 = 0; q0 < n; q0 += 32) {
                const int q = q0 + lane;
                const bool is_st = q < n && (t.act[q] >> 10) == kStaged;
                const unsigned m = __ballot_sync(0xffffffffu, is_st);
                if (is_st) t.stg[count + __popc(m & ((1u << lane) - 1u))] = t.act[q] & 1023;
                count += __popc(m);
            }
            if (lane == 0) t.n_stg = count;
            __syncwarp();
            if (lane == 0) {
                // the first copies of the chunk
                for (int k = 0; k < kStages && k < count; ++k) {
                    const unsigned st = (base + k) % kStages;
                    stage_issue<NH, A, (int)sizeof(T)>(a, tmaps, v0, t.stg[k], t.sbox, stages, full0, st);
                    ++sb.nissue[st];
                }
            }
        }
        __syncthreads();
        const unsigned ns = (unsigned)t.n_stg;
        unsigned kst = 0;     // staged views of this chunk consumed so far (uniform)
        for (int q = 0; q < n; ++q) {
            const int ev = t.act[q];
            const int lv = ev & 1023, c = ev >> 10;
            if (c == kStaged) {
                const unsigned slot = base + kst;
                const unsigned st = slot % kStages;
                if (!mbar_wait(full0 + 8u * st, (slot / kStages) & 1u, wait_limit)) sb.failed = 1u;
                const ViewEntry e = t.tab[lv];
                view_staged<R, T>(acc, e, dxf, dyf, stages + (size_t)st * kStageFloats);
                ++kst;
                __syncthreads();
                if (sb.failed) {
                    if (tid == 0) {
                        atomicOr(err, 1u);
                        // drain with the full limit: no copy may still be
                        // writing this CTA's shared memory when it exits
                        for (int s = 0; s < kStages; ++s)
                            if (sb.nissue[s] > 0) mbar_wait(full0 + 8u * s, (sb.nissue[s] - 1) & 1u, kWaitLimit);
                    }
                    return false;
                }
                if (tid == 0) {
                    const unsigned nk = kst - 1 + kStages;
                    if (nk < ns) {
                        stage_issue<NH, A, (int)sizeof(T)>(a, tmaps, v0, t.stg[nk], t.sbox, stages, full0, st);
                        ++sb.nissue[st];
                    }
                }
                continue;
            }
            const ViewEntry e = t.tab[lv];
            const T *img = proj + (long long)a.vidx[v0 + lv] * a.plane;
            if (c == kInterior) view_interior_ldg<R, T, FIDX>(acc, e, dxf, dyf, img, W);
            else if (c == kBoundary) view_checked_ldg<R, T, false>(acc, e, dxf, dyf, img, W, H);
            else view_checked_ldg<R, T, true>(acc, e, dxf, dyf, img, W, H);
        }
        base += ns;
        __syncthreads();   // the next chunk overwrites the table
    }
    if (tid == 0) sb.consumed = base;

    const int x = x0 + lx, y = y0 + ly;
    if (x < a.g.nx && y < a.g.ny) {
        const long long sxy = (long long)a.g.nx * a.g.ny;
        add_to_column<R>(a.vol + (long long)y * a.g.nx + x, sxy, z0, a.g.nz, acc);
    }
    return true;
}

}  // namespace fdk
