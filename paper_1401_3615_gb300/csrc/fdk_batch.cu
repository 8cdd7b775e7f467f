// Batched back-projection: many scans of uneven size in one persistent
// launch.  A device work list holds (scan, tile) items; CTAs pull items from
// an atomic counter until the list is exhausted (no CTA ever waits on
// another).  Each item back-projects one tile of one scan: first the views
// whose rays run mostly along x with 4 x 8 warp patches, then the views
// along y with 8 x 4 patches -- the same per-voxel view order as the plain
// entry point, so a batch equals sequential plain calls bit for bit.
//
// Scans marked staged (tmap_slot >= 0: FP32 rows of a multiple of 16 bytes,
// footprints that fit the stages) take the staged pipeline of fdk_stage.cuh
// on 16 x 16 x 16 tiles, like fdk_backproject's default path for them; the
// others take the global-load path on the plan's tile variant.  A CTA keeps
// its stages' mbarriers across items.
#include "fdk_stage.cuh"

namespace fdk {

// The two per-item paths as real calls, so that each gets its own register
// allocation instead of one allocation for the whole persistent kernel (which
// spilled in the hot loops).
template <int WX, bool FIDX>
__device__ __noinline__ bool batch_stage_tile(const ScanDesc &d, const CUtensorMap *maps, unsigned *err,
                                              long long wait_limit, int x0, int y0, int z0, StageTables &t,
                                              StageBarriers &sb, float *stages)
{
    return stage_tile<kStageTileXY, kStageTileXY, WX, kStageTileZ, FIDX, 1>(d, maps, err, wait_limit, x0, y0, z0,
                                                                         t, sb, stages);
}

template <int BX, int BY, int WX, int R, int KCHUNK, bool FIDX>
__device__ __noinline__ void batch_ldg_tile(const ScanDesc &d, int x0, int y0, int z0, ViewEntry *tab,
                                            unsigned char *cls, unsigned short *act, int *n_act)
{
    bp_tile<BX, BY, WX, R, KCHUNK, kLdg, float, FIDX>(d, x0, y0, z0, tab, cls, act, n_act);
}

template <int BX, int BY, int R, int MINB, bool FIDX, bool STAGED>
__global__ void __launch_bounds__(BX * BY, MINB)
fdk_bp_batched_kernel(const __grid_constant__ BatchLaunch b)
{
    static_assert(!STAGED || (BX == kStageTileXY && BY == kStageTileXY), "staged scans need 256-thread CTAs");
    constexpr int KCHUNK = 128;
    struct LdgTables {
        ViewEntry tab[KCHUNK];
        unsigned char cls[KCHUNK];
        unsigned short act[KCHUNK];
        int n_act;
    };
    union Tables {
        LdgTables ldg;
        StageTables st;
    };
    __shared__ Tables u;
    __shared__ __align__(8) StageBarriers sb;
    __shared__ ScanDesc sd[2];
    __shared__ int item_s;
    extern __shared__ __align__(1024) float stages[];

    if constexpr (STAGED) stage_init(sb);
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(b.counter, 1);
        __syncthreads();
        const int item = item_s;
        if (item >= b.total) break;   // uniform across the CTA
        // scan of this item: tile_start[s] <= item < tile_start[s + 1]
        int lo = 0, hi = b.n_scans - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(b.tile_start + mid) <= item) lo = mid;
            else hi = mid - 1;
        }
        const int s = lo;
        if (threadIdx.x < 2) sd[threadIdx.x] = b.descs[2 * s + threadIdx.x];
        __syncthreads();
        const Geom &g = sd[0].g;
        const int t = item - __ldg(b.tile_start + s);
        bool staged_item = false;
        if constexpr (STAGED) staged_item = sd[0].tmap_slot >= 0;
        if (staged_item) {
            const int slot = sd[0].tmap_slot;
            constexpr int SX = kStageTileXY, SZ = kStageTileZ;
            const int ntx = (g.nx + SX - 1) / SX, nty = (g.ny + SX - 1) / SX;
            const int x0 = (t % ntx) * SX, y0 = ((t / ntx) % nty) * SX, z0 = (t / (ntx * nty)) * SZ;
            const CUtensorMap *maps = b.tmaps + slot * kNumBoxW;
            if constexpr (STAGED) {
                if (sd[0].n_views > 0 &&
                    !batch_stage_tile<4, FIDX>(sd[0], maps, b.err, b.wait_limit, x0, y0, z0, u.st, sb, stages))
                    return;   // a bounded wait gave up: stop using the stages
                __syncthreads();   // the box's first update is visible before the second
                if (sd[1].n_views > 0 &&
                    !batch_stage_tile<8, FIDX>(sd[1], maps, b.err, b.wait_limit, x0, y0, z0, u.st, sb, stages))
                    return;
            }
        } else {
            const int ntx = (g.nx + BX - 1) / BX, nty = (g.ny + BY - 1) / BY;
            const int tx = t % ntx, ty = (t / ntx) % nty, tz = t / (ntx * nty);
            if (sd[0].n_views > 0)
                batch_ldg_tile<BX, BY, 4, R, KCHUNK, FIDX>(sd[0], tx * BX, ty * BY, tz * R, u.ldg.tab, u.ldg.cls,
                                                          u.ldg.act, &u.ldg.n_act);
            __syncthreads();   // the box's first update is visible before the second
            if (sd[1].n_views > 0)
                batch_ldg_tile<BX, BY, 8, R, KCHUNK, FIDX>(sd[1], tx * BX, ty * BY, tz * R, u.ldg.tab, u.ldg.cls,
                                                          u.ldg.act, &u.ldg.n_act);
        }
        __syncthreads();   // before the next item overwrites sd and item_s
    }
}

template <int TILE, bool FIDX, bool STAGED>
static fdk_status launch_batched_kernel(const BatchLaunch &b, cudaStream_t s)
{
    constexpr TileCfg c = kTiles[TILE];
    constexpr int MINB = STAGED ? 3 : c.minb;
    auto k = fdk_bp_batched_kernel<c.bx, c.by, c.r, MINB, FIDX, STAGED>;
    const int smem = STAGED ? kStages * kStageFloats * (int)sizeof(float) : 0;
    cudaError_t err = cudaSuccess;
    if (STAGED) {
        err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared);
        if (err != cudaSuccess) {
            cudaGetLastError();
            set_error("batched launch: cudaFuncSetAttribute failed: %s", cudaGetErrorString(err));
            return FDK_ERR_CUDA;
        }
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, c.bx * c.by, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    int grid = sms * per_sm;
    if (grid > b.total) grid = b.total;
    if (grid < 1) return FDK_OK;
    k<<<grid, c.bx * c.by, smem, s>>>(b);
    err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("batched launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

template <int TILE, bool FIDX>
static fdk_status launch_batched_tile(const BatchLaunch &b, cudaStream_t s)
{
    constexpr TileCfg c = kTiles[TILE];
    if constexpr (c.bx == kStageTileXY && c.by == kStageTileXY) {
        if (b.n_staged > 0) return launch_batched_kernel<TILE, FIDX, true>(b, s);
    }
    return launch_batched_kernel<TILE, FIDX, false>(b, s);
}

template <bool FIDX>
static fdk_status launch_batched_fidx(const BatchLaunch &b, int tile, cudaStream_t s)
{
    switch (tile) {
    case 2: return launch_batched_tile<2, FIDX>(b, s);
    case 3: return launch_batched_tile<3, FIDX>(b, s);
    case 4: return launch_batched_tile<4, FIDX>(b, s);
    case 5: return launch_batched_tile<5, FIDX>(b, s);
    case 7: return launch_batched_tile<7, FIDX>(b, s);
    default: return launch_batched_tile<0, FIDX>(b, s);
    }
}

void batched_tile_dims(int tile, int *bx, int *by, int *r)
{
    const TileCfg c = kTiles[(tile >= 0 && tile < kNumTiles) ? tile : 0];
    *bx = c.bx;
    *by = c.by;
    *r = c.r;
}

fdk_status launch_batched(const BatchLaunch &b, int tile, bool fidx, cudaStream_t s)
{
    return fidx ? launch_batched_fidx<true>(b, tile, s) : launch_batched_fidx<false>(b, tile, s);
}

}  // namespace fdk
