// Batched back-projection: many scans of uneven size in one persistent
// launch.  A device work list holds (scan, tile) items; CTAs pull items from
// an atomic counter until the list is exhausted (no CTA ever waits on
// another).  Each item back-projects one tile of one scan: first the views
// whose rays run mostly along x with 4 x 8 warp patches, then the views
// along y with 8 x 4 patches -- the same per-voxel view order as the plain
// entry point, so a batch equals sequential plain calls with the same tile.
#include "fdk_bp_kernel.cuh"

namespace fdk {

template <int BX, int BY, int R, int MINB, bool FIDX>
__global__ void __launch_bounds__(BX * BY, MINB)
fdk_bp_batched_kernel(const ScanDesc *__restrict__ descs, const int *__restrict__ tile_start,
                      int n_scans, int total, int *counter)
{
    constexpr int KCHUNK = 128;
    __shared__ ViewEntry tab[KCHUNK];
    __shared__ unsigned char cls[KCHUNK];
    __shared__ unsigned short act[KCHUNK];
    __shared__ int n_act;
    __shared__ ScanDesc sd[2];
    __shared__ int item_s;

    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int item = item_s;
        if (item >= total) break;   // uniform across the CTA
        // scan of this item: tile_start[s] <= item < tile_start[s + 1]
        int lo = 0, hi = n_scans - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(tile_start + mid) <= item) lo = mid;
            else hi = mid - 1;
        }
        const int s = lo;
        if (threadIdx.x < 2) sd[threadIdx.x] = descs[2 * s + threadIdx.x];
        __syncthreads();
        const Geom &g = sd[0].g;
        const int ntx = (g.nx + BX - 1) / BX, nty = (g.ny + BY - 1) / BY;
        const int t = item - __ldg(tile_start + s);
        const int tx = t % ntx, ty = (t / ntx) % nty, tz = t / (ntx * nty);
        if (sd[0].n_views > 0)
            bp_tile<BX, BY, 4, R, KCHUNK, kLdg, float, FIDX>(sd[0], tx * BX, ty * BY, tz * R, tab, cls, act, &n_act);
        __syncthreads();   // the box's first update is visible before the second
        if (sd[1].n_views > 0)
            bp_tile<BX, BY, 8, R, KCHUNK, kLdg, float, FIDX>(sd[1], tx * BX, ty * BY, tz * R, tab, cls, act, &n_act);
        __syncthreads();   // before the next item overwrites sd and item_s
    }
}

template <int TILE, bool FIDX>
static fdk_status launch_batched_tile(const BatchLaunch &b, cudaStream_t s)
{
    constexpr TileCfg c = kTiles[TILE];
    auto k = fdk_bp_batched_kernel<c.bx, c.by, c.r, c.minb, FIDX>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, c.bx * c.by, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    int grid = sms * per_sm;
    if (grid > b.total) grid = b.total;
    if (grid < 1) return FDK_OK;
    k<<<grid, c.bx * c.by, 0, s>>>(b.descs, b.tile_start, b.n_scans, b.total, b.counter);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("batched launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
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
