// Internal declarations shared by the libfdk translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "fdk.h"
#include "fdk_testing.h"

namespace fdk {

// Views handled by one kernel pass: their matrices (and texture handles)
// travel in the kernel parameter block, so no device memory is needed for
// them and concurrent calls on different streams cannot race.
constexpr int KMAX = 512;

// Polls of an mbarrier before a device-side wait gives up (a healthy copy
// completes within a few polls).
constexpr long long kWaitLimit = 1LL << 22;

// Staged fetch path: per (tile, view), the pixel box holding every tap of
// the tile is copied into shared memory by TMA as a stack of 8-row boxes of
// one of kNumBoxW widths (32, 48, ..., 128 pixels), at most kStageFloats
// pixels (32 KB); views whose box is larger keep the global-load path.
constexpr int kNumBoxW = 7;
constexpr int kBoxRows = 8;
constexpr int kNumBoxH = 4;        // plain launches: boxes of 8, 16, 32 and 64 rows
constexpr int kStageFloats = 8192;
__host__ __device__ constexpr int box_width(int m) { return 32 + 16 * m; }

struct Geom {
    int nx, ny, nz;
    int W, H;
    float vs[3];
    float org[3];
};

// Everything one back-projection pass needs.  ~31 KB, under the 32 KB
// kernel-parameter limit.
struct BpArgs {
    Geom g;
    float *vol;
    const void *proj;          // first image of this pass
    const float *mats_dev;     // device matrices of this pass, or nullptr
    const void *quads;         // quad images of this pass (quad fetch path), or nullptr
    int qpitch;                // quad cells per quad-image row: W + 3
    long long qplane;          // quad cells per quad image: (W + 3) * (H + 3)
    long long plane;           // W*H elements per image
    int n_views;               // views in this launch (<= KMAX)
    int warp_x;                // voxels along x per warp patch: 8 (8x4) or 4 (4x8)
    int walk_y;                // staged path: 1 = blockIdx.x runs along y (CTAs scheduled in
                               // turn walk along rays that run mostly along y), 0 = along x
    unsigned *err;             // device word set when a bounded wait gives up (staged path)
    long long wait_limit;      // polls before a consumer's wait for a staged view gives up
    float mats[KMAX * 12];     // host matrices of this pass (when mats_dev == nullptr)
    union {
        unsigned long long tex[KMAX];  // texture objects (texture fetch path only)
        CUtensorMap tmap[kNumBoxW * kNumBoxH];  // staged path: the pass's images as a
                                                // W x H x n tensor, one map per box width
                                                // and height (8 << h rows), [m * kNumBoxH + h]
    };
    int vidx[KMAX];            // image index (within the pass's images) of each view
};
static_assert(sizeof(BpArgs) <= 32764, "kernel parameter block limit");

// Per (tile, view) entry computed in each CTA's prologue (shared memory).
// Detector coordinates are kept relative to an integer cell (U, V) near the
// tile's projected centre and the voxel offsets relative to the tile centre,
// so the FP32 arithmetic in the hot loop works on small numbers.  u and v
// coefficients are interleaved so the hot loop can use packed f32x2 math.
struct __align__(16) ViewEntry {
    float4 a;    // (c_u, c_v, gx_u, gx_v): value at the tile centre, step in x
    float4 b;    // (gy_u, gy_v, gz_u, gz_v): steps in y and z
    float4 w;    // (c_w, gx_w, gy_w, gz_w)
    float4 o;    // (U, V, V*W + U + 2^23, (V+2)*(W+3) + U + 2 + 2^23); staged views:
                 // (U, V, (V-j0)*BW + U-x0 + 2^23, BW) for the box at (x0, j0), BW wide
};

// One orientation group of one scan in a batch (device memory).  The field
// names match BpArgs so the same tile code serves both.
struct ScanDesc {
    Geom g;
    float *vol;
    const void *proj;          // the scan's first image
    long long plane;           // W*H
    const float *mats_dev;     // this group's matrices, 12 per view
    const float *mats;         // unused (always nullptr)
    const int *vidx;           // image index of each view of the group
    int n_views;               // views in this group
    int tmap_slot;             // staged scans: index of the scan's tensor maps in the launch; -1: LDG
};

// Scans of one batch that can take the staged path (their tensor maps travel
// in the kernel parameters, kNumBoxW per scan).
constexpr int kMaxStagedScans = 32;

// Arguments of one batched launch (device pointers, plus the staged scans'
// tensor maps).  About 28.7 KB, under the 32 KB kernel-parameter limit.
struct BatchLaunch {
    const ScanDesc *descs;     // 2 per scan: views along x, views along y
    const int *tile_start;     // n_scans + 1 prefix counts of (scan, tile) items
    int *counter;              // work counter, zeroed before the launch
    unsigned *err;             // device word set when a bounded wait gives up (staged scans)
    long long wait_limit;      // polls before a consumer's wait for a staged view gives up
    int n_scans;
    int total;                 // work items
    int n_staged;              // scans with tensor maps (tmap_slot >= 0)
    CUtensorMap tmaps[kMaxStagedScans * kNumBoxW];   // one per box width per staged scan,
                                                     // over the scan's W x H x n_views images
};
static_assert(sizeof(BatchLaunch) <= 32764, "kernel parameter block limit");

enum TileClass : int { kSkip = 0, kInterior = 1, kBoundary = 2, kGeneral = 3, kStaged = 4 };

// Thread-local error message setter (fdk_api.cu).
void set_error(const char *fmt, ...);

// The library's device allocations, all through these wrappers (fdk_api.cu),
// so that the testing hook fdk_testing_fail_allocations can make the next
// ones fail as an out-of-memory device would.
cudaError_t lib_malloc(void **p, size_t bytes);
cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s);
cudaError_t lib_malloc_array(cudaArray_t *arr, const cudaChannelFormatDesc *ch, size_t w, size_t h,
                             unsigned flags);
// Poll limit for the consumer waits of the next launches: kWaitLimit unless a
// test lowered it with fdk_testing_set_wait_limit.
long long consumer_wait_limit();

fdk_status launch_backproject(const BpArgs &a, int fetch, int dtype, int tile,
                              cudaStream_t stream);
void release_textures();
fdk_status launch_ramlak_spectrum(float *spec, int N, cudaStream_t stream);
fdk_status launch_twiddles(float2 *tw, int N, cudaStream_t stream);
fdk_status launch_filter(float *out, const float *in, const float *spec, const float2 *tw, float scale,
                         const float *mats_host, const float *mats_dev, int W, int H, int n_views,
                         int N, unsigned *err, cudaStream_t stream);
fdk_status launch_batched(const BatchLaunch &b, int tile, bool fidx, cudaStream_t stream);
void batched_tile_dims(int tile, int *bx, int *by, int *r);
// Tile of a staged scan in a batch: the staged path's 16 x 16 x 16.
constexpr int kStageTileXY = 16, kStageTileZ = 16;
size_t quad_elem_size(int dtype);
fdk_status launch_make_quads(const void *proj, void *quads, int n, int W, int H, int dtype,
                             cudaStream_t stream);
fdk_status launch_adjoint(const BpArgs &a, float *proj_out, int z_run, cudaStream_t stream);
fdk_status launch_count(const BpArgs &a, unsigned long long *count_dev, cudaStream_t stream);

}  // namespace fdk
