// C ABI of libfdk: argument checks, error reporting, view passes and the
// fetch-path choice.  Declarations and conventions: include/fdk.h.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <math.h>
#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>
#include <vector>

#include "fdk_internal.cuh"

namespace fdk {

static thread_local char g_err[512];

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

static fdk_status fail(fdk_status st, const char *msg)
{
    set_error("%s", msg);
    return st;
}

// Testing hooks (include/fdk_testing.h): allocations still to fail, and the
// poll limit of the consumer waits.
static std::atomic<int> g_fail_allocs{0};
static std::atomic<long long> g_wait_limit{kWaitLimit};

// True when this allocation is to fail (and counts it).
static bool injected_alloc_failure()
{
    int n = g_fail_allocs.load();
    while (n > 0)
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return true;
    return false;
}

cudaError_t lib_malloc(void **p, size_t bytes)
{
    if (injected_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s)
{
    if (injected_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, s);
}

cudaError_t lib_malloc_array(cudaArray_t *arr, const cudaChannelFormatDesc *ch, size_t w, size_t h,
                             unsigned flags)
{
    if (injected_alloc_failure()) {
        *arr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocArray(arr, ch, w, h, flags);
}

long long consumer_wait_limit() { return g_wait_limit.load(); }

static const fdk_opts kDefaultOpts = {FDK_F32, 0, nullptr, FDK_FETCH_AUTO, 0, 0, 0, {0}};

// Shared checks for the geometry arguments of every entry point.
static fdk_status check_geometry(const int32_t dims[3], const float voxel_size[3],
                                 const float origin[3], const int32_t det[2],
                                 const float *matrices, int32_t n_views, Geom *g)
{
    if (!dims || !voxel_size || !origin || !det) return fail(FDK_ERR_INVALID_ARG, "null geometry pointer");
    if (n_views < 0) return fail(FDK_ERR_INVALID_ARG, "n_views < 0");
    if (n_views > 0 && !matrices) return fail(FDK_ERR_INVALID_ARG, "matrices is null");
    for (int q = 0; q < 3; ++q) {
        if (dims[q] < 1) return fail(FDK_ERR_INVALID_ARG, "dims must be >= 1");
        if (!(voxel_size[q] > 0.0f) || !(voxel_size[q] < 3.0e38f))
            return fail(FDK_ERR_INVALID_ARG, "voxel_size must be finite and > 0");
        if (!(origin[q] > -3.0e38f && origin[q] < 3.0e38f))
            return fail(FDK_ERR_INVALID_ARG, "origin must be finite");
    }
    if (det[0] < 1 || det[1] < 1) return fail(FDK_ERR_INVALID_ARG, "det must be >= 1");
    // 32-bit in-image offsets: (H + 1) * W must fit in int
    if ((int64_t)det[0] * ((int64_t)det[1] + 1) >= (int64_t)INT32_MAX)
        return fail(FDK_ERR_INVALID_ARG, "detector too large (W*H must be < 2^31)");
    // voxel count must fit int64 with room for byte offsets
    const int64_t nxy = (int64_t)dims[0] * dims[1];
    if (nxy > ((int64_t)1 << 40) / dims[2]) return fail(FDK_ERR_INVALID_ARG, "volume too large");
    if ((int64_t)det[0] * det[1] > ((int64_t)1 << 40) / (n_views > 0 ? n_views : 1))
        return fail(FDK_ERR_INVALID_ARG, "projection stack too large");
    g->nx = dims[0]; g->ny = dims[1]; g->nz = dims[2];
    g->W = det[0]; g->H = det[1];
    for (int q = 0; q < 3; ++q) { g->vs[q] = voxel_size[q]; g->org[q] = origin[q]; }
    return FDK_OK;
}

static fdk_status check_opts(const fdk_opts *o, bool allow_overwrite = false)
{
    if (o->overwrite && !allow_overwrite)
        return fail(FDK_ERR_INVALID_ARG, "overwrite applies to fdk_backproject_host only");
    if (o->proj_dtype != FDK_F32 && o->proj_dtype != FDK_BF16 && o->proj_dtype != FDK_F16)
        return fail(FDK_ERR_INVALID_ARG, "unknown proj_dtype");
    if (o->matrices_on_device != 0 && o->matrices_on_device != 1)
        return fail(FDK_ERR_INVALID_ARG, "matrices_on_device must be 0 or 1");
    if (o->fetch < FDK_FETCH_AUTO || o->fetch > FDK_FETCH_STAGE)
        return fail(FDK_ERR_INVALID_ARG, "unknown fetch path");
    if (o->tile < 0 || o->tile > 7) return fail(FDK_ERR_INVALID_ARG, "tile must be 0..7");
    if (o->autotune != 0 && o->autotune != 1) return fail(FDK_ERR_INVALID_ARG, "autotune must be 0 or 1");
    if (o->overwrite != 0 && o->overwrite != 1) return fail(FDK_ERR_INVALID_ARG, "overwrite must be 0 or 1");
    for (int q = 0; q < 8; ++q)
        if (o->reserved[q] != 0) return fail(FDK_ERR_INVALID_ARG, "reserved option fields must be zero");
    return FDK_OK;
}

static size_t dtype_size(int dt) { return dt == FDK_F32 ? 4 : 2; }

static fdk_status check_matrices(const float *m, int32_t n_views, int on_device)
{
    if (on_device || n_views == 0) return FDK_OK;
    for (int64_t q = 0; q < (int64_t)n_views * 12; ++q)
        if (!(m[q] > -3.0e38f && m[q] < 3.0e38f))
            return fail(FDK_ERR_INVALID_ARG, "matrices must be finite");
    return FDK_OK;
}

// Pointers the library dereferences on the device must be device-accessible.
static fdk_status check_device_ptr(const void *p, const char *what)
{
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("%s: cudaPointerGetAttributes failed: %s", what, cudaGetErrorString(e));
        return FDK_ERR_INVALID_ARG;
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) {
        set_error("%s must be device memory", what);
        return FDK_ERR_INVALID_ARG;
    }
    // kernels run on the current device: memory of another GPU would be a
    // fault there (or a silent peer read), so it is refused
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        set_error("%s: cudaGetDevice failed", what);
        return FDK_ERR_CUDA;
    }
    if (attr.type == cudaMemoryTypeDevice && attr.device != cur) {
        set_error("%s lives on device %d but device %d is current", what, attr.device, cur);
        return FDK_ERR_INVALID_ARG;
    }
    return FDK_OK;
}

static fdk_status check_alignment(const void *p, size_t align, const char *what)
{
    if (((uintptr_t)p) % align != 0) {
        set_error("%s must be %zu-byte aligned", what, align);
        return FDK_ERR_INVALID_ARG;
    }
    return FDK_OK;
}

// ---------------------------------------------------------------------------
// Texture staging.  Texture gather (tld4) is defined for CUDA arrays created
// with cudaArrayTextureGather, so the texture fetch path copies each view into
// a 2D array (block-linear layout, zero border from the sampler) before the
// kernel -- the GPU form of the paper's zero-padding copy (Sec. VI).  The
// arrays are cached per (device, W, H, dtype) and reused by later calls; an
// event recorded after each call's kernels makes the next call, on whatever
// stream, wait before it overwrites them.
struct TexStage {
    int dev, W, H, dtype;
    std::vector<cudaArray_t> arrays;
    std::vector<cudaTextureObject_t> texs;
    cudaEvent_t done = nullptr;
};

static std::mutex g_tex_mu;
static std::vector<std::unique_ptr<TexStage>> g_tex;

static cudaChannelFormatDesc tex_channel(int dtype)
{
    if (dtype == FDK_F32) return cudaCreateChannelDesc<float>();
    if (dtype == FDK_F16) return cudaCreateChannelDescHalf();
    return cudaCreateChannelDesc<unsigned short>();  // BF16 bits, widened in the kernel
}

static void tex_stage_free(TexStage *t)
{
    for (auto o : t->texs) cudaDestroyTextureObject(o);
    for (auto a : t->arrays) cudaFreeArray(a);
    if (t->done) cudaEventDestroy(t->done);
    t->texs.clear();
    t->arrays.clear();
    t->done = nullptr;
}

// Whether this device can gather from W x H arrays at all.
static bool tex_supported(int dev, int W, int H)
{
    int mw = 0, mh = 0;
    if (cudaDeviceGetAttribute(&mw, cudaDevAttrMaxTexture2DGatherWidth, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&mh, cudaDevAttrMaxTexture2DGatherHeight, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return W <= mw && H <= mh;
}

// Find or grow the staging set for (dev, W, H, dtype) to n arrays.  Caller
// holds g_tex_mu.  On failure everything allocated here is released.
static fdk_status tex_stage_get(int dev, int W, int H, int dtype, int n, TexStage **out)
{
    TexStage *t = nullptr;
    for (auto &p : g_tex)
        if (p->dev == dev && p->W == W && p->H == H && p->dtype == dtype) t = p.get();
    if (!t) {
        g_tex.emplace_back(new TexStage());
        t = g_tex.back().get();
        t->dev = dev; t->W = W; t->H = H; t->dtype = dtype;
    }
    if (!t->done && cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(FDK_ERR_CUDA, "cudaEventCreate failed");
    }
    const cudaChannelFormatDesc ch = tex_channel(dtype);
    while ((int)t->arrays.size() < n) {
        cudaArray_t arr = nullptr;
        cudaError_t e = lib_malloc_array(&arr, &ch, W, H, cudaArrayTextureGather);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("texture staging: cudaMallocArray failed: %s", cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? FDK_ERR_OOM : FDK_ERR_CUDA;
        }
        cudaResourceDesc rd;
        memset(&rd, 0, sizeof rd);
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = arr;
        cudaTextureDesc td;
        memset(&td, 0, sizeof td);
        td.addressMode[0] = cudaAddressModeBorder;   // zero outside the image
        td.addressMode[1] = cudaAddressModeBorder;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        cudaTextureObject_t tex = 0;
        e = cudaCreateTextureObject(&tex, &rd, &td, nullptr);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFreeArray(arr);
            set_error("texture staging: cudaCreateTextureObject failed: %s", cudaGetErrorString(e));
            return FDK_ERR_CUDA;
        }
        t->arrays.push_back(arr);
        t->texs.push_back(tex);
    }
    *out = t;
    return FDK_OK;
}

// ---------------------------------------------------------------------------
// Quad staging: one device buffer of quad images per (device, W, H, dtype),
// grown to the largest pass seen, reused by later calls and ordered across
// streams by an event recorded after each call's kernels.
struct QuadStage {
    int dev, W, H, dtype;
    void *buf = nullptr;
    size_t bytes = 0;
    cudaEvent_t done = nullptr;
};

static std::mutex g_quad_mu;
static std::vector<std::unique_ptr<QuadStage>> g_quad;

// Quad cell indices, including those of boundary tiles whose reference cell
// lies up to 64 cells off the image, must be exact FP32 integers.
static bool quad_supported(int W, int H)
{
    return (long long)(W + 3 + 130) * (H + 3 + 130) < (1LL << 23);
}

// Caller holds g_quad_mu.
static fdk_status quad_stage_get(int dev, int W, int H, int dtype, int n, QuadStage **out)
{
    QuadStage *t = nullptr;
    for (auto &p : g_quad)
        if (p->dev == dev && p->W == W && p->H == H && p->dtype == dtype) t = p.get();
    if (!t) {
        g_quad.emplace_back(new QuadStage());
        t = g_quad.back().get();
        t->dev = dev; t->W = W; t->H = H; t->dtype = dtype;
    }
    if (!t->done && cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(FDK_ERR_CUDA, "cudaEventCreate failed");
    }
    const size_t need = (size_t)(W + 3) * (size_t)(H + 3) * quad_elem_size(dtype) * (size_t)n;
    if (t->bytes < need) {
        if (t->buf) {
            cudaEventSynchronize(t->done);   // the old buffer may still be read
            cudaFree(t->buf);
            t->buf = nullptr;
            t->bytes = 0;
        }
        cudaError_t e = lib_malloc(&t->buf, need);
        if (e != cudaSuccess) {
            t->buf = nullptr;
            cudaGetLastError();
            set_error("quad staging: cudaMalloc(%zu) failed: %s", need, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? FDK_ERR_OOM : FDK_ERR_CUDA;
        }
        t->bytes = need;
    }
    *out = t;
    return FDK_OK;
}

static void release_quads()
{
    std::lock_guard<std::mutex> lk(g_quad_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &p : g_quad) {
        cudaSetDevice(p->dev);
        if (p->done) {
            cudaEventSynchronize(p->done);
            cudaEventDestroy(p->done);
        }
        if (p->buf) cudaFree(p->buf);
    }
    g_quad.clear();
    cudaSetDevice(cur);
    cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Staged path: tensor maps are encoded on the host per pass into the kernel
// parameter block (no device memory).  The encoder is a driver entry point.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn tmap_encoder()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// One map per box width (maps[0..kNumBoxW)) over nv FP32 images at base
// (W x H x nv; the row and image strides are multiples of 16 bytes because
// W % 4 == 0).
static fdk_status encode_stage_maps_at(CUtensorMap *maps, const void *base, int W, int H, int nv, int nh = 1,
                                       int dtype = FDK_F32)
{
    EncodeTiledFn enc = tmap_encoder();
    const cuuint64_t esz = dtype == FDK_F32 ? 4u : 2u;
    const CUtensorMapDataType dt = dtype == FDK_F16    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : dtype == FDK_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t gdim[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)nv};
    const cuuint64_t gstride[2] = {(cuuint64_t)W * esz, (cuuint64_t)W * (cuuint64_t)H * esz};
    const cuuint32_t estride[3] = {1, 1, 1};
    for (int q = 0; q < kNumBoxW * nh; ++q) {
        const int m = q / nh, h = q % nh;
        const cuuint32_t box[3] = {(cuuint32_t)box_width(m), (cuuint32_t)(kBoxRows << h), 1};
        CUresult r = enc(&maps[q], dt, 3, const_cast<void *>(base), gdim,
                         gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
            return FDK_ERR_CUDA;
        }
    }
    return FDK_OK;
}

// The pass's maps in the kernel parameters.
static fdk_status encode_stage_maps(BpArgs &a, int W, int H, int nv, int dtype = FDK_F32)
{
    return encode_stage_maps_at(a.tmap, a.proj, W, H, nv, kNumBoxH, dtype);
}

// Host matrices: the views of pass [v0, v0 + nv) whose rays run mostly along
// x (group 0) or along y (group 1) into a's matrices and view indices, with
// the warp patch that touches the fewest L1 banks for them (4 x 8 along x,
// 8 x 4 along y) and, on the staged path, CTAs walking along y for group 1.
// Returns the views taken.
static int fill_orientation_group(BpArgs &a, const float *matrices, int v0, int nv, int group, bool staged)
{
    int cnt = 0;
    for (int k = 0; k < nv; ++k) {
        const float *P = matrices + (size_t)(v0 + k) * 12;
        const bool along_x = fabsf(P[8]) > fabsf(P[9]);
        if (along_x != (group == 0)) continue;
        memcpy(a.mats + 12 * cnt, P, sizeof(float) * 12);
        a.vidx[cnt++] = k;
    }
    a.n_views = cnt;
    a.warp_x = group == 0 ? 4 : 8;
    a.walk_y = group == 1 && staged;
    return cnt;
}

// Adjoint warp patches (voxels along x) for views whose rays run mostly along
// x (2 x 16: 16 across the rays) and along y (16 x 2).  Lanes along a ray
// mostly reduce into the same shared cell, and those reductions serialise;
// 2 x 16 took 1.4% less than 4 x 8 at 512^3 x 496, and 8 x 4 for every view
// 3% more.
constexpr int kAdjPatchAlongX = 2, kAdjPatchAlongY = 16;

// z-run of the adjoint's tiles for host matrices.  A 16-voxel run halves the
// table builds and CTA barriers per voxel but doubles each tile's footprint,
// so it is taken only when
//  - the whole volume lies in front of every source with its smallest w at
//    least half its largest (w is affine, so the corners bound it): no tile
//    reaches near the source, where the longer FP32 tile offsets of a
//    16-voxel run, amplified by 1/w, cost accuracy (a volume that holds
//    the source circle missed the accuracy bar with it); and
//  - the volume-centre 16 x 16 x 16 tile's footprint box, with the kernel's
//    margins and 4-pixel widening, fits half the shared buffer (8192 cells)
//    for at least 90% of up to 32 views spread over the scan, so that the
//    double-buffered splat keeps one barrier per view.
// Measured when the choice was made, on 512^3 x 496 views of 1248 x 960: the
// 16-voxel run took 9% less time than the 8-voxel run (62.1 against 68.5
// ms); at 256^3 (1 mm voxels, boxes of about 14k cells) it took 15% more
// (8.27 against 7.18 ms).
static int adj_z_run(const Geom &g, const float *mats, int n_views)
{
    double wlo = 1e300, whi = -1e300;
    for (int k = 0; k < n_views; ++k) {
        const float *P = mats + (size_t)k * 12;
        for (int c = 0; c < 8; ++c) {
            const double X = (double)g.org[0] + ((c & 1) ? (double)(g.nx - 1) * g.vs[0] : 0.0);
            const double Y = (double)g.org[1] + ((c & 2) ? (double)(g.ny - 1) * g.vs[1] : 0.0);
            const double Z = (double)g.org[2] + ((c & 4) ? (double)(g.nz - 1) * g.vs[2] : 0.0);
            const double w = P[8] * X + P[9] * Y + P[10] * Z + P[11];
            wlo = std::min(wlo, w);
            whi = std::max(whi, w);
        }
    }
    if (!(wlo > 0.0) || wlo < 0.5 * whi) return 8;
    const int BX = 16, BY = 16, R = 16;
    const int tx = (g.nx / 2) / BX * BX, ty = (g.ny / 2) / BY * BY, tz = (g.nz / 2) / R * R;
    const int step = n_views > 32 ? n_views / 32 : 1;
    int tried = 0, fit = 0;
    for (int k = 0; k < n_views; k += step) {
        const float *P = mats + (size_t)k * 12;
        double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
        for (int c = 0; c < 8; ++c) {
            const double X = (double)g.org[0] + (double)(tx + ((c & 1) ? BX - 1 : 0)) * g.vs[0];
            const double Y = (double)g.org[1] + (double)(ty + ((c & 2) ? BY - 1 : 0)) * g.vs[1];
            const double Z = (double)g.org[2] + (double)(tz + ((c & 4) ? R - 1 : 0)) * g.vs[2];
            const double w = P[8] * X + P[9] * Y + P[10] * Z + P[11];
            const double u = (P[0] * X + P[1] * Y + P[2] * Z + P[3]) / w;
            const double v = (P[4] * X + P[5] * Y + P[6] * Z + P[7]) / w;
            umin = std::min(umin, u); umax = std::max(umax, u);
            vmin = std::min(vmin, v); vmax = std::max(vmax, v);
        }
        ++tried;
        const double i0 = std::max(0.0, floor(umin) - 1), i1 = std::min((double)g.W - 1, floor(umax) + 2);
        const double j0 = std::max(0.0, floor(vmin) - 1), j1 = std::min((double)g.H - 1, floor(vmax) + 2);
        if (i1 < i0 || j1 < j0) { ++fit; continue; }       // off the detector: nothing to splat
        const double wide = floor((i1 + 4.0) / 4.0) * 4.0 - floor(i0 / 4.0) * 4.0;
        if (wide * (j1 - j0 + 1) <= 8192.0) ++fit;
    }
    return tried > 0 && fit * 10 >= tried * 9 ? 16 : 8;
}

// Whether the staged path pays for this geometry: the 16 x 16 x 16 tile at
// the volume centre is projected, as the kernel's table builder does, for up
// to 32 views spread over the scan, and the path is taken when at least 90%
// of its pixel boxes fit a stage (coarse voxels on a fine detector give
// boxes too large to stage, and those views would fall back to LDG).
static bool stage_pays(const Geom &g, const float *mats, int n_views, int esz = 4)
{
    const int BX = 16, BY = 16, R = 16;
    const int tx = (g.nx / 2) / BX * BX, ty = (g.ny / 2) / BY * BY, tz = (g.nz / 2) / R * R;
    const int step = n_views > 32 ? n_views / 32 : 1;
    int tried = 0, fit = 0;
    for (int k = 0; k < n_views; k += step) {
        const float *P = mats + (size_t)k * 12;
        double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
        bool front = true;
        for (int c = 0; c < 8; ++c) {
            const double X = (double)g.org[0] + (double)(tx + ((c & 1) ? BX - 1 : 0)) * g.vs[0];
            const double Y = (double)g.org[1] + (double)(ty + ((c & 2) ? BY - 1 : 0)) * g.vs[1];
            const double Z = (double)g.org[2] + (double)(tz + ((c & 4) ? R - 1 : 0)) * g.vs[2];
            const double w = P[8] * X + P[9] * Y + P[10] * Z + P[11];
            if (!(w > 0.0)) { front = false; break; }
            const double u = (P[0] * X + P[1] * Y + P[2] * Z + P[3]) / w;
            const double v = (P[4] * X + P[5] * Y + P[6] * Z + P[7]) / w;
            umin = std::min(umin, u); umax = std::max(umax, u);
            vmin = std::min(vmin, v); vmax = std::max(vmax, v);
        }
        ++tried;
        if (!front || umax - umin > 4096.0 || vmax - vmin > 4096.0) continue;
        const long long i0 = (long long)floor(umin) - 1, i1 = (long long)floor(umax) + 2;
        const long long j0 = (long long)floor(vmin) - 1, j1 = (long long)floor(vmax) + 2;
        const long long wpx = i1 - (i0 & ~(long long)(16 / esz - 1)) + 1;
        const long long m = wpx <= 32 ? 0 : (wpx - 32 + 15) / 16;
        const long long rows8 = (j1 - j0 + kBoxRows) / kBoxRows;
        if (m < kNumBoxW && rows8 * kBoxRows * box_width((int)m) <= (long long)kStageFloats * 4 / esz) ++fit;
    }
    return tried > 0 && fit * 10 >= tried * 9;
}

// What FDK_FETCH_AUTO resolves to the staged path for: tile 0, rows of a
// multiple of 16 bytes, 16-byte aligned images, host matrices, and a
// geometry for which staging pays; FP32, FP16 and BF16 pixels alike.
static bool auto_takes_stage(const Geom &g, const void *projections, const float *matrices, int n_views,
                             const fdk_opts *o)
{
    const int esz = (int)dtype_size(o->proj_dtype);
    return o->tile == 0 && g.W % (16 / esz) == 0 && ((uintptr_t)projections) % 16 == 0 &&
           !o->matrices_on_device && tmap_encoder() && stage_pays(g, matrices, n_views, esz);
}

// One device word per device, set by a bounded wait that gave up.
static std::mutex g_errw_mu;
static std::vector<std::pair<int, unsigned *>> g_errw;

static fdk_status err_word(int dev, unsigned **out)
{
    std::lock_guard<std::mutex> lk(g_errw_mu);
    for (auto &p : g_errw)
        if (p.first == dev) { *out = p.second; return FDK_OK; }
    unsigned *w = nullptr;
    if (lib_malloc((void **)&w, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return fail(FDK_ERR_OOM, "error-word allocation failed");
    }
    if (cudaMemset(w, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(w);
        return fail(FDK_ERR_CUDA, "error-word initialisation failed");
    }
    g_errw.push_back({dev, w});
    *out = w;
    return FDK_OK;
}

static void release_err_words()
{
    std::lock_guard<std::mutex> lk(g_errw_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &p : g_errw) {
        cudaSetDevice(p.first);
        cudaFree(p.second);
    }
    g_errw.clear();
    cudaSetDevice(cur);
    cudaGetLastError();
}

// Ram-Lak spectra and twiddle tables per (device, N), computed once and
// cached: N spectrum floats followed by N twiddles in one allocation.
struct Spectrum {
    int dev, N;
    float *spec;
};
static std::mutex g_spec_mu;
static std::vector<Spectrum> g_spec;

static fdk_status spectrum_get(int dev, int N, const float **out, const float2 **tw)
{
    std::lock_guard<std::mutex> lk(g_spec_mu);
    for (auto &s : g_spec)
        if (s.dev == dev && s.N == N) {
            *out = s.spec;
            *tw = reinterpret_cast<const float2 *>(s.spec + N);
            return FDK_OK;
        }
    float *p = nullptr;
    if (lib_malloc((void **)&p, sizeof(float) * N + sizeof(float2) * N) != cudaSuccess) {
        cudaGetLastError();
        return fail(FDK_ERR_OOM, "filter spectrum allocation failed");
    }
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    fdk_status st = launch_ramlak_spectrum(p, N, s);
    if (st == FDK_OK) st = launch_twiddles(reinterpret_cast<float2 *>(p + N), N, s);
    if (st == FDK_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        st = fail(FDK_ERR_CUDA, "filter spectrum failed");
    }
    cudaStreamDestroy(s);
    if (st) { cudaFree(p); return st; }
    g_spec.push_back({dev, N, p});
    *out = p;
    *tw = reinterpret_cast<const float2 *>(p + N);
    return FDK_OK;
}

static void release_spectra()
{
    std::lock_guard<std::mutex> lk(g_spec_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &s : g_spec) {
        cudaSetDevice(s.dev);
        cudaFree(s.spec);
    }
    g_spec.clear();
    cudaSetDevice(cur);
    cudaGetLastError();
}

void release_textures()
{
    std::lock_guard<std::mutex> lk(g_tex_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &p : g_tex) {
        cudaSetDevice(p->dev);
        cudaDeviceSynchronize();
        tex_stage_free(p.get());
    }
    g_tex.clear();
    cudaSetDevice(cur);
    cudaGetLastError();
}

}  // namespace fdk

using namespace fdk;

extern "C" {

const char *fdk_last_error(void) { return g_err; }

int32_t fdk_version(void) { return 1; }

static void release_host_stages();
namespace fdk { static void release_static_ptrs(); }

void fdk_release(void)
{
    release_textures();
    release_quads();
    release_spectra();
    release_err_words();
    release_host_stages();
    release_static_ptrs();
}

fdk_status fdk_testing_set_wait_limit(int64_t polls)
{
    g_err[0] = 0;
    g_wait_limit.store(polls < 0 ? kWaitLimit : (long long)polls);
    return FDK_OK;
}

fdk_status fdk_testing_fail_allocations(int32_t n)
{
    g_err[0] = 0;
    if (n < 0) return fail(FDK_ERR_INVALID_ARG, "n must be >= 0");
    g_fail_allocs.store(n);
    return FDK_OK;
}

fdk_status fdk_device_status(void)
{
    g_err[0] = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        set_error("device error: %s", cudaGetErrorString(e));
        return FDK_ERR_CUDA;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    unsigned *w = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_errw_mu);
        for (auto &p : g_errw)
            if (p.first == dev) w = p.second;
    }
    if (!w) return FDK_OK;
    unsigned h = 0;
    if (cudaMemcpy(&h, w, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return fail(FDK_ERR_CUDA, "reading the device error word failed");
    }
    if (h) {
        cudaMemset(w, 0, sizeof(unsigned));
        return fail(FDK_ERR_TIMEOUT, "a bounded device-side wait gave up (staged back-projection or "
                                     "row filter); the tiles or rows concerned were not written");
    }
    return FDK_OK;
}

fdk_status fdk_backproject(float *volume, const int32_t dims[3], const float voxel_size[3],
                           const float origin[3], const void *projections, const int32_t det[2],
                           const float *matrices, int32_t n_views, const fdk_opts *opts)
{
    g_err[0] = 0;
    const fdk_opts *o = opts ? opts : &kDefaultOpts;
    fdk_status st = check_opts(o);
    if (st) return st;
    if (o->autotune) return fail(FDK_ERR_INVALID_ARG, "autotune applies to fdk_batch_plan_create only");
    // ~29 KB of kernel parameters, filled per pass; one copy per host thread
    static thread_local BpArgs a;
    Geom g;
    if ((st = check_geometry(dims, voxel_size, origin, det, matrices, n_views, &g))) return st;
    if (!volume) return fail(FDK_ERR_INVALID_ARG, "volume is null");
    if (n_views > 0 && !projections) return fail(FDK_ERR_INVALID_ARG, "projections is null");
    if ((st = check_alignment(volume, 4, "volume"))) return st;
    if (n_views == 0) return FDK_OK;
    if ((st = check_alignment(projections, dtype_size(o->proj_dtype), "projections"))) return st;
    if ((st = check_matrices(matrices, n_views, o->matrices_on_device))) return st;
    if (o->fetch == FDK_FETCH_STAGE) {
        // the staged path's own requirements, checked before any CUDA call
        if (o->tile != 0) return fail(FDK_ERR_INVALID_ARG, "the staged path uses tile 0");
        const int esz = (int)dtype_size(o->proj_dtype);
        if (g.W % (16 / esz) != 0 || ((uintptr_t)projections) % 16 != 0)
            return fail(FDK_ERR_UNSUPPORTED,
                        "the staged path needs rows of a multiple of 16 bytes (W % 4 == 0 for FP32, W % 8 == 0 "
                        "for FP16 / BF16) and 16-byte aligned projections");
    }
    if ((st = check_device_ptr(volume, "volume"))) return st;
    if ((st = check_device_ptr(projections, "projections"))) return st;
    if (o->matrices_on_device && (st = check_device_ptr(matrices, "matrices"))) return st;
    cudaStream_t s = (cudaStream_t)o->stream;
    const size_t esz = dtype_size(o->proj_dtype);
    const long long plane = (long long)g.W * g.H;
    int dev = 0;
    cudaGetDevice(&dev);

    // AUTO takes the staged path where it applies (FP32, tile 0, rows of a
    // multiple of 16 bytes, 16-byte aligned images, host matrices) and pays
    // (the tiles' pixel boxes fit a stage); it is bitwise equal to LDG and
    // measures faster on GB300 there.  LDG elsewhere.  The texture and
    // quad paths only on request: both measure slower than LDG.
    int want = o->fetch;
    if (want == FDK_FETCH_AUTO && auto_takes_stage(g, projections, matrices, n_views, o))
        want = FDK_FETCH_STAGE;
    bool use_tex = false, use_quad = false;
    TexStage *stage = nullptr;
    QuadStage *qstage = nullptr;
    std::unique_lock<std::mutex> lk(g_tex_mu, std::defer_lock);
    std::unique_lock<std::mutex> qlk(g_quad_mu, std::defer_lock);
    const int n_pass = n_views < KMAX ? n_views : KMAX;
    bool use_stage = false;
    a.err = nullptr;
    a.wait_limit = consumer_wait_limit();
    if (want == FDK_FETCH_STAGE) {
        if (!tmap_encoder()) return fail(FDK_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
        if ((st = err_word(dev, &a.err))) return st;
        use_stage = true;
    } else if (want == FDK_FETCH_TEX) {
        if (!tex_supported(dev, g.W, g.H))
            return fail(FDK_ERR_UNSUPPORTED, "detector exceeds the device's texture-gather size");
        lk.lock();
        if ((st = tex_stage_get(dev, g.W, g.H, o->proj_dtype, n_pass, &stage))) return st;
        use_tex = true;
    } else if (want == FDK_FETCH_QUAD) {
        if (!quad_supported(g.W, g.H))
            return fail(FDK_ERR_UNSUPPORTED, "detector too large for quad images (2^23 cells)");
        qlk.lock();
        if ((st = quad_stage_get(dev, g.W, g.H, o->proj_dtype, n_pass, &qstage))) return st;
        use_quad = true;
    }
    cudaEvent_t guard = use_tex ? stage->done : (use_quad ? qstage->done : nullptr);
    if (guard && cudaStreamWaitEvent(s, guard, 0) != cudaSuccess) {
        cudaGetLastError();
        return fail(FDK_ERR_CUDA, "cudaStreamWaitEvent failed");
    }

    int fetch = 1;
    if (use_tex) fetch = 2;
    if (use_quad) fetch = 3;
    if (use_stage) fetch = 4;
    for (int v0 = 0; v0 < n_views; v0 += KMAX) {
        const int nv = (n_views - v0 < KMAX) ? (n_views - v0) : KMAX;
        a.g = g;
        a.vol = volume;
        a.proj = static_cast<const char *>(projections) + (size_t)v0 * plane * esz;
        a.plane = plane;
        a.quads = nullptr;
        a.qpitch = g.W + 3;
        a.qplane = (long long)(g.W + 3) * (g.H + 3);
        if (use_stage && (st = encode_stage_maps(a, g.W, g.H, nv, o->proj_dtype))) return st;
        if (use_tex) {
            for (int k = 0; k < nv; ++k) {
                const char *src = static_cast<const char *>(a.proj) + (size_t)k * plane * esz;
                cudaError_t e = cudaMemcpy2DToArrayAsync(stage->arrays[k], 0, 0, src, g.W * esz,
                                                         g.W * esz, g.H, cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    set_error("texture staging copy failed: %s", cudaGetErrorString(e));
                    return FDK_ERR_CUDA;
                }
                a.tex[k] = (unsigned long long)stage->texs[k];
            }
        }
        if (use_quad) {
            if ((st = launch_make_quads(a.proj, qstage->buf, nv, g.W, g.H, o->proj_dtype, s))) return st;
            a.quads = qstage->buf;
        }
        a.walk_y = 0;
        if (o->matrices_on_device || use_tex) {
            // one launch over the pass in view order with 8 x 4 warp patches
            a.n_views = nv;
            a.warp_x = 8;
            for (int k = 0; k < nv; ++k) a.vidx[k] = k;
            if (o->matrices_on_device) {
                a.mats_dev = matrices + (size_t)v0 * 12;
            } else {
                a.mats_dev = nullptr;
                memcpy(a.mats, matrices + (size_t)v0 * 12, sizeof(float) * 12 * nv);
            }
            if ((st = launch_backproject(a, fetch, o->proj_dtype, o->tile, s))) return st;
            continue;
        }
        // host matrices: one launch per ray orientation, each with the warp
        // patch that touches the fewest L1 banks for its views (rays mostly
        // along x: 4 x 8; along y: 8 x 4); each voxel still sums every view
        a.mats_dev = nullptr;
        for (int group = 0; group < 2; ++group) {
            if (fill_orientation_group(a, matrices, v0, nv, group, use_stage) == 0) continue;
            if ((st = launch_backproject(a, fetch, o->proj_dtype, o->tile, s))) return st;
        }
    }
    if (guard) cudaEventRecord(guard, s);
    return FDK_OK;
}

// ---------------------------------------------------------------------------
// Host-buffer entry point: per device a volume buffer and two projection
// chunk buffers (grown on demand, reused), a copy stream and events.
struct HostStage {
    int dev = 0;
    float *vol = nullptr;
    size_t vol_bytes = 0;
    void *chunk[2] = {nullptr, nullptr};
    size_t chunk_bytes = 0;
    cudaStream_t copy = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
    cudaEvent_t slab_done[4] = {nullptr, nullptr, nullptr, nullptr};
};
constexpr int kHostSlabs = 4;
static std::mutex g_host_mu;
static std::vector<std::unique_ptr<HostStage>> g_host;

static void host_stage_free(HostStage *h)
{
    if (h->copy) cudaStreamSynchronize(h->copy);
    cudaFree(h->vol);
    cudaFree(h->chunk[0]);
    cudaFree(h->chunk[1]);
    for (int b = 0; b < 2; ++b) {
        if (h->copied[b]) cudaEventDestroy(h->copied[b]);
        if (h->consumed[b]) cudaEventDestroy(h->consumed[b]);
    }
    for (cudaEvent_t ev : h->slab_done)
        if (ev) cudaEventDestroy(ev);
    if (h->copy) cudaStreamDestroy(h->copy);
    *h = HostStage();
}

static void release_host_stages()
{
    std::lock_guard<std::mutex> lk(g_host_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &p : g_host) {
        cudaSetDevice(p->dev);
        cudaDeviceSynchronize();
        host_stage_free(p.get());
    }
    g_host.clear();
    cudaSetDevice(cur);
    cudaGetLastError();
}

// Caller holds g_host_mu.
static fdk_status host_stage_get(int dev, size_t vol_bytes, size_t chunk_bytes, HostStage **out)
{
    HostStage *h = nullptr;
    for (auto &p : g_host)
        if (p->dev == dev) h = p.get();
    if (!h) {
        g_host.emplace_back(new HostStage());
        h = g_host.back().get();
        h->dev = dev;
    }
    // created on first use, and again by a later call if a creation failed
    if (!h->copy && cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking) != cudaSuccess) {
        h->copy = nullptr;
        cudaGetLastError();
        return fail(FDK_ERR_CUDA, "copy stream creation failed");
    }
    std::vector<cudaEvent_t *> events;
    for (int b = 0; b < 2; ++b) {
        events.push_back(&h->copied[b]);
        events.push_back(&h->consumed[b]);
    }
    for (cudaEvent_t &ev : h->slab_done) events.push_back(&ev);
    for (cudaEvent_t *ev : events)
        if (!*ev && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess) {
            *ev = nullptr;
            cudaGetLastError();
            return fail(FDK_ERR_CUDA, "event creation failed");
        }
    if (h->vol_bytes < vol_bytes) {
        cudaFree(h->vol);
        h->vol = nullptr;
        h->vol_bytes = 0;
        if (lib_malloc((void **)&h->vol, vol_bytes) != cudaSuccess) {
            h->vol = nullptr;
            cudaGetLastError();
            return fail(FDK_ERR_OOM, "device volume allocation failed");
        }
        h->vol_bytes = vol_bytes;
    }
    if (h->chunk_bytes < chunk_bytes) {
        for (int b = 0; b < 2; ++b) {
            cudaFree(h->chunk[b]);
            h->chunk[b] = nullptr;
        }
        h->chunk_bytes = 0;
        for (int b = 0; b < 2; ++b)
            if (lib_malloc(&h->chunk[b], chunk_bytes) != cudaSuccess) {
                h->chunk[b] = nullptr;
                cudaGetLastError();
                return fail(FDK_ERR_OOM, "device projection chunk allocation failed");
            }
        h->chunk_bytes = chunk_bytes;
    }
    *out = h;
    return FDK_OK;
}

fdk_status fdk_backproject_host(float *volume, const int32_t dims[3], const float voxel_size[3],
                                const float origin[3], const void *projections, const int32_t det[2],
                                const float *matrices, int32_t n_views, const fdk_opts *opts)
{
    g_err[0] = 0;
    const fdk_opts *o = opts ? opts : &kDefaultOpts;
    fdk_status st = check_opts(o, true);
    if (st) return st;
    if (o->autotune) return fail(FDK_ERR_INVALID_ARG, "autotune applies to fdk_batch_plan_create only");
    if (o->matrices_on_device) return fail(FDK_ERR_INVALID_ARG, "fdk_backproject_host takes host matrices");
    Geom g;
    if ((st = check_geometry(dims, voxel_size, origin, det, matrices, n_views, &g))) return st;
    if (!volume) return fail(FDK_ERR_INVALID_ARG, "volume is null");
    if (n_views > 0 && !projections) return fail(FDK_ERR_INVALID_ARG, "projections is null");
    if ((st = check_alignment(volume, 4, "volume"))) return st;
    if (n_views == 0) return FDK_OK;
    const size_t esz = dtype_size(o->proj_dtype);
    if ((st = check_alignment(projections, esz, "projections"))) return st;
    if ((st = check_matrices(matrices, n_views, 0))) return st;
    for (const void *p : {(const void *)volume, projections}) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
            cudaGetLastError();
        } else if (attr.type == cudaMemoryTypeDevice) {
            return fail(FDK_ERR_INVALID_ARG, "fdk_backproject_host takes host buffers (use fdk_backproject)");
        }
    }
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t plane = (size_t)g.W * g.H;
    const size_t vol_bytes = (size_t)g.nx * g.ny * g.nz * sizeof(float);
    // Chunks of views through two device buffers: the copy of one overlaps
    // the back-projection of the one before.  From 64 views on, the chunks
    // double in size from max(8, ceil(n/16)) views, and a chunk takes every
    // remaining view once fewer than twice its size remain.  So the
    // back-projection starts after a short copy, and each chunk's copy hides
    // under the back-projection of the chunk before it, half as large, while
    // the host link moves a view in less than half the time a view's
    // back-projection takes.  Every extra chunk costs a pass over the volume
    // (about 0.25 ms at 512^3), so there are few: 31, 62, 124 and 279 views
    // for 496.
    std::vector<int> sizes;
    if (n_views >= 64) {
        int next = std::max(8, (n_views + 15) / 16), rem = n_views;
        while (rem > 0) {
            const int take = (rem < 2 * next) ? rem : next;
            sizes.push_back(take);
            rem -= take;
            next *= 2;
        }
    } else {
        sizes = {n_views};
    }
    const int C = *std::max_element(sizes.begin(), sizes.end());
    // The last chunk runs as z-slabs of whole 16-voxel tile layers, each
    // copied back while the next is back-projected, when nz >= 64 and every
    // slab origin is exact in FP32 (each voxel keeps its world position and
    // its tile, so the slabs compute what one call over the volume does).
    const int slab_z = ((g.nz + kHostSlabs - 1) / kHostSlabs + 15) / 16 * 16;
    bool slabs = g.nz >= 64 && (o->fetch == FDK_FETCH_AUTO || o->fetch == FDK_FETCH_LDG ||
                                o->fetch == FDK_FETCH_STAGE);   // TEX and QUAD would re-stage per slab
    for (int z0 = slab_z; slabs && z0 < g.nz; z0 += slab_z) {
        const double zo = (double)origin[2] + (double)z0 * (double)voxel_size[2];
        slabs = (double)(float)zo == zo;
    }
    std::lock_guard<std::mutex> lk(g_host_mu);
    HostStage *h = nullptr;
    if ((st = host_stage_get(dev, vol_bytes, (size_t)C * plane * esz, &h))) return st;
    cudaStream_t s = (cudaStream_t)o->stream;
    fdk_opts oc = *o;
    oc.stream = s;
    oc.overwrite = 0;
    const size_t slice = (size_t)g.nx * g.ny;
    cudaError_t e = o->overwrite ? cudaMemsetAsync(h->vol, 0, vol_bytes, s)
                                 : cudaMemcpyAsync(h->vol, volume, vol_bytes, cudaMemcpyHostToDevice, s);
    bool copied_back = false;
    for (int c = 0, v0 = 0; e == cudaSuccess && st == FDK_OK && c < (int)sizes.size(); v0 += sizes[c++]) {
        const int b = c & 1, nv = sizes[c];
        if (c >= 2) e = cudaStreamWaitEvent(h->copy, h->consumed[b], 0);   // buffer b is free
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->chunk[b], static_cast<const char *>(projections) + (size_t)v0 * plane * esz,
                                (size_t)nv * plane * esz, cudaMemcpyHostToDevice, h->copy);
        if (e == cudaSuccess) e = cudaEventRecord(h->copied[b], h->copy);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->copied[b], 0);
        if (e != cudaSuccess) break;
        const float *mk = matrices + (size_t)v0 * 12;
        // AUTO resolved once per chunk on the whole volume, so that slabs take the same path
        oc.fetch = o->fetch;
        if (oc.fetch == FDK_FETCH_AUTO)
            oc.fetch = auto_takes_stage(g, h->chunk[b], mk, nv, &oc) ? FDK_FETCH_STAGE : FDK_FETCH_LDG;
        if (c + 1 < (int)sizes.size() || !slabs) {
            st = fdk_backproject(h->vol, dims, voxel_size, origin, h->chunk[b], det, mk, nv, &oc);
        } else {
            for (int z0 = 0, k = 0; st == FDK_OK && e == cudaSuccess && z0 < g.nz; z0 += slab_z, ++k) {
                const int nz = (g.nz - z0 < slab_z) ? g.nz - z0 : slab_z;
                const int32_t sd[3] = {g.nx, g.ny, nz};
                const float so[3] = {origin[0], origin[1],
                                     (float)((double)origin[2] + (double)z0 * (double)voxel_size[2])};
                st = fdk_backproject(h->vol + (size_t)z0 * slice, sd, voxel_size, so, h->chunk[b], det, mk, nv,
                                     &oc);
                if (st == FDK_OK) e = cudaEventRecord(h->slab_done[k], s);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy, h->slab_done[k], 0);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(volume + (size_t)z0 * slice, h->vol + (size_t)z0 * slice,
                                        (size_t)nz * slice * sizeof(float), cudaMemcpyDeviceToHost, h->copy);
            }
            copied_back = true;
        }
        if (st == FDK_OK && e == cudaSuccess) e = cudaEventRecord(h->consumed[b], s);
    }
    if (e == cudaSuccess && st == FDK_OK && !copied_back)
        e = cudaMemcpyAsync(volume, h->vol, vol_bytes, cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaError_t e3 = cudaStreamSynchronize(h->copy);
    if (st) return st;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = e3;
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("host back-projection: %s", cudaGetErrorString(e));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

fdk_status fdk_forwardproject_adjoint(void *projections, const int32_t det[2], const float *volume,
                                      const int32_t dims[3], const float voxel_size[3],
                                      const float origin[3], const float *matrices,
                                      int32_t n_views, const fdk_opts *opts)
{
    g_err[0] = 0;
    const fdk_opts *o = opts ? opts : &kDefaultOpts;
    fdk_status st = check_opts(o);
    if (st) return st;
    if (o->autotune) return fail(FDK_ERR_INVALID_ARG, "autotune applies to fdk_batch_plan_create only");
    if (o->proj_dtype != FDK_F32) return fail(FDK_ERR_INVALID_ARG, "the adjoint writes FP32 projections only");
    Geom g;
    if ((st = check_geometry(dims, voxel_size, origin, det, matrices, n_views, &g))) return st;
    if (!volume) return fail(FDK_ERR_INVALID_ARG, "volume is null");
    if (n_views > 0 && !projections) return fail(FDK_ERR_INVALID_ARG, "projections is null");
    if ((st = check_alignment(volume, 4, "volume"))) return st;
    if (n_views == 0) return FDK_OK;
    if ((st = check_alignment(projections, 4, "projections"))) return st;
    if ((st = check_matrices(matrices, n_views, o->matrices_on_device))) return st;
    if ((st = check_device_ptr(volume, "volume"))) return st;
    if ((st = check_device_ptr(projections, "projections"))) return st;
    if (o->matrices_on_device && (st = check_device_ptr(matrices, "matrices"))) return st;
    static thread_local BpArgs a;
    cudaStream_t s = (cudaStream_t)o->stream;
    const long long plane = (long long)g.W * g.H;
    // device matrices cannot be read here: the 8-voxel run suits any geometry
    const int z_run = o->matrices_on_device ? 8 : adj_z_run(g, matrices, n_views);
    for (int v0 = 0; v0 < n_views; v0 += KMAX) {
        const int nv = (n_views - v0 < KMAX) ? (n_views - v0) : KMAX;
        a.g = g;
        a.vol = const_cast<float *>(volume);   // read only in the adjoint
        a.proj = nullptr;
        a.quads = nullptr;
        a.plane = plane;
        float *out = static_cast<float *>(projections) + (size_t)v0 * plane;
        if (o->matrices_on_device) {
            // one launch over the pass in view order with 8 x 4 warp patches
            a.n_views = nv;
            a.warp_x = 8;
            a.mats_dev = matrices + (size_t)v0 * 12;
            for (int k = 0; k < nv; ++k) a.vidx[k] = k;
            if ((st = launch_adjoint(a, out, 8, s))) return st;
            continue;
        }
        // host matrices: one launch per ray orientation, with warp patches
        // that lie across the rays (voxels on one ray splat into the same
        // cells, and atomics on one address serialise)
        a.mats_dev = nullptr;
        for (int group = 0; group < 2; ++group) {
            int cnt = 0;
            for (int k = 0; k < nv; ++k) {
                const float *P = matrices + (size_t)(v0 + k) * 12;
                const bool along_x = fabsf(P[8]) > fabsf(P[9]);
                if (along_x != (group == 0)) continue;
                memcpy(a.mats + 12 * cnt, P, sizeof(float) * 12);
                a.vidx[cnt++] = k;
            }
            if (cnt == 0) continue;
            a.n_views = cnt;
            a.warp_x = group == 0 ? kAdjPatchAlongX : kAdjPatchAlongY;
            if ((st = launch_adjoint(a, out, z_run, s))) return st;
        }
    }
    return FDK_OK;
}

fdk_status fdk_count_updates(int64_t *count, const int32_t dims[3], const float voxel_size[3],
                             const float origin[3], const int32_t det[2], const float *matrices,
                             int32_t n_views, const fdk_opts *opts)
{
    g_err[0] = 0;
    const fdk_opts *o = opts ? opts : &kDefaultOpts;
    fdk_status st = check_opts(o);
    if (st) return st;
    if (o->autotune) return fail(FDK_ERR_INVALID_ARG, "autotune applies to fdk_batch_plan_create only");
    if (!count) return fail(FDK_ERR_INVALID_ARG, "count is null");
    *count = 0;
    Geom g;
    if ((st = check_geometry(dims, voxel_size, origin, det, matrices, n_views, &g))) return st;
    if (n_views == 0) return FDK_OK;
    if ((st = check_matrices(matrices, n_views, o->matrices_on_device))) return st;
    if (o->matrices_on_device && (st = check_device_ptr(matrices, "matrices"))) return st;
    cudaStream_t s = (cudaStream_t)o->stream;
    unsigned long long *dcount = nullptr;
    cudaError_t e = lib_malloc_async((void **)&dcount, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("count buffer: cudaMallocAsync failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? FDK_ERR_OOM : FDK_ERR_CUDA;
    }
    cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), s);
    static thread_local BpArgs a;
    for (int v0 = 0; v0 < n_views && st == FDK_OK; v0 += KMAX) {
        const int nv = (n_views - v0 < KMAX) ? (n_views - v0) : KMAX;
        a.g = g;
        a.vol = nullptr;
        a.proj = nullptr;
        a.plane = 0;
        a.n_views = nv;
        if (o->matrices_on_device) {
            a.mats_dev = matrices + (size_t)v0 * 12;
        } else {
            a.mats_dev = nullptr;
            memcpy(a.mats, matrices + (size_t)v0 * 12, sizeof(float) * 12 * nv);
        }
        st = launch_count(a, dcount, s);
    }
    unsigned long long h = 0;
    cudaMemcpyAsync(&h, dcount, sizeof h, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(dcount, s);
    e = cudaStreamSynchronize(s);
    if (st) return st;
    if (e != cudaSuccess) { set_error("count: %s", cudaGetErrorString(e)); return FDK_ERR_CUDA; }
    *count = (int64_t)h;
    return FDK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free back-projection: quad images staged in a fixed array that
// is part of the library image, for callers that must not allocate.
namespace fdk {

static __device__ __align__(256) unsigned char g_static_quads[FDK_STATIC_QUAD_BYTES];

static std::mutex g_static_mu;
static void *g_static_ptr[256] = {};

// Forget the looked-up addresses (fdk_release): after a device reset the
// array lives at a new address in the new context.
static void release_static_ptrs()
{
    std::lock_guard<std::mutex> lk(g_static_mu);
    for (void *&p : g_static_ptr) p = nullptr;
}

// Device address of g_static_quads on the current device, looked up once per
// device (per context: again after fdk_release) with that device current.
// (In host code the symbol is only a host-side stand-in; kernels must get
// this address, never the symbol.)  Under CUDA's lazy module loading this
// lookup is what loads this file's module on the device, and with it
// allocates the array.
static fdk_status static_quads_ptr(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaGetDevice failed: %s", cudaGetErrorString(e));
        return FDK_ERR_CUDA;
    }
    if (dev < 0 || dev >= 256) return fail(FDK_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_quads);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error("cudaGetSymbolAddress of the static staging array failed: %s",
                      cudaGetErrorString(e));
            return FDK_ERR_CUDA;
        }
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return FDK_OK;
}

}  // namespace fdk

extern "C" fdk_status fdk_backproject_static(float *volume, const int32_t dims[3],
                                             const float voxel_size[3], const float origin[3],
                                             const void *projections, const int32_t det[2],
                                             const float *matrices, int32_t n_views,
                                             const fdk_opts *opts)
{
    g_err[0] = 0;
    const fdk_opts *o = opts ? opts : &kDefaultOpts;
    fdk_status st = check_opts(o);
    if (st) return st;
    if (o->autotune) return fail(FDK_ERR_INVALID_ARG, "autotune applies to fdk_batch_plan_create only");
    if (o->fetch != FDK_FETCH_AUTO && o->fetch != FDK_FETCH_QUAD)
        return fail(FDK_ERR_INVALID_ARG, "fdk_backproject_static serves FDK_FETCH_AUTO or FDK_FETCH_QUAD only");
    Geom g;
    if ((st = check_geometry(dims, voxel_size, origin, det, matrices, n_views, &g))) return st;
    if (!volume) return fail(FDK_ERR_INVALID_ARG, "volume is null");
    if (n_views > 0 && !projections) return fail(FDK_ERR_INVALID_ARG, "projections is null");
    if ((st = check_alignment(volume, 4, "volume"))) return st;
    if (!quad_supported(g.W, g.H))
        return fail(FDK_ERR_INVALID_ARG, "detector too large for quad images (2^23 cells)");
    const size_t qbytes = (size_t)(g.W + 3) * (size_t)(g.H + 3) * quad_elem_size(o->proj_dtype);
    if (qbytes > (size_t)FDK_STATIC_QUAD_BYTES) {
        set_error("one quad image needs %zu bytes, more than the %u-byte static staging array",
                  qbytes, (unsigned)FDK_STATIC_QUAD_BYTES);
        return FDK_ERR_INVALID_ARG;
    }
    void *scratch = nullptr;
    if (n_views == 0) return static_quads_ptr(&scratch);   // set-up only
    if ((st = check_alignment(projections, dtype_size(o->proj_dtype), "projections"))) return st;
    if ((st = check_matrices(matrices, n_views, o->matrices_on_device))) return st;
    if ((st = check_device_ptr(volume, "volume"))) return st;
    if ((st = check_device_ptr(projections, "projections"))) return st;
    if (o->matrices_on_device && (st = check_device_ptr(matrices, "matrices"))) return st;
    if ((st = static_quads_ptr(&scratch))) return st;

    static thread_local BpArgs a;
    cudaStream_t s = (cudaStream_t)o->stream;
    const size_t esz = dtype_size(o->proj_dtype);
    const long long plane = (long long)g.W * g.H;
    int per = (int)((size_t)FDK_STATIC_QUAD_BYTES / qbytes);
    if (per > KMAX) per = KMAX;
    for (int v0 = 0; v0 < n_views; v0 += per) {
        const int nv = (n_views - v0 < per) ? (n_views - v0) : per;
        a.g = g;
        a.vol = volume;
        a.proj = static_cast<const char *>(projections) + (size_t)v0 * plane * esz;
        a.plane = plane;
        a.n_views = nv;
        a.qpitch = g.W + 3;
        a.qplane = (long long)(g.W + 3) * (g.H + 3);
        if (o->matrices_on_device) {
            a.mats_dev = matrices + (size_t)v0 * 12;
        } else {
            a.mats_dev = nullptr;
            memcpy(a.mats, matrices + (size_t)v0 * 12, sizeof(float) * 12 * nv);
        }
        if ((st = launch_make_quads(a.proj, scratch, nv, g.W, g.H, o->proj_dtype, s))) return st;
        a.quads = scratch;
        a.warp_x = 8;
        for (int k = 0; k < nv; ++k) a.vidx[k] = k;
        if ((st = launch_backproject(a, FDK_FETCH_QUAD, o->proj_dtype, o->tile, s))) return st;
    }
    return FDK_OK;
}

// ---------------------------------------------------------------------------
// Batched back-projection plans.
struct fdk_batch_plan_t {
    int dev = 0;
    int n_scans = 0;
    int tile = 0;
    bool fidx = true;
    int total = 0;
    void *buf = nullptr;             // descriptors | tile_start | counter | matrices | view indices
    fdk::ScanDesc *d_descs = nullptr;
    int *d_tile_start = nullptr;
    int *d_counter = nullptr;
    std::vector<fdk::ScanDesc> h_descs;
    std::unique_ptr<fdk::BatchLaunch> launch;   // kernel arguments, staged scans' tensor maps included
    std::vector<int> stage_slot;     // per scan: its tensor maps' slot if it can be staged, else -1
    int n_stageable = 0;
    // Scans that fill the GPU on their own may run as their own launches
    // (exactly fdk_backproject's) instead of inside the persistent kernel:
    // staged where the staged path applies, else on the global-load path with
    // the plan's tile variant.
    std::vector<char> alone_ok;      // per scan: may run alone
    std::vector<char> alone;         // per scan: runs alone in this plan
    std::vector<char> alone_staged;  // per scan: its own launches are staged
    std::vector<std::pair<int, std::unique_ptr<fdk::BpArgs>>> alone_args;   // (scan, one launch's arguments)
};

namespace fdk {

// Work-list prefix counts for a tile variant; returns the item total.
static int plan_tile_start(const fdk_batch_plan_t *p, int tile, std::vector<int> &ts)
{
    int bx, by, r;
    batched_tile_dims(tile, &bx, &by, &r);
    ts.assign(p->n_scans + 1, 0);
    long long acc = 0;
    for (int s = 0; s < p->n_scans; ++s) {
        ts[s] = (int)acc;
        const Geom &g = p->h_descs[2 * s].g;
        const bool any = !p->alone[s] && p->h_descs[2 * s].n_views + p->h_descs[2 * s + 1].n_views > 0;
        // staged scans are cut into the staged path's tiles
        const bool staged = p->h_descs[2 * s].tmap_slot >= 0;
        const int sx = staged ? kStageTileXY : bx, sy = staged ? kStageTileXY : by, sz = staged ? kStageTileZ : r;
        if (any) acc += (long long)((g.nx + sx - 1) / sx) * ((g.ny + sy - 1) / sy) * ((g.nz + sz - 1) / sz);
    }
    ts[p->n_scans] = (int)acc;
    return acc > INT32_MAX ? -1 : (int)acc;
}

static fdk_status plan_set_tile(fdk_batch_plan_t *p, int tile)
{
    std::vector<int> ts;
    const int total = plan_tile_start(p, tile, ts);
    if (total < 0) return fail(FDK_ERR_INVALID_ARG, "batch has more than 2^31 work items");
    if (cudaMemcpy(p->d_tile_start, ts.data(), sizeof(int) * ts.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return fail(FDK_ERR_CUDA, "batch plan: upload of the work list failed");
    }
    p->tile = tile;
    p->total = total;
    return FDK_OK;
}

// The persistent kernel over the plan's work list, then the launches of the
// scans that run alone (into vol_override instead of their volumes when it
// is given, for the autotuner).
static fdk_status plan_launch(fdk_batch_plan_t *p, cudaStream_t s, float *vol_override = nullptr)
{
    fdk_status st = FDK_OK;
    if (p->total > 0) {
        if (cudaMemsetAsync(p->d_counter, 0, sizeof(int), s) != cudaSuccess) {
            cudaGetLastError();
            return fail(FDK_ERR_CUDA, "batch: counter reset failed");
        }
        BatchLaunch &b = *p->launch;
        b.total = p->total;
        b.wait_limit = consumer_wait_limit();
        if ((st = launch_batched(b, p->tile, p->fidx, s))) return st;
    }
    for (auto &al : p->alone_args) {
        if (!p->alone[al.first]) continue;
        BpArgs &a = *al.second;
        a.vol = vol_override ? vol_override : p->h_descs[2 * (size_t)al.first].vol;
        a.wait_limit = consumer_wait_limit();
        const bool staged = p->alone_staged[al.first] != 0;
        if ((st = launch_backproject(a, staged ? FDK_FETCH_STAGE : FDK_FETCH_LDG, FDK_F32, staged ? 0 : p->tile, s)))
            return st;
    }
    return FDK_OK;
}

// Tile variants whose CTAs are 16 x 16 threads, as the staged scans' are:
// the only ones a plan with staged scans can run.
static bool tile_is_16x16(int tile)
{
    int bx, by, r;
    batched_tile_dims(tile, &bx, &by, &r);
    return bx == kStageTileXY && by == kStageTileXY;
}

// Stage, inside the persistent kernel, the scans that can be staged and do
// not run alone (on), or none of them (off).  The caller uploads the
// descriptors.
static void plan_set_staging(fdk_batch_plan_t *p, bool on)
{
    int n = 0;
    for (int s = 0; s < p->n_scans; ++s) {
        const int slot = (on && !p->alone[s]) ? p->stage_slot[s] : -1;
        p->h_descs[2 * s].tmap_slot = p->h_descs[2 * s + 1].tmap_slot = slot;
        n += slot >= 0;
    }
    p->launch->n_staged = n;
}

// Time the tile variants, with and without the scans that may run alone
// running alone, and with and without the staged path inside the kernel for
// the other scans that can take it, on the batch with every volume
// redirected to one scratch buffer (the scans' volumes are never written);
// keep the fastest.
static fdk_status plan_autotune(fdk_batch_plan_t *p)
{
    size_t vmax = 0;
    for (int s = 0; s < p->n_scans; ++s) {
        const Geom &g = p->h_descs[2 * s].g;
        vmax = std::max(vmax, (size_t)g.nx * g.ny * g.nz * sizeof(float));
    }
    float *scratch = nullptr;
    if (lib_malloc((void **)&scratch, vmax) != cudaSuccess) {
        cudaGetLastError();
        return fail(FDK_ERR_OOM, "autotune: scratch volume allocation failed");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cands[] = {0, 2, 3, 4, 5, 7};
    int best = 0;
    bool best_staged = false, best_alone = false;
    float best_ms = 3.0e38f;
    fdk_status st = FDK_OK;
    bool any_alone = false;
    for (int s = 0; s < p->n_scans; ++s) any_alone |= p->alone_ok[s] != 0;
    for (int alone = 0; alone < 2 && st == FDK_OK; ++alone) {
        if (alone && !any_alone) break;
        for (int s = 0; s < p->n_scans; ++s) p->alone[s] = alone ? p->alone_ok[s] : 0;
        for (int staged = 0; staged < 2 && st == FDK_OK; ++staged) {
            plan_set_staging(p, staged != 0);
            if (staged && p->launch->n_staged == 0) break;
            std::vector<ScanDesc> tuned = p->h_descs;
            for (auto &d : tuned) d.vol = scratch;
            cudaMemcpy(p->d_descs, tuned.data(), sizeof(ScanDesc) * tuned.size(), cudaMemcpyHostToDevice);
            for (int c : cands) {
                if (staged && !tile_is_16x16(c)) continue;
                if ((st = plan_set_tile(p, c))) break;
                if ((st = plan_launch(p, 0, scratch))) break;            // warm-up
                cudaEventRecord(e0, 0);
                for (int rep = 0; rep < 2 && st == FDK_OK; ++rep) st = plan_launch(p, 0, scratch);
                cudaEventRecord(e1, 0);
                if (cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); st = fail(FDK_ERR_CUDA, "autotune: timing failed"); }
                if (st) break;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_ms) { best_ms = ms; best = c; best_staged = staged != 0; best_alone = alone != 0; }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int s = 0; s < p->n_scans; ++s) p->alone[s] = best_alone ? p->alone_ok[s] : 0;
    plan_set_staging(p, best_staged);
    cudaMemcpy(p->d_descs, p->h_descs.data(), sizeof(ScanDesc) * p->h_descs.size(), cudaMemcpyHostToDevice);
    cudaDeviceSynchronize();
    cudaFree(scratch);
    if (st) return st;
    return plan_set_tile(p, best);
}

}  // namespace fdk

extern "C" {

fdk_status fdk_batch_plan_create(fdk_batch_plan *plan, const fdk_scan *scans, int32_t n_scans,
                                 const fdk_opts *opts)
{
    g_err[0] = 0;
    if (!plan) return fail(FDK_ERR_INVALID_ARG, "plan is null");
    *plan = nullptr;
    fdk_opts o = opts ? *opts : kDefaultOpts;
    const int autotune = o.autotune;
    o.autotune = 0;
    fdk_status st = check_opts(&o);
    if (st) return st;
    if (autotune != 0 && autotune != 1) return fail(FDK_ERR_INVALID_ARG, "autotune must be 0 or 1");
    if (o.proj_dtype != FDK_F32) return fail(FDK_ERR_INVALID_ARG, "batches take FP32 projections");
    if (o.fetch != FDK_FETCH_AUTO && o.fetch != FDK_FETCH_LDG)
        return fail(FDK_ERR_INVALID_ARG, "batches take FDK_FETCH_AUTO (staged where it pays) or FDK_FETCH_LDG");
    if (o.matrices_on_device) return fail(FDK_ERR_INVALID_ARG, "batches take host matrices");
    if (o.tile == 6 || o.tile > 7) return fail(FDK_ERR_INVALID_ARG, "batches take tile variants 0..5 and 7");
    if (n_scans < 1 || !scans) return fail(FDK_ERR_INVALID_ARG, "need at least one scan");
    std::unique_ptr<fdk_batch_plan_t> p(new fdk_batch_plan_t());
    cudaGetDevice(&p->dev);
    p->n_scans = n_scans;
    p->h_descs.resize(2 * (size_t)n_scans);
    size_t total_views = 0;
    for (int s = 0; s < n_scans; ++s) {
        const fdk_scan &sc = scans[s];
        Geom g;
        if ((st = check_geometry(sc.dims, sc.voxel_size, sc.origin, sc.det, sc.matrices, sc.n_views, &g))) {
            char msg[512];
            snprintf(msg, sizeof msg, "scan %d: %s", s, g_err);
            return fail(st, msg);
        }
        if (!sc.volume || (sc.n_views > 0 && !sc.projections)) return fail(FDK_ERR_INVALID_ARG, "scan has a null buffer");
        if ((st = check_alignment(sc.volume, 4, "volume")) || (st = check_alignment(sc.projections, 4, "projections")))
            return st;
        if ((st = check_matrices(sc.matrices, sc.n_views, 0))) return st;
        if ((st = check_device_ptr(sc.volume, "volume"))) return st;
        if (sc.n_views > 0 && (st = check_device_ptr(sc.projections, "projections"))) return st;
        if ((long long)g.W * (g.H + 1) >= (1LL << 23)) p->fidx = false;
        total_views += (size_t)sc.n_views;
    }
    // one device buffer: descriptors | tile_start | counter | matrices | view indices
    const size_t off_ts = sizeof(ScanDesc) * 2 * (size_t)n_scans;
    const size_t off_ctr = off_ts + sizeof(int) * ((size_t)n_scans + 1);
    const size_t off_mats = (off_ctr + sizeof(int) + 15) & ~(size_t)15;
    const size_t off_vidx = off_mats + sizeof(float) * 12 * total_views;
    const size_t bytes = off_vidx + sizeof(int) * total_views + 16;
    if (lib_malloc(&p->buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(FDK_ERR_OOM, "batch plan: device allocation failed");
    }
    char *base = static_cast<char *>(p->buf);
    p->d_descs = reinterpret_cast<ScanDesc *>(base);
    p->d_tile_start = reinterpret_cast<int *>(base + off_ts);
    p->d_counter = reinterpret_cast<int *>(base + off_ctr);
    std::vector<float> hm(12 * total_views);
    std::vector<int> hv(total_views);
    size_t at = 0;
    for (int s = 0; s < n_scans; ++s) {
        const fdk_scan &sc = scans[s];
        for (int group = 0; group < 2; ++group) {
            ScanDesc &d = p->h_descs[2 * s + group];
            memset(&d, 0, sizeof d);
            check_geometry(sc.dims, sc.voxel_size, sc.origin, sc.det, sc.matrices, sc.n_views, &d.g);
            d.vol = sc.volume;
            d.proj = sc.projections;
            d.plane = (long long)sc.det[0] * sc.det[1];
            d.mats_dev = reinterpret_cast<const float *>(base + off_mats) + 12 * at;
            d.mats = nullptr;
            d.vidx = reinterpret_cast<const int *>(base + off_vidx) + at;
            int cnt = 0;
            for (int k = 0; k < sc.n_views; ++k) {
                const float *P = sc.matrices + 12 * (size_t)k;
                const bool along_x = fabsf(P[8]) > fabsf(P[9]);
                if (along_x != (group == 0)) continue;
                memcpy(hm.data() + 12 * (at + cnt), P, sizeof(float) * 12);
                hv[at + cnt] = k;
                ++cnt;
            }
            d.n_views = cnt;
            d.tmap_slot = -1;
            at += cnt;
        }
    }
    // Scans that can take the staged path (where fdk_backproject's AUTO
    // would, on 16 x 16 x 16 tiles): their tensor maps go into the kernel
    // parameters.  They are staged when the plan's tile variant has 16 x 16
    // threads, or, with the autotuner, when staging them measures faster.
    p->launch.reset(new BatchLaunch());
    BatchLaunch &L = *p->launch;
    memset(&L, 0, sizeof L);
    p->stage_slot.assign(n_scans, -1);
    const bool may_stage = o.fetch == FDK_FETCH_AUTO && (autotune || tile_is_16x16(o.tile)) && tmap_encoder();
    for (int s = 0; s < n_scans && may_stage; ++s) {
        const fdk_scan &sc = scans[s];
        const Geom &g = p->h_descs[2 * s].g;
        if (p->n_stageable >= kMaxStagedScans || sc.n_views < 1 || g.W % 4 != 0 ||
            ((uintptr_t)sc.projections) % 16 != 0 || !stage_pays(g, sc.matrices, sc.n_views))
            continue;
        const int slot = p->n_stageable++;
        if ((st = encode_stage_maps_at(L.tmaps + slot * kNumBoxW, sc.projections, g.W, g.H, sc.n_views))) {
            cudaFree(p->buf);
            return st;
        }
        p->stage_slot[s] = slot;
    }
    // Scans that cover two waves of the staged kernel's CTAs on their own run
    // alone by default: their launches (per pass and ray orientation, as
    // fdk_backproject builds them) are prepared here, so that an execution
    // only launches.  Staged where fdk_backproject's AUTO would stage them.
    p->alone_ok.assign(n_scans, 0);
    p->alone.assign(n_scans, 0);
    p->alone_staged.assign(n_scans, 0);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 0;
    }
    const long long alone_tiles = 2LL * 3 * (sms > 0 ? sms : 1);
    unsigned *alone_err = nullptr;
    for (int s = 0; s < n_scans; ++s) {
        const fdk_scan &sc = scans[s];
        const Geom &g = p->h_descs[2 * s].g;
        const long long tiles = (long long)((g.nx + kStageTileXY - 1) / kStageTileXY) *
                                ((g.ny + kStageTileXY - 1) / kStageTileXY) * ((g.nz + kStageTileZ - 1) / kStageTileZ);
        if (sc.n_views < 1 || tiles < alone_tiles) continue;
        const bool staged = o.fetch == FDK_FETCH_AUTO && tmap_encoder() && g.W % 4 == 0 &&
                            ((uintptr_t)sc.projections) % 16 == 0 && stage_pays(g, sc.matrices, sc.n_views);
        if (staged && !alone_err && (st = err_word(p->dev, &alone_err))) {
            cudaFree(p->buf);
            return st;
        }
        const long long plane = (long long)g.W * g.H;
        for (int v0 = 0; v0 < sc.n_views; v0 += KMAX) {
            const int nv = (sc.n_views - v0 < KMAX) ? (sc.n_views - v0) : KMAX;
            for (int group = 0; group < 2; ++group) {
                std::unique_ptr<BpArgs> a(new BpArgs());
                a->g = g;
                a->vol = sc.volume;
                a->proj = static_cast<const float *>(sc.projections) + (size_t)v0 * plane;
                a->plane = plane;
                a->quads = nullptr;
                a->qpitch = g.W + 3;
                a->qplane = (long long)(g.W + 3) * (g.H + 3);
                a->mats_dev = nullptr;
                a->err = staged ? alone_err : nullptr;
                if (staged && (st = encode_stage_maps(*a, g.W, g.H, nv))) {
                    cudaFree(p->buf);
                    return st;
                }
                if (fill_orientation_group(*a, sc.matrices, v0, nv, group, staged) == 0) continue;
                p->alone_args.emplace_back(s, std::move(a));
            }
        }
        p->alone_ok[s] = 1;
        p->alone[s] = 1;
        p->alone_staged[s] = staged;
    }
    plan_set_staging(p.get(), true);
    L.descs = p->d_descs;
    L.tile_start = p->d_tile_start;
    L.counter = p->d_counter;
    L.n_scans = n_scans;
    if (p->n_stageable > 0 && (st = err_word(p->dev, &L.err))) {
        cudaFree(p->buf);
        return st;
    }
    cudaError_t e = cudaMemcpy(base + off_mats, hm.data(), sizeof(float) * hm.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + off_vidx, hv.data(), sizeof(int) * hv.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_descs, p->h_descs.data(), sizeof(ScanDesc) * p->h_descs.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p->buf);
        return fail(FDK_ERR_CUDA, "batch plan: upload failed");
    }
    st = autotune ? plan_autotune(p.get()) : plan_set_tile(p.get(), o.tile);
    if (st) {
        cudaFree(p->buf);
        return st;
    }
    *plan = p.release();
    return FDK_OK;
}

fdk_status fdk_batch_plan_execute(fdk_batch_plan plan, void *stream)
{
    g_err[0] = 0;
    if (!plan) return fail(FDK_ERR_INVALID_ARG, "plan is null");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != plan->dev) return fail(FDK_ERR_INVALID_ARG, "the plan's device is not current");
    return plan_launch(plan, (cudaStream_t)stream);
}

fdk_status fdk_batch_plan_tile(fdk_batch_plan plan, int32_t *tile)
{
    g_err[0] = 0;
    if (!plan || !tile) return fail(FDK_ERR_INVALID_ARG, "null argument");
    *tile = plan->tile;
    return FDK_OK;
}

fdk_status fdk_batch_plan_scan_fetch(fdk_batch_plan plan, int32_t scan, int32_t *fetch)
{
    g_err[0] = 0;
    if (!plan || !fetch) return fail(FDK_ERR_INVALID_ARG, "null argument");
    if (scan < 0 || scan >= plan->n_scans) return fail(FDK_ERR_INVALID_ARG, "scan index out of range");
    const bool staged = plan->alone[scan] ? plan->alone_staged[scan] != 0 : plan->h_descs[2 * (size_t)scan].tmap_slot >= 0;
    *fetch = staged ? FDK_FETCH_STAGE : FDK_FETCH_LDG;
    return FDK_OK;
}

void fdk_batch_plan_destroy(fdk_batch_plan plan)
{
    if (!plan) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(plan->dev);
    cudaFree(plan->buf);
    cudaSetDevice(cur);
    delete plan;
}

fdk_status fdk_backproject_batched(const fdk_scan *scans, int32_t n_scans, const fdk_opts *opts)
{
    fdk_batch_plan plan = nullptr;
    fdk_status st = fdk_batch_plan_create(&plan, scans, n_scans, opts);
    if (st) return st;
    cudaStream_t s = opts ? (cudaStream_t)opts->stream : nullptr;
    st = fdk_batch_plan_execute(plan, s);
    cudaError_t e = cudaStreamSynchronize(s);
    fdk_batch_plan_destroy(plan);
    if (st) return st;
    if (e != cudaSuccess) {
        set_error("batched back-projection: %s", cudaGetErrorString(e));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

}  // extern "C"

extern "C" fdk_status fdk_preweight_filter(float *out, const float *in, const int32_t det[2],
                                           const float *matrices, int32_t n_views, float scale,
                                           const fdk_opts *opts)
{
    g_err[0] = 0;
    const fdk_opts *o = opts ? opts : &kDefaultOpts;
    fdk_status st = check_opts(o);
    if (st) return st;
    if (o->autotune) return fail(FDK_ERR_INVALID_ARG, "autotune applies to fdk_batch_plan_create only");
    if (o->proj_dtype != FDK_F32) return fail(FDK_ERR_INVALID_ARG, "the filter reads and writes FP32");
    if (!det) return fail(FDK_ERR_INVALID_ARG, "det is null");
    if (det[0] < 1 || det[1] < 1) return fail(FDK_ERR_INVALID_ARG, "det must be >= 1");
    if (det[0] > 4096) return fail(FDK_ERR_INVALID_ARG, "the filter takes rows of at most 4096 pixels");
    if (n_views < 0) return fail(FDK_ERR_INVALID_ARG, "n_views < 0");
    if (!(scale > -3.0e38f && scale < 3.0e38f)) return fail(FDK_ERR_INVALID_ARG, "scale must be finite");
    if (n_views == 0) return FDK_OK;
    if (!out || !in || !matrices) return fail(FDK_ERR_INVALID_ARG, "null pointer");
    if ((long long)det[0] * det[1] > ((long long)1 << 40) / n_views)
        return fail(FDK_ERR_INVALID_ARG, "projection stack too large");
    if ((st = check_alignment(out, 4, "out")) || (st = check_alignment(in, 4, "in"))) return st;
    if ((st = check_matrices(matrices, n_views, o->matrices_on_device))) return st;
    if (!o->matrices_on_device) {
        for (int k = 0; k < n_views; ++k) {
            const float *P = matrices + 12 * (size_t)k;
            if (!(P[8] * P[8] + P[9] * P[9] + P[10] * P[10] > 0.0f))
                return fail(FDK_ERR_INVALID_ARG, "matrix row 3 is zero: not a camera");
        }
    }
    if ((st = check_device_ptr(out, "out")) || (st = check_device_ptr(in, "in"))) return st;
    if (o->matrices_on_device && (st = check_device_ptr(matrices, "matrices"))) return st;
    int N = 1;
    while (N < 2 * det[0]) N <<= 1;
    if (N < 4) N = 4;
    if (N == 4096 && 2 * det[0] <= 2560) N = 2560;   // 10 x 16 x 16: 60% of the work
    int dev = 0;
    cudaGetDevice(&dev);
    const float *spec = nullptr;
    const float2 *tw = nullptr;
    if ((st = spectrum_get(dev, N, &spec, &tw))) return st;
    unsigned *errw = nullptr;
    if ((st = err_word(dev, &errw))) return st;
    cudaStream_t s = (cudaStream_t)o->stream;
    const size_t plane = (size_t)det[0] * det[1];
    for (int v0 = 0; v0 < n_views; v0 += KMAX) {
        const int nv = (n_views - v0 < KMAX) ? (n_views - v0) : KMAX;
        if ((st = launch_filter(out + (size_t)v0 * plane, in + (size_t)v0 * plane, spec, tw, scale,
                                o->matrices_on_device ? nullptr : matrices + (size_t)v0 * 12,
                                o->matrices_on_device ? matrices + (size_t)v0 * 12 : nullptr,
                                det[0], det[1], nv, N, errw, s)))
            return st;
    }
    return FDK_OK;
}
