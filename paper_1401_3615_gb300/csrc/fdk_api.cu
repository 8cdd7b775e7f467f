// C ABI of libfdk: argument checks, error reporting, view passes and the
// fetch-path choice.  Declarations and conventions: include/fdk.h.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

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

static const fdk_opts kDefaultOpts = {FDK_F32, 0, nullptr, FDK_FETCH_AUTO, 0, {0}};

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

static fdk_status check_opts(const fdk_opts *o)
{
    if (o->proj_dtype != FDK_F32 && o->proj_dtype != FDK_BF16 && o->proj_dtype != FDK_F16)
        return fail(FDK_ERR_INVALID_ARG, "unknown proj_dtype");
    if (o->matrices_on_device != 0 && o->matrices_on_device != 1)
        return fail(FDK_ERR_INVALID_ARG, "matrices_on_device must be 0 or 1");
    if (o->fetch < FDK_FETCH_AUTO || o->fetch > FDK_FETCH_TEX)
        return fail(FDK_ERR_INVALID_ARG, "unknown fetch path");
    if (o->zrun != 0 && o->zrun != 4 && o->zrun != 8 && o->zrun != 16)
        return fail(FDK_ERR_INVALID_ARG, "zrun must be 0, 4, 8 or 16");
    for (int q = 0; q < 10; ++q)
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

static int pick_fetch(const fdk_opts *o) { return o->fetch == FDK_FETCH_TEX ? 2 : 1; }

}  // namespace fdk

using namespace fdk;

extern "C" {

const char *fdk_last_error(void) { return g_err; }

int32_t fdk_version(void) { return 1; }

void fdk_release(void) {}

fdk_status fdk_backproject(float *volume, const int32_t dims[3], const float voxel_size[3],
                           const float origin[3], const void *projections, const int32_t det[2],
                           const float *matrices, int32_t n_views, const fdk_opts *opts)
{
    g_err[0] = 0;
    const fdk_opts *o = opts ? opts : &kDefaultOpts;
    fdk_status st = check_opts(o);
    if (st) return st;
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
    if ((st = check_device_ptr(volume, "volume"))) return st;
    if ((st = check_device_ptr(projections, "projections"))) return st;
    if (o->matrices_on_device && (st = check_device_ptr(matrices, "matrices"))) return st;
    if (o->fetch == FDK_FETCH_TEX) return fail(FDK_ERR_UNSUPPORTED, "texture fetch path not built");
    const int fetch = pick_fetch(o);
    cudaStream_t s = (cudaStream_t)o->stream;
    const size_t esz = dtype_size(o->proj_dtype);
    const long long plane = (long long)g.W * g.H;

    for (int v0 = 0; v0 < n_views; v0 += KMAX) {
        const int nv = (n_views - v0 < KMAX) ? (n_views - v0) : KMAX;
        a.g = g;
        a.vol = volume;
        a.proj = static_cast<const char *>(projections) + (size_t)v0 * plane * esz;
        a.plane = plane;
        a.n_views = nv;
        if (o->matrices_on_device) {
            a.mats_dev = matrices + (size_t)v0 * 12;
        } else {
            a.mats_dev = nullptr;
            memcpy(a.mats, matrices + (size_t)v0 * 12, sizeof(float) * 12 * nv);
        }
        if ((st = launch_backproject(a, fetch, o->proj_dtype, o->zrun ? o->zrun : 8, s))) return st;
    }
    return FDK_OK;
}

fdk_status fdk_forwardproject_adjoint(void *projections, const int32_t det[2], const float *volume,
                                      const int32_t dims[3], const float voxel_size[3],
                                      const float origin[3], const float *matrices,
                                      int32_t n_views, const fdk_opts *opts)
{
    (void)projections; (void)det; (void)volume; (void)dims; (void)voxel_size; (void)origin;
    (void)matrices; (void)n_views; (void)opts;
    g_err[0] = 0;
    return fail(FDK_ERR_UNSUPPORTED, "adjoint not built yet");
}

fdk_status fdk_count_updates(int64_t *count, const int32_t dims[3], const float voxel_size[3],
                             const float origin[3], const int32_t det[2], const float *matrices,
                             int32_t n_views, const fdk_opts *opts)
{
    g_err[0] = 0;
    const fdk_opts *o = opts ? opts : &kDefaultOpts;
    fdk_status st = check_opts(o);
    if (st) return st;
    if (!count) return fail(FDK_ERR_INVALID_ARG, "count is null");
    *count = 0;
    Geom g;
    if ((st = check_geometry(dims, voxel_size, origin, det, matrices, n_views, &g))) return st;
    if (n_views == 0) return FDK_OK;
    if ((st = check_matrices(matrices, n_views, o->matrices_on_device))) return st;
    if (o->matrices_on_device && (st = check_device_ptr(matrices, "matrices"))) return st;
    cudaStream_t s = (cudaStream_t)o->stream;
    unsigned long long *dcount = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&dcount, sizeof(unsigned long long), s);
    if (e != cudaSuccess) { set_error("cudaMallocAsync: %s", cudaGetErrorString(e)); return FDK_ERR_OOM; }
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
