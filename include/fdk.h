/*
 * fdk.h -- C ABI of libfdk, voxel-driven cone-beam back-projection on GB300.
 *
 * The operation (Sec. IV, Listing 1 of Hofmann, Treibig, Hager, Wellein,
 * "Performance Engineering for a Medical Imaging Application on the Intel
 * Xeon Phi Accelerator"): for every projection image k with its 3x4 matrix
 * P_k and every voxel (x, y, z) of the volume,
 *
 *   X = origin + (x, y, z) * voxel_size              world position (mm)
 *   (u', v', w) = P_k (X, 1),  u = u'/w,  v = v'/w    detector position (px)
 *   val = bilinear interpolation of image k at (u, v), zero outside
 *   volume[z][y][x] += val / w^2                      inverse-square weight
 *
 * Conventions (readings of the listing, fixed for this library):
 *  - matrices are row-major 3x4 FP32, 12 floats per view (the listing
 *    stores them column-major; convert at the edge);
 *  - pixel (m, n) -- column m, row n -- is centred at detector position
 *    (m, n) and stored at image[n * W + m]; the cell of (u, v) is
 *    (floor(u), floor(v)) and taps outside 0 <= m < W, 0 <= n < H read 0;
 *  - voxels with w <= 0 (at or behind the source) contribute nothing;
 *  - the volume is x-fastest: volume[(z * ny + y) * nx + x], FP32;
 *  - the library ACCUMULATES (volume +=, as the listing is called once per
 *    projection); the caller zeroes the volume first if needed.
 *
 * Memory: every buffer is owned by the caller.  "device" means memory of the
 * CURRENT CUDA device (cudaMalloc, torch CUDA tensors); kernels run on the
 * current device, so device memory of another GPU is refused
 * (FDK_ERR_INVALID_ARG), managed memory is accepted.  The
 * QUAD and TEX fetch paths stage the images in library-owned device buffers
 * that are allocated on first use for a detector shape, cached per device and
 * reused by later calls (fdk_release() frees them); calls that share one
 * cache entry are ordered by an event, whatever their streams.  The LDG path
 * allocates nothing; the STAGE path allocates only a 4-byte error word per
 * device on first use.  Calls enqueue kernels on opts->stream and return;
 * asynchronous faults surface at the caller's next synchronisation.
 *
 * Sizes: W * (H + 1) < 2^31 cells per image, nx * ny * nz <= 2^40 voxels and
 * W * H * n_views <= 2^40 pixels; every offset into the volume and the image
 * stack is 64-bit (volumes past 2^31 voxels are supported).  On images of
 * 2^23 cells or more the direct-read paths form tap indices in integers
 * instead of FP32, with the same results.  The tile counts along y and z
 * (tiles of 4 to 16 voxels; on the staged path also along x) go in the CUDA
 * grid's y and z dimensions, at most 65535 each: a volume beyond that (from
 * 262,141 voxels along one of those axes with the smallest tiles) makes the
 * launch return FDK_ERR_CUDA.
 *
 * Errors: argument problems return FDK_ERR_INVALID_ARG before anything is
 * enqueued; fdk_last_error() then gives a message (thread-local).  No C++
 * exception crosses this boundary.
 */
#ifndef FDK_H
#define FDK_H

#include <stdint.h>

#if defined(__GNUC__)
#define FDK_API __attribute__((visibility("default")))
#else
#define FDK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fdk_status {
    FDK_OK = 0,
    FDK_ERR_INVALID_ARG = 1,   /* bad pointer, size, dtype or option; nothing enqueued */
    FDK_ERR_UNSUPPORTED = 2,   /* valid request the library cannot serve (e.g. fetch path) */
    FDK_ERR_OOM = 3,           /* a library-side allocation failed */
    FDK_ERR_CUDA = 4,          /* a CUDA runtime call failed; see fdk_last_error() */
    FDK_ERR_TIMEOUT = 5        /* a bounded device-side wait gave up */
} fdk_status;

/* Storage type of the projection images.  Interpolation and accumulation
 * are FP32 whatever the storage type. */
typedef enum fdk_dtype {
    FDK_F32 = 0,
    FDK_BF16 = 1,
    FDK_F16 = 2
} fdk_dtype;

/* How the four taps are fetched.  AUTO picks the fastest path measured on
 * GB300: STAGE where it applies (rows of a multiple of 16 bytes -- W a
 * multiple of 4 for FP32, of 8 for FP16 / BF16 --, a 16-byte aligned base,
 * tile 0, host matrices) and where the footprints of
 * its 16 x 16 x 16 voxel tiles fit its shared-memory stages (judged on the tile
 * at the volume centre for up to 32 views; e.g. 0.5 mm voxels on 0.308 mm
 * pixels at magnification 2), LDG otherwise.  STAGE gives the same bits as
 * LDG with the same tile (tile variant 7, 16 x 16 x 16). */
typedef enum fdk_fetch {
    FDK_FETCH_AUTO = 0,
    FDK_FETCH_LDG = 1,         /* read-only global loads, bounds checked per tile class */
    FDK_FETCH_TEX = 2,         /* 2x2 texture gather with zero border (taps in FP32); the
                                  images are first copied into cached CUDA arrays */
    FDK_FETCH_QUAD = 3,        /* one load per voxel from a zero-bordered "quad image" (each
                                  cell holds its 2x2 taps) built on the device per call in a
                                  cached staging buffer: 16 B per pixel (FP32), 8 B (FP16/BF16) */
    FDK_FETCH_STAGE = 4        /* per (tile, view) the footprint is copied into shared memory
                                  by the tensor-memory accelerator (zeros outside the image)
                                  and the taps read from there (16-bit images as 16-bit boxes,
                                  widened to FP32 per tap); rows of a multiple of 16 bytes
                                  (W % 4 == 0 for FP32, W % 8 == 0 for FP16 / BF16) and a
                                  16-byte aligned base, opts->tile 0 (the
                                  path's own 16 x 16 x 16 tiles), host or device matrices; no
                                  staging memory.  A bounded wait that gives up is reported by
                                  fdk_device_status() */
} fdk_fetch;

/* Optional knobs; pass NULL for defaults.  Zero in any field means default. */
typedef struct fdk_opts {
    int32_t proj_dtype;          /* fdk_dtype of `projections` (default FDK_F32) */
    int32_t matrices_on_device;  /* 1: `matrices` is a device pointer; 0: host */
    void *stream;                /* cudaStream_t; NULL = the legacy default stream */
    int32_t fetch;               /* fdk_fetch */
    int32_t tile;                /* CTA tile variant 0..7 (x by y voxels, z-run per thread):
                                    0: default (currently 16x16, 8)
                                    1: 16x16, 8   2: 32x16, 4   3: 32x16, 8   4: 32x8, 4
                                    5: 16x16, 4   6: 32x8, 16   7: 16x16, 16 */
    int32_t autotune;            /* fdk_batch_plan_create only: 1 = time the tile variants on
                                    the batch and keep the fastest; elsewhere must be 0 */
    int32_t overwrite;           /* fdk_backproject_host only: 1 = the result replaces the host
                                    volume (the device copy starts at zero, so the volume is not
                                    copied in); 0 = accumulate (+=); elsewhere must be 0 */
    int32_t reserved[8];         /* must be zero */
} fdk_opts;

/*
 * fdk_backproject -- accumulate the back-projection of n_views projection
 * images into `volume` (Listing 1, Sec. IV).
 *
 *  volume       device, nz*ny*nx FP32, x fastest; read and written (+=).
 *  dims         host, {nx, ny, nz}, each >= 1.
 *  voxel_size   host, {sx, sy, sz} in mm, each > 0 (the paper's MM).
 *  origin       host, world position (mm) of the centre of voxel (0,0,0)
 *               (the paper's O; -(n-1)/2*size centres the volume).
 *  projections  device, n_views*H*W values of opts->proj_dtype, row-major
 *               per image, images back to back.
 *  det          host, {W, H}: columns (u) and rows (v) per image, >= 1.
 *  matrices     n_views*12 FP32, row-major 3x4 per view; host memory unless
 *               opts->matrices_on_device (then device memory).
 *  n_views      >= 0; 0 is a no-op.
 *
 * Returns FDK_OK once the work is enqueued on opts->stream.
 */
FDK_API fdk_status fdk_backproject(float *volume, const int32_t dims[3], const float voxel_size[3],
                           const float origin[3], const void *projections, const int32_t det[2],
                           const float *matrices, int32_t n_views, const fdk_opts *opts);

/*
 * fdk_forwardproject_adjoint -- the transpose of fdk_backproject (the paper
 * has only the back-projection, Listing 1; its transpose is what gradient
 * based reconstruction needs).  For every view k and voxel, with the same
 * FP32 detector arithmetic as fdk_backproject, volume[z][y][x] / w^2 is
 * spread over the four pixels around (u, v) with the bilinear weights
 * (1-a)(1-b), a(1-b), (1-a)b, ab, accumulating (+=) into `projections`
 * (device, FP32, n_views*H*W); pixels outside the image receive nothing.
 * Same geometry arguments and conventions as fdk_backproject; `volume` is
 * read only; opts->proj_dtype must be FDK_F32.  Accumulation uses atomics,
 * so the result is deterministic only up to FP32 summation order.
 */
FDK_API fdk_status fdk_forwardproject_adjoint(void *projections, const int32_t det[2],
                                      const float *volume, const int32_t dims[3],
                                      const float voxel_size[3], const float origin[3],
                                      const float *matrices, int32_t n_views,
                                      const fdk_opts *opts);

/*
 * fdk_count_updates -- count the voxel/view pairs whose footprint can touch
 * the detector (w > 0, -1 < u < W, -1 < v < H): the "clipped" update count
 * the paper's GUp/s figures are based on (Sec. VII), evaluated in FP32 on
 * the device.  Synchronises opts->stream and writes the count to *count
 * (host).  A reporting aid; it does not change any result.
 */
FDK_API fdk_status fdk_count_updates(int64_t *count, const int32_t dims[3], const float voxel_size[3],
                             const float origin[3], const int32_t det[2],
                             const float *matrices, int32_t n_views, const fdk_opts *opts);

/* Bytes of the fixed staging array behind fdk_backproject_static. */
#define FDK_STATIC_QUAD_BYTES (64u * 1024u * 1024u)

/*
 * fdk_backproject_host -- the back-projection of fdk_backproject (Listing 1,
 * Sec. IV) for buffers in HOST memory.  volume (nz, ny, nx) FP32 is
 * accumulated (+=), or replaced with opts->overwrite = 1 (then it is not
 * copied to the device, whose copy starts at zero); projections
 * (n_views, H, W) in opts->proj_dtype; matrices row-major 3x4 in host memory
 * (matrices_on_device must be 0).  Pinned (page-locked) buffers give
 * overlapped copies; pageable ones work but copy synchronously.
 *
 * How: the volume is copied to the device (or zeroed there).  The
 * projections follow in chunks of views through two device buffers on a copy
 * stream, so the copy of one chunk overlaps the back-projection of the
 * previous one (fdk_backproject on opts->stream, same fetch path and tile;
 * FDK_FETCH_AUTO is resolved once per chunk for the whole volume).
 *   - n_views < 64: one chunk;
 *   - from 64: chunks double in size from max(8, ceil(n/16)) views, and a
 *     chunk takes every remaining view once fewer than twice its size
 *     remain (31, 62, 124 and 279 views for 496), so back-projection starts
 *     after a short copy and each copy hides under the previous chunk's
 *     back-projection.
 * The volume is copied back at the end.  With nz >= 64 the last chunk runs
 * instead as up to 4 z-slabs of whole 16-voxel layers, each copied back
 * while the next is back-projected.  This applies only where every slab
 * origin (origin z + z0 * voxel z) is exact in FP32, and not with
 * FDK_FETCH_TEX or FDK_FETCH_QUAD.  Each voxel then keeps its world position
 * and its tile, so the result is the same as without slabs.  The call
 * synchronises opts->stream before it returns.  Each chunk is its own pass,
 * so the per-voxel summation order differs from one fdk_backproject call
 * over all views by FP32 rounding; with one chunk the results are equal.
 *
 * Device buffers (the volume and two chunks) are cached per device and
 * reused; fdk_release() frees them.  Calls are serialised by the library.
 * Errors: as fdk_backproject; INVALID_ARG also for device buffers or device
 * matrices.
 */
FDK_API fdk_status fdk_backproject_host(float *volume, const int32_t dims[3], const float voxel_size[3],
                                        const float origin[3], const void *projections,
                                        const int32_t det[2], const float *matrices, int32_t n_views,
                                        const fdk_opts *opts);

/*
 * fdk_backproject_static -- the same back-projection as fdk_backproject,
 * for callers that must not allocate device memory.  The paper has no
 * counterpart; this is a service of the library.
 *
 * Who needs it: host applications that reserve the GPU's memory for their
 * own pool at start-up (a cudaMalloc of theirs or ours would then fail or
 * fragment that pool), reconstruction loops with a fixed memory budget that
 * forbid allocation once running, and plugins inside frameworks that own
 * all device memory.  The QUAD and TEX paths of fdk_backproject allocate
 * their staging buffers on first use; this entry point allocates nothing.
 *
 * How: the quad images (see FDK_FETCH_QUAD) are staged in one array of
 * FDK_STATIC_QUAD_BYTES (64 MiB) compiled into the library; every GPU that
 * loads the library holds that array until the process exits.  Views are
 * processed in passes of as many quad images as fit: 16 B per cell of a
 * (W + 3) x (H + 3) grid for FP32 images, 8 B for FP16/BF16 (a 1248 x 960
 * FP32 image takes 19.3 MB, three per pass).  A detector whose single quad
 * image is larger than the array is rejected with FDK_ERR_INVALID_ARG.
 *
 * Arguments, layouts and results are those of fdk_backproject; opts->fetch
 * must be FDK_FETCH_AUTO or FDK_FETCH_QUAD.
 *
 * Set-up: the first call on a device looks up the array's device address
 * with that device current; make that first call before any stream capture.
 * When the array takes device memory: CUDA loads the library's device code
 * per device lazily by default (CUDA_MODULE_LOADING=LAZY), and that lookup
 * is what loads the array's module, so the 64 MiB are taken at the first
 * call on a device, not when the library is loaded.  A caller that reserves
 * the device's memory for its own pool makes one call before reserving it:
 * a call with n_views = 0 (projections and matrices may then be NULL) does
 * the set-up and nothing else.  With CUDA_MODULE_LOADING=EAGER the array is
 * taken when the library's code is loaded.  After cudaDeviceReset, call
 * fdk_release() first: the looked-up address belongs to the old context.
 *
 * All calls on a device share the array, and each call writes every cell it
 * reads before reading it, so nothing carries over from an earlier call;
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on the array and give undefined results.
 */
FDK_API fdk_status fdk_backproject_static(float *volume, const int32_t dims[3],
                                          const float voxel_size[3], const float origin[3],
                                          const void *projections, const int32_t det[2],
                                          const float *matrices, int32_t n_views,
                                          const fdk_opts *opts);

/*
 * fdk_preweight_filter -- the FDK pre-processing that turns raw line
 * integrals into the filtered projections fdk_backproject takes (the paper's
 * data arrives in this form, Sec. IV):
 *
 *   out[k][n][m] = scale * sum_{m'} h(m - m') c_k(m', n) in[k][n][m']
 *   h(0) = 1/4, h(d) = -1/(pi^2 d^2) for odd d, h(d) = 0 for even d != 0
 *   c_k(m, n) = f / sqrt(f^2 + (m - u0)^2 + (n - v0)^2)
 *
 * a cosine pre-weight and a Ram-Lak (ramp) filter along every detector row,
 * the kernel in pixel units: for the FDK weighting with w = depth/SID in the
 * matrices, scale = d_beta / tau, the angular step over the detector pitch
 * scaled to the isocentre (in the length unit of the line integrals).  (f, u0, v0) are
 * read off each matrix through M M^T, assuming square pixels and no skew.
 * The sum is a linear convolution over the row (zero outside it), computed
 * by FFT on the device.
 *
 *  out, in      device, n_views*H*W FP32; out may equal in (in place).
 *  det          host, {W, H}; W <= 4096.
 *  matrices     n_views*12 FP32 row-major, host unless opts->matrices_on_device.
 *  scale        finite.
 * The first call for a row length on a device computes and caches the
 * kernel's spectrum (a few KB; freed by fdk_release) and synchronises once.
 */
FDK_API fdk_status fdk_preweight_filter(float *out, const float *in, const int32_t det[2],
                                        const float *matrices, int32_t n_views, float scale,
                                        const fdk_opts *opts);

/* One scan of a batch: the arguments of one fdk_backproject call (FP32
 * projections, host matrices). */
typedef struct fdk_scan {
    float *volume;               /* device, nz*ny*nx FP32, accumulated (+=) */
    int32_t dims[3];             /* nx, ny, nz */
    float voxel_size[3];
    float origin[3];
    const float *projections;    /* device, n_views*H*W FP32 */
    int32_t det[2];              /* W, H */
    const float *matrices;       /* host, n_views*12 FP32, row-major 3x4 */
    int32_t n_views;
} fdk_scan;

/* Opaque plan for back-projecting a fixed set of scans (the batched form). */
typedef struct fdk_batch_plan_t *fdk_batch_plan;

/*
 * fdk_batch_plan_create -- prepare the back-projection of n_scans scans of
 * uneven volume, view and detector size as one persistent launch (plus the
 * own launches of scans that fill the GPU alone, below).  Each
 * scan is exactly one fdk_backproject call (Listing 1, Sec. IV); the batch
 * only changes how the work is scheduled.  The plan copies the scans'
 * descriptors, matrices and a (scan, tile) work list to device memory it
 * owns (synchronously, on the current device) and keeps the scans' device
 * pointers: the volumes and projections must stay allocated while the plan
 * is used.  With opts->autotune = 1 it times the tile variants 0, 2..5 and 7
 * on the batch (writing into a scratch volume, never into the scans'
 * volumes) and keeps the fastest; otherwise opts->tile (0..5 or 7) is used.
 * opts->proj_dtype must be FDK_F32.
 *
 * Fetch path per scan: with opts->fetch = FDK_FETCH_AUTO (the default) a
 * scan takes the staged path where fdk_backproject's AUTO would (W a
 * multiple of 4, a 16-byte aligned base, footprints that fit the stages),
 * on its own 16 x 16 x 16 tiles, for up to 32 scans of the batch, provided
 * the plan's tile variant has 16 x 16 threads (0, 5, 7); the other scans
 * take the global-load path on the plan's tile variant.  A scan with at
 * least two waves of the staged kernel's 16 x 16 x 16 tiles on its own
 * (2 x 3 CTAs per SM) runs alone instead: its own launches, exactly those of
 * fdk_backproject, prepared at plan creation and issued after the persistent
 * kernel -- with FDK_FETCH_STAGE where the staged path applies as above (no
 * limit on their number), else with FDK_FETCH_LDG and the plan's tile
 * variant.  The autotuner
 * times the plan with and without those scans running alone, and with and
 * without staging the other stageable scans inside the persistent kernel
 * (which then runs both paths at the staged path's 3 CTAs per SM, which can
 * cost the global-load scans more than staging saves), and keeps the
 * fastest.  FDK_FETCH_LDG: every scan takes the global-load path inside the
 * persistent kernel.  fdk_batch_plan_scan_fetch tells which path a scan
 * takes.  A staged scan's bounded waits are reported by fdk_device_status(),
 * as for fdk_backproject.
 */
FDK_API fdk_status fdk_batch_plan_create(fdk_batch_plan *plan, const fdk_scan *scans,
                                         int32_t n_scans, const fdk_opts *opts);

/*
 * fdk_batch_plan_execute -- enqueue the batch on `stream` (cudaStream_t,
 * NULL = legacy default stream): a reset of the plan's work counter and one
 * persistent kernel in which CTAs take (scan, tile) items from that counter
 * until none are left, then the launches of the scans that run alone.  Every
 * volume is accumulated (+=) exactly as by fdk_backproject, bit for bit: with
 * FDK_FETCH_STAGE for the staged scans (inside the kernel or alone), with
 * FDK_FETCH_LDG and the plan's tile variant for the others.  It allocates nothing and does not synchronise.  Executions of one plan must not
 * overlap on the GPU (they share the counter); the plan's device must be
 * current.
 */
FDK_API fdk_status fdk_batch_plan_execute(fdk_batch_plan plan, void *stream);

/* The tile variant a plan uses (the autotuner's pick when it ran).  A service
 * call of the batched form; the paper has no counterpart. */
FDK_API fdk_status fdk_batch_plan_tile(fdk_batch_plan plan, int32_t *tile);

/* The fetch path scan `scan` of a plan takes: FDK_FETCH_STAGE or
 * FDK_FETCH_LDG, in *fetch.  A service call of the batched form; the paper has
 * no counterpart. */
FDK_API fdk_status fdk_batch_plan_scan_fetch(fdk_batch_plan plan, int32_t scan, int32_t *fetch);

/* Free a plan's device memory.  No execution of it may still be in flight.
 * A service call; the paper has no counterpart. */
FDK_API void fdk_batch_plan_destroy(fdk_batch_plan plan);

/* The batched form in one call (each scan as fdk_backproject, Listing 1,
 * Sec. IV): create, execute on opts->stream, synchronise that stream,
 * destroy. */
FDK_API fdk_status fdk_backproject_batched(const fdk_scan *scans, int32_t n_scans,
                                           const fdk_opts *opts);

/* A service call (the paper has no counterpart).  Synchronise the current
 * device, then report whether a bounded device-side wait of an earlier call
 * on it gave up (FDK_ERR_TIMEOUT) or the device reported an error
 * (FDK_ERR_CUDA).  Clears the timeout record.  Two paths have such waits:
 * the FDK_FETCH_STAGE back-projection (a tile whose wait gave up is left
 * unwritten) and fdk_preweight_filter's staged rows (a CTA whose wait gave
 * up leaves its remaining row pairs unwritten). */
FDK_API fdk_status fdk_device_status(void);

/* Gather micro-benchmarks of the device (the GB300 counterpart of the
 * paper's gather measurements, Sec. V, Table II).  Synchronous; allocates
 * and frees its own scratch memory (up to param KiB for FDK_MICRO_CHASE).
 *   FDK_MICRO_LDG    warp-wide 4-byte loads from L1-resident data whose 32
 *                    lanes touch `param` distinct 128-byte lines (param
 *                    divides 32) -> warp loads per SM per cycle
 *   FDK_MICRO_LDS    shared-memory loads with a `param`-way bank conflict
 *                    (param divides 32) -> warp loads per SM per cycle
 *   FDK_MICRO_TLD4   2x2 texture gathers at random texels of a param x param
 *                    FP32 texture (2..4096) -> warp gathers per SM per cycle
 *   FDK_MICRO_RCP    rcp.approx -> warp instructions per SM per cycle
 *   FDK_MICRO_CHASE  one thread's dependent loads over a param-KiB ring
 *                    (1 KiB .. 4 GiB) -> cycles per load
 * The SM clock is measured alongside.  INVALID_ARG for an unknown
 * benchmark or parameter, OOM when scratch cannot be allocated. */
typedef enum fdk_micro {
    FDK_MICRO_LDG = 1,
    FDK_MICRO_LDS = 2,
    FDK_MICRO_TLD4 = 3,
    FDK_MICRO_RCP = 4,
    FDK_MICRO_CHASE = 5
} fdk_micro;
FDK_API fdk_status fdk_microbench(int32_t which, int32_t param, double *result);

/* Message for the last non-OK status returned on this thread ("" if none).
 * The service calls below have no counterpart in the paper. */
FDK_API const char *fdk_last_error(void);

/* Drop cached per-buffer state (texture arrays, staging buffers, spectra,
 * host-path buffers, error words, the static array's looked-up addresses) on
 * all devices.  Call only when no work that uses them is in flight, and
 * after a cudaDeviceReset before the next call. */
FDK_API void fdk_release(void);

/* ABI version, currently 1. */
FDK_API int32_t fdk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FDK_H */
