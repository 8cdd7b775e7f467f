/*
 * FP64 CPU oracle for voxel-driven cone-beam back-projection.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * definition that the CUDA library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * path never does.  It shares no code, header or constant with the CUDA
 * library.
 *
 * What it computes (Sec. IV, Listing 1 of Hofmann et al., "Performance
 * Engineering for a Medical Imaging Application on the Intel Xeon Phi
 * Accelerator"): for every projection k and every voxel (x, y, z)
 *   X = origin + (x, y, z) * voxel_size                   world coordinates
 *   (u', v', w) = P_k (X, 1)                              forward projection
 *   u = u'/w, v = v'/w                                    dehomogenisation
 *   i = floor(u), j = floor(v), a = u - i, b = v - j      cell and weights
 *   p(m, n) = I_k[n*W + m] inside the detector, else 0    four taps
 *   val = (1-b)((1-a)p(i,j) + a p(i+1,j)) + b((1-a)p(i,j+1) + a p(i+1,j+1))
 *   f[z][y][x] += val / w^2                               inverse-square weight
 * in double precision, views in index order, the volume accumulated (+=).
 *
 * Readings of the listing where it is silent or garbled:
 *  - P_k is row-major 3x4 (the listing stores it column-major);
 *  - the bounds are 0 <= m < W (columns, u) and 0 <= n < H (rows, v); the
 *    listing swaps the names width/height in its tests but addresses the
 *    image as iiy*width + iix;
 *  - float to int is floor (the listing's (int) cast truncates, which only
 *    differs for u or v in (-1, 0)); literal_trunc = 1 selects truncation;
 *  - a voxel with w <= 0 (behind the source) contributes nothing;
 *  - integer (u, v) is the centre of pixel (u, v).
 *
 * Parity pins live in the tests: constant projections (closed form
 * c * sum_k 1/w_k^2), an orthographic matrix that copies the image into the
 * volume, brute-force tent sums, linearity, scale, view chunking, view
 * permutation, the adjoint dot product and the thread split; for the
 * clipped update count, orthographic closed forms and a vectorised count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_THREADS 1024

/* One voxel against one view (Sec. IV, Listing 1: the projection, the
 * dehomogenisation and the cell of the bilinear taps): detector cell
 * (i, j), weights (a, b) and 1/w^2.  Returns 0 when the voxel contributes
 * nothing: w <= 0 (behind the source), or all four taps outside the W x H
 * image (then every tap reads zero, so skipping is exact and keeps the int64
 * conversion defined). */
static int oracle_cell(const double P[12], double X, double Y, double Z, int64_t W, int64_t H,
                       int literal_trunc, int64_t *i, int64_t *j, double *a, double *b,
                       double *inv_w2)
{
    double up = P[0] * X + P[1] * Y + P[2] * Z + P[3];
    double vp = P[4] * X + P[5] * Y + P[6] * Z + P[7];
    double w = P[8] * X + P[9] * Y + P[10] * Z + P[11];
    if (!(w > 0.0)) return 0;
    double u = up / w;
    double v = vp / w;
    double fu = literal_trunc ? trunc(u) : floor(u);
    double fv = literal_trunc ? trunc(v) : floor(v);
    if (!(fu >= -1.0 && fu < (double)W && fv >= -1.0 && fv < (double)H)) return 0;
    *i = (int64_t)fu;
    *j = (int64_t)fv;
    *a = u - fu;
    *b = v - fv;
    *inv_w2 = 1.0 / (w * w);
    return 1;
}

static double oracle_tap(const float *img, int64_t W, int64_t H, int64_t m, int64_t n)
{
    if (m < 0 || m >= W || n < 0 || n >= H) return 0.0;
    return (double)img[n * W + m];
}

typedef struct {
    double *vol;
    const float *proj;
    const float *mats;
    int64_t nx, ny, nz, W, H, n_views;
    double vs[3], org[3];
    int literal_trunc;
    int64_t line_begin, line_end;   /* collapsed (z, y) lines owned by this worker */
} bp_job;

static void *bp_worker(void *arg)
{
    bp_job *jb = (bp_job *)arg;
    const int64_t plane = jb->W * jb->H;
    for (int64_t k = 0; k < jb->n_views; ++k) {
        double P[12];
        for (int q = 0; q < 12; ++q) P[q] = (double)jb->mats[k * 12 + q];
        const float *img = jb->proj + k * plane;
        for (int64_t line = jb->line_begin; line < jb->line_end; ++line) {
            int64_t z = line / jb->ny, y = line % jb->ny;
            double Z = jb->org[2] + (double)z * jb->vs[2];
            double Y = jb->org[1] + (double)y * jb->vs[1];
            double *row = jb->vol + (z * jb->ny + y) * jb->nx;
            for (int64_t x = 0; x < jb->nx; ++x) {
                double X = jb->org[0] + (double)x * jb->vs[0];
                int64_t i, j;
                double a, b, iw2;
                if (!oracle_cell(P, X, Y, Z, jb->W, jb->H, jb->literal_trunc, &i, &j, &a, &b, &iw2)) continue;
                double p00 = oracle_tap(img, jb->W, jb->H, i, j);
                double p10 = oracle_tap(img, jb->W, jb->H, i + 1, j);
                double p01 = oracle_tap(img, jb->W, jb->H, i, j + 1);
                double p11 = oracle_tap(img, jb->W, jb->H, i + 1, j + 1);
                double lo = (1.0 - a) * p00 + a * p10;
                double hi = (1.0 - a) * p01 + a * p11;
                double val = (1.0 - b) * lo + b * hi;
                row[x] += val * iw2;
            }
        }
    }
    return NULL;
}

static int check_geom(const int64_t dims[3], int64_t W, int64_t H, int64_t n_views)
{
    if (!dims || dims[0] < 0 || dims[1] < 0 || dims[2] < 0) return -1;
    if (W <= 0 || H <= 0 || n_views < 0) return -1;
    return 0;
}

/* Back-project n_views projections into vol (nz, ny, nx) doubles, +=
 * (Sec. IV, Listing 1, applied once per projection).
 * The thread split is over collapsed (z, y) lines in equal static chunks,
 * as the paper's OpenMP collapse(z, y) schedule (Sec. VI); every voxel still
 * sums its views in index order, so any nthreads gives the same bits. */
int oracle_backproject(double *vol, const int64_t dims[3], const double voxel_size[3],
                       const double origin[3], const float *proj, int64_t W, int64_t H,
                       const float *mats, int64_t n_views, int nthreads, int literal_trunc)
{
    if (check_geom(dims, W, H, n_views)) return -1;
    int64_t lines = dims[1] * dims[2];
    if (lines == 0 || dims[0] == 0 || n_views == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ORACLE_MAX_THREADS) nthreads = ORACLE_MAX_THREADS;
    if (nthreads > lines) nthreads = (int)lines;
    bp_job *jobs = (bp_job *)calloc((size_t)nthreads, sizeof(bp_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    for (int t = 0; t < nthreads; ++t) {
        bp_job *jb = &jobs[t];
        jb->vol = vol; jb->proj = proj; jb->mats = mats;
        jb->nx = dims[0]; jb->ny = dims[1]; jb->nz = dims[2];
        jb->W = W; jb->H = H; jb->n_views = n_views;
        for (int q = 0; q < 3; ++q) { jb->vs[q] = voxel_size[q]; jb->org[q] = origin[q]; }
        jb->literal_trunc = literal_trunc;
        jb->line_begin = lines * t / nthreads;
        jb->line_end = lines * (t + 1) / nthreads;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, bp_worker, &jobs[t]) != 0) break;
        started = t;
    }
    bp_worker(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    /* if a thread failed to start, do its lines here (same per-voxel order) */
    for (int t = started + 1; t < nthreads; ++t) bp_worker(&jobs[t]);
    free(jobs);
    free(th);
    return 0;
}

/* Back-project into a list of voxels only (Sec. IV, Listing 1, restricted
 * to the listed voxels): out[q] += f at voxel
 * (xyz[3q], xyz[3q+1], xyz[3q+2]).  Same arithmetic as oracle_backproject,
 * used to check sampled voxels of volumes too large for the full oracle. */
int oracle_backproject_voxels(double *out, const int64_t *xyz, int64_t n_vox,
                              const double voxel_size[3], const double origin[3],
                              const float *proj, int64_t W, int64_t H, const float *mats,
                              int64_t n_views)
{
    if (W <= 0 || H <= 0 || n_views < 0 || n_vox < 0) return -1;
    const int64_t plane = W * H;
    for (int64_t q = 0; q < n_vox; ++q) {
        double X = origin[0] + (double)xyz[3 * q + 0] * voxel_size[0];
        double Y = origin[1] + (double)xyz[3 * q + 1] * voxel_size[1];
        double Z = origin[2] + (double)xyz[3 * q + 2] * voxel_size[2];
        double acc = out[q];
        for (int64_t k = 0; k < n_views; ++k) {
            double P[12];
            for (int c = 0; c < 12; ++c) P[c] = (double)mats[k * 12 + c];
            int64_t i, j;
            double a, b, iw2;
            if (!oracle_cell(P, X, Y, Z, W, H, 0, &i, &j, &a, &b, &iw2)) continue;
            const float *img = proj + k * plane;
            double lo = (1.0 - a) * oracle_tap(img, W, H, i, j) + a * oracle_tap(img, W, H, i + 1, j);
            double hi = (1.0 - a) * oracle_tap(img, W, H, i, j + 1) + a * oracle_tap(img, W, H, i + 1, j + 1);
            acc += ((1.0 - b) * lo + b * hi) * iw2;
        }
        out[q] = acc;
    }
    return 0;
}

typedef struct {
    double *proj_out;
    const float *vol;
    const float *mats;
    int64_t nx, ny, nz, W, H;
    double vs[3], org[3];
    int64_t view_begin, view_end;   /* views owned by this worker */
} adj_job;

static void *adj_worker(void *arg)
{
    adj_job *jb = (adj_job *)arg;
    const int64_t plane = jb->W * jb->H;
    for (int64_t k = jb->view_begin; k < jb->view_end; ++k) {
        double P[12];
        for (int q = 0; q < 12; ++q) P[q] = (double)jb->mats[k * 12 + q];
        double *img = jb->proj_out + k * plane;
        for (int64_t z = 0; z < jb->nz; ++z) {
            double Z = jb->org[2] + (double)z * jb->vs[2];
            for (int64_t y = 0; y < jb->ny; ++y) {
                double Y = jb->org[1] + (double)y * jb->vs[1];
                const float *row = jb->vol + (z * jb->ny + y) * jb->nx;
                for (int64_t x = 0; x < jb->nx; ++x) {
                    double X = jb->org[0] + (double)x * jb->vs[0];
                    int64_t i, j;
                    double a, b, iw2;
                    if (!oracle_cell(P, X, Y, Z, jb->W, jb->H, 0, &i, &j, &a, &b, &iw2)) continue;
                    double g = (double)row[x] * iw2;
                    /* transpose of the four taps: scatter g with the same weights */
                    int64_t ms[4] = {i, i + 1, i, i + 1};
                    int64_t ns[4] = {j, j, j + 1, j + 1};
                    double ws[4] = {(1.0 - b) * (1.0 - a), (1.0 - b) * a, b * (1.0 - a), b * a};
                    for (int t = 0; t < 4; ++t) {
                        if (ms[t] < 0 || ms[t] >= jb->W || ns[t] < 0 || ns[t] >= jb->H) continue;
                        img[ns[t] * jb->W + ms[t]] += g * ws[t];
                    }
                }
            }
        }
    }
    return NULL;
}

/* Transpose of oracle_backproject, the operator of Sec. IV, Listing 1 (the
 * paper has no adjoint; this is the plain transpose of that definition):
 * proj_out (n_views, H, W) doubles +=
 * sum over voxels of vol * (tap weight) / w^2.  Threads split views, so each
 * detector pixel is written by one thread in (z, y, x) voxel order. */
int oracle_adjoint(double *proj_out, const int64_t dims[3], const double voxel_size[3],
                   const double origin[3], const float *vol, int64_t W, int64_t H,
                   const float *mats, int64_t n_views, int nthreads)
{
    if (check_geom(dims, W, H, n_views)) return -1;
    if (n_views == 0 || dims[0] * dims[1] * dims[2] == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ORACLE_MAX_THREADS) nthreads = ORACLE_MAX_THREADS;
    if (nthreads > n_views) nthreads = (int)n_views;
    adj_job *jobs = (adj_job *)calloc((size_t)nthreads, sizeof(adj_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    for (int t = 0; t < nthreads; ++t) {
        adj_job *jb = &jobs[t];
        jb->proj_out = proj_out; jb->vol = vol; jb->mats = mats;
        jb->nx = dims[0]; jb->ny = dims[1]; jb->nz = dims[2];
        jb->W = W; jb->H = H;
        for (int q = 0; q < 3; ++q) { jb->vs[q] = voxel_size[q]; jb->org[q] = origin[q]; }
        jb->view_begin = n_views * t / nthreads;
        jb->view_end = n_views * (t + 1) / nthreads;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, adj_worker, &jobs[t]) != 0) break;
        started = t;
    }
    adj_worker(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    for (int t = started + 1; t < nthreads; ++t) adj_worker(&jobs[t]);
    free(jobs);
    free(th);
    return 0;
}

/* Brute force for tiny cases of Sec. IV, Listing 1, whose bilinear
 * interpolation with zero outside the detector is, written as a sum over
 * every pixel, f(X) = sum_k sum_{m,n} I_k[n,m] tent(u-m)
 * tent(v-n) / w^2 with tent(t) = max(0, 1-|t|), evaluated over every pixel.
 * No floor, no cell, no bounds branches: a different route to the same
 * bilinear, zero-extended interpolation. */
int oracle_bruteforce(double *vol, const int64_t dims[3], const double voxel_size[3],
                      const double origin[3], const float *proj, int64_t W, int64_t H,
                      const float *mats, int64_t n_views)
{
    if (check_geom(dims, W, H, n_views)) return -1;
    for (int64_t z = 0; z < dims[2]; ++z)
        for (int64_t y = 0; y < dims[1]; ++y)
            for (int64_t x = 0; x < dims[0]; ++x) {
                double X = origin[0] + (double)x * voxel_size[0];
                double Y = origin[1] + (double)y * voxel_size[1];
                double Z = origin[2] + (double)z * voxel_size[2];
                double acc = 0.0;
                for (int64_t k = 0; k < n_views; ++k) {
                    const float *A = mats + 12 * k;
                    double w = A[8] * X + A[9] * Y + A[10] * Z + A[11];
                    if (!(w > 0.0)) continue;
                    double u = (A[0] * X + A[1] * Y + A[2] * Z + A[3]) / w;
                    double v = (A[4] * X + A[5] * Y + A[6] * Z + A[7]) / w;
                    double s = 0.0;
                    for (int64_t n = 0; n < H; ++n) {
                        double tv = 1.0 - fabs(v - (double)n);
                        if (tv <= 0.0) continue;
                        for (int64_t m = 0; m < W; ++m) {
                            double tu = 1.0 - fabs(u - (double)m);
                            if (tu <= 0.0) continue;
                            s += (double)proj[(k * H + n) * W + m] * tu * tv;
                        }
                    }
                    acc += s / (w * w);
                }
                vol[(z * dims[1] + y) * dims[0] + x] += acc;
            }
    return 0;
}

/*
 * FDK pre-processing (the step before the back-projection; the paper's data
 * arrives pre-filtered, Sec. IV): cosine pre-weighting and Ram-Lak filtering
 * of every detector row, in FP64.
 *
 * The camera of view k is read off its matrix P = s K [R | t] with
 * K = [[f, 0, u0], [0, f, v0], [0, 0, 1]] (square pixels, no skew): with
 * M = P[:, 0:3], M M^T = s^2 K K^T, so s^2 = (M M^T)[2][2],
 * u0 = (M M^T)[0][2] / s^2, v0 = (M M^T)[1][2] / s^2 and
 * f^2 = (M M^T)[0][0] / s^2 - u0^2.  The cosine of the angle between the ray
 * through pixel (m, n) and the principal axis is f / sqrt(f^2 + (m-u0)^2 +
 * (n-v0)^2).  The row filter is the discrete Ram-Lak kernel in pixel units,
 * h(0) = 1/4, h(d) = -1 / (pi^2 d^2) for odd d, 0 for even d != 0, applied
 * as a linear convolution over the row (zero outside it):
 *   out[k][n][m] = scale * sum_{m'} h(m - m') cos_k(m', n) in[k][n][m'].
 */
int oracle_camera(const float *mats, int64_t n_views, double *f_u0_v0)
{
    for (int64_t k = 0; k < n_views; ++k) {
        const float *P = mats + 12 * k;
        double G[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                G[a][b] = 0.0;
                for (int c = 0; c < 3; ++c) G[a][b] += (double)P[4 * a + c] * (double)P[4 * b + c];
            }
        const double s2 = G[2][2];
        if (!(s2 > 0.0)) return -1;
        const double u0 = G[0][2] / s2, v0 = G[1][2] / s2;
        const double f2 = G[0][0] / s2 - u0 * u0;
        if (!(f2 > 0.0)) return -1;
        f_u0_v0[3 * k + 0] = sqrt(f2);
        f_u0_v0[3 * k + 1] = u0;
        f_u0_v0[3 * k + 2] = v0;
    }
    return 0;
}

int oracle_preweight_filter(double *out, const float *proj, int64_t W, int64_t H,
                            const float *mats, int64_t n_views, double scale)
{
    if (W <= 0 || H <= 0 || n_views < 0) return -1;
    double *cam = (double *)malloc(sizeof(double) * 3 * (size_t)(n_views > 0 ? n_views : 1));
    double *h = (double *)malloc(sizeof(double) * (size_t)W);
    double *g = (double *)malloc(sizeof(double) * (size_t)W);
    if (!cam || !h || !g) { free(cam); free(h); free(g); return -2; }
    if (oracle_camera(mats, n_views, cam)) { free(cam); free(h); free(g); return -1; }
    const double pi = 3.14159265358979323846;
    for (int64_t d = 0; d < W; ++d)
        h[d] = (d == 0) ? 0.25 : ((d % 2) ? -1.0 / (pi * pi * (double)d * (double)d) : 0.0);
    for (int64_t k = 0; k < n_views; ++k) {
        const double f = cam[3 * k], u0 = cam[3 * k + 1], v0 = cam[3 * k + 2];
        for (int64_t n = 0; n < H; ++n) {
            const float *row = proj + (k * H + n) * W;
            for (int64_t m = 0; m < W; ++m) {
                const double du = (double)m - u0, dv = (double)n - v0;
                g[m] = (double)row[m] * f / sqrt(f * f + du * du + dv * dv);
            }
            double *o = out + (k * H + n) * W;
            for (int64_t m = 0; m < W; ++m) {
                double acc = 0.0;
                for (int64_t mp = 0; mp < W; ++mp) {
                    const int64_t d = m > mp ? m - mp : mp - m;
                    acc += h[d] * g[mp];
                }
                o[m] = scale * acc;
            }
        }
    }
    free(cam);
    free(h);
    free(g);
    return 0;
}

/* The clipped update count (the basis of the paper's GUp/s figures,
 * Sec. VII): the (voxel, view) pairs with w > 0, -1 < u < W and -1 < v < H,
 * the pairs that can touch the detector under the bilinear taps with zero
 * outside.  Also counted, in *band, are the pairs that sit within eps of one
 * of those decisions (|w| <= eps_w, or u or v within eps pixels of -1, W or
 * H while w > 0): an evaluation in lower precision may decide those either
 * way, and no other pair.  Threads split (z, y) lines; the counts are exact
 * integers, so the split does not change them. */
typedef struct {
    const float *mats;
    int64_t nx, ny, W, H, n_views;
    double vs[3], org[3], eps, eps_w;
    int64_t line_begin, line_end;
    int64_t count, band;
} count_job;

static void *count_worker(void *arg)
{
    count_job *jb = (count_job *)arg;
    int64_t count = 0, band = 0;
    const double Wd = (double)jb->W, Hd = (double)jb->H, e = jb->eps;
    for (int64_t k = 0; k < jb->n_views; ++k) {
        double P[12];
        for (int q = 0; q < 12; ++q) P[q] = (double)jb->mats[k * 12 + q];
        for (int64_t line = jb->line_begin; line < jb->line_end; ++line) {
            int64_t z = line / jb->ny, y = line % jb->ny;
            double Z = jb->org[2] + (double)z * jb->vs[2];
            double Y = jb->org[1] + (double)y * jb->vs[1];
            for (int64_t x = 0; x < jb->nx; ++x) {
                double X = jb->org[0] + (double)x * jb->vs[0];
                double w = P[8] * X + P[9] * Y + P[10] * Z + P[11];
                if (fabs(w) <= jb->eps_w) { ++band; continue; }
                if (!(w > 0.0)) continue;
                double u = (P[0] * X + P[1] * Y + P[2] * Z + P[3]) / w;
                double v = (P[4] * X + P[5] * Y + P[6] * Z + P[7]) / w;
                if (u > -1.0 && u < Wd && v > -1.0 && v < Hd) ++count;
                if (fabs(u + 1.0) <= e || fabs(u - Wd) <= e || fabs(v + 1.0) <= e || fabs(v - Hd) <= e) ++band;
            }
        }
    }
    jb->count = count;
    jb->band = band;
    return NULL;
}

int oracle_count_updates(int64_t *count, int64_t *band, const int64_t dims[3], const double voxel_size[3],
                         const double origin[3], int64_t W, int64_t H, const float *mats, int64_t n_views,
                         double eps, double eps_w, int nthreads)
{
    if (!count || !band || check_geom(dims, W, H, n_views)) return -1;
    *count = 0;
    *band = 0;
    int64_t lines = dims[1] * dims[2];
    if (lines == 0 || dims[0] == 0 || n_views == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ORACLE_MAX_THREADS) nthreads = ORACLE_MAX_THREADS;
    if (nthreads > lines) nthreads = (int)lines;
    count_job *jobs = (count_job *)calloc((size_t)nthreads, sizeof(count_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    for (int t = 0; t < nthreads; ++t) {
        count_job *jb = &jobs[t];
        jb->mats = mats;
        jb->nx = dims[0]; jb->ny = dims[1];
        jb->W = W; jb->H = H; jb->n_views = n_views;
        for (int q = 0; q < 3; ++q) { jb->vs[q] = voxel_size[q]; jb->org[q] = origin[q]; }
        jb->eps = eps;
        jb->eps_w = eps_w;
        jb->line_begin = lines * t / nthreads;
        jb->line_end = lines * (t + 1) / nthreads;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, count_worker, &jobs[t]) != 0) break;
        started = t;
    }
    count_worker(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    for (int t = started + 1; t < nthreads; ++t) count_worker(&jobs[t]);
    for (int t = 0; t < nthreads; ++t) {
        *count += jobs[t].count;
        *band += jobs[t].band;
    }
    free(jobs);
    free(th);
    return 0;
}
