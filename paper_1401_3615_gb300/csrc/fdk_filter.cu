// FDK pre-processing on the device: cosine pre-weighting and Ram-Lak row
// filtering (the data of the paper arrives in this form, Sec. IV).
//
//   out[k][n][m] = scale * sum_{m'} h(m - m') c_k(m', n) in[k][n][m']
//   h(0) = 1/4, h(d) = -1/(pi^2 d^2) for odd d, 0 for even d != 0
//   c_k(m, n) = f / sqrt(f^2 + (m - u0)^2 + (n - v0)^2)
//
// with (f, u0, v0) read off view k's matrix through M M^T (square pixels, no
// skew).  The linear convolution along a row is evaluated as a circular one
// of length N >= 2W (so every lag |m - m'| < W is within N/2 and nothing
// wraps): N = 2560 for rows of 1025..1280 pixels, else 2^ceil(log2(2W)).
// Two rows are packed as the real and imaginary parts of one complex signal,
// transformed by a Stockham FFT, multiplied by the kernel's spectrum (real,
// since h is even) and transformed back: for N = 2560 radix-10 and radix-16
// passes, for N = 4096 three radix-16 passes, with the points in registers;
// otherwise radix-4 passes in shared memory.
#include <math.h>

#include "fdk_internal.cuh"

namespace fdk {

// Spectrum of the circularly laid-out kernel: H[k] = h(0) + 2 sum_{odd d < N/2}
// h(d) cos(2 pi k d / N), times 1/N (the inverse transform's normalisation).
__global__ void fdk_ramlak_spectrum_kernel(float *spec, int N)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const float inv_pi2 = 0.10132118364233778f;   // 1 / pi^2
    float s = 0.25f, comp = 0.0f;                  // Kahan-compensated sum
    for (int d = 1; d < N / 2; d += 2) {
        // cos(2 pi k d / N) with the argument reduced exactly in integers
        const long long num = (2LL * k * d) % (2LL * N);
        const float t = -2.0f * inv_pi2 / ((float)d * (float)d) * cospif((float)num / (float)N);
        const float y = t - comp;
        const float z = s + y;
        comp = (z - s) - y;
        s = z;
    }
    spec[k] = s / (float)N;
}

// Twiddle table tw[t] = exp(-2 pi i t / N), t < N.
__global__ void fdk_twiddle_kernel(float2 *tw, int N)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    float sv, cv;
    // 2t/N is exact for N a power of two, and rounded to half an ulp for
    // N = 2560 (twiddles within about 2e-7)
    sincospif(2.0f * (float)t / (float)N, &sv, &cv);
    tw[t] = make_float2(cv, -sv);
}

struct FilterArgs {
    float *out;
    const float *in;
    const float *spec;      // N spectrum values (1/N folded in)
    const float2 *tw;       // N twiddles exp(-2 pi i t / N) (the N = 4096 kernel)
    unsigned *err;          // device word set when a bounded wait gives up (staged rows)
    long long wait_limit;   // polls before the wait for a staged row pair gives up
    float scale;
    const float *mats_dev;  // device matrices, or nullptr
    int W, H, n_views, N;
    float mats[KMAX * 12];  // host matrices of this pass
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One N-point transform (radix-4 Stockham passes, one radix-2 pass first
// when log2 N is odd), src -> (ping-pong) -> result pointer returned.
// Forward uses tw[t] = exp(-2 pi i t / N), t < 3N/4; inverse its conjugate.
template <int NT>
__device__ float2 *stockham(float2 *src, float2 *dst, const float2 *tw, int N, bool inverse)
{
    int Ns = 1;
    if (!(__ffs(N) & 1)) {   // log2 N = ffs - 1 odd: one radix-2 pass, no twiddles
        for (int j = threadIdx.x; j < N / 2; j += NT) {
            const float2 u = src[j], v = src[j + N / 2];
            dst[2 * j] = make_float2(u.x + v.x, u.y + v.y);
            dst[2 * j + 1] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
        float2 *t = src;
        src = dst;
        dst = t;
        Ns = 2;
    }
    const float sg = inverse ? -1.0f : 1.0f;
    for (; Ns < N; Ns <<= 2) {
        const int tstep = N / (4 * Ns);
        for (int j = threadIdx.x; j < N / 4; j += NT) {
            const int k = j & (Ns - 1);
            float2 w1 = tw[k * tstep], w2 = tw[2 * k * tstep], w3 = tw[3 * k * tstep];
            w1.y *= sg;
            w2.y *= sg;
            w3.y *= sg;
            const float2 a0 = src[j];
            const float2 a1 = cmul(src[j + N / 4], w1);
            const float2 a2 = cmul(src[j + N / 2], w2);
            const float2 a3 = cmul(src[j + 3 * N / 4], w3);
            // 4-point DFT: y_q = sum_m a_m (-i sg)^(m q)
            const float2 s02 = make_float2(a0.x + a2.x, a0.y + a2.y);
            const float2 d02 = make_float2(a0.x - a2.x, a0.y - a2.y);
            const float2 s13 = make_float2(a1.x + a3.x, a1.y + a3.y);
            const float2 d13 = make_float2(a1.x - a3.x, a1.y - a3.y);
            // -i sg * d13 = (sg * d13.y, -sg * d13.x)
            const float2 r = make_float2(sg * d13.y, -sg * d13.x);
            const int base = ((j - k) << 2) + k;
            dst[base] = make_float2(s02.x + s13.x, s02.y + s13.y);
            dst[base + Ns] = make_float2(d02.x + r.x, d02.y + r.y);
            dst[base + 2 * Ns] = make_float2(s02.x - s13.x, s02.y - s13.y);
            dst[base + 3 * Ns] = make_float2(d02.x - r.x, d02.y - r.y);
        }
        __syncthreads();
        float2 *t = src;
        src = dst;
        dst = t;
    }
    return src;
}

template <int NT>
__global__ void __launch_bounds__(NT)
fdk_filter_kernel(const __grid_constant__ FilterArgs a)
{
    extern __shared__ float2 sm[];
    const int N = a.N;
    float2 *b0 = sm, *b1 = sm + N, *tw = sm + 2 * N;
    for (int t = threadIdx.x; t < 3 * N / 4; t += NT) {
        float s, c;
        sincospif(-2.0f * (float)t / (float)N, &s, &c);
        tw[t] = make_float2(c, s);
    }
    __syncthreads();
    const int pairs = (a.H + 1) / 2;
    const long long total = (long long)pairs * a.n_views;
    for (long long rp = blockIdx.x; rp < total; rp += gridDim.x) {
        const int k = (int)(rp / pairs), p = (int)(rp % pairs);
        const int r1 = 2 * p, r2 = 2 * p + 1;
        // camera of view k from M M^T
        float P[9];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                P[3 * q + c] = a.mats_dev ? __ldg(a.mats_dev + 12 * k + 4 * q + c) : a.mats[12 * k + 4 * q + c];
        const float s2 = P[6] * P[6] + P[7] * P[7] + P[8] * P[8];
        const float u0 = (P[0] * P[6] + P[1] * P[7] + P[2] * P[8]) / s2;
        const float v0 = (P[3] * P[6] + P[4] * P[7] + P[5] * P[8]) / s2;
        const float f2 = (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / s2 - u0 * u0;
        const float f = sqrtf(f2);
        const float *row1 = a.in + ((long long)k * a.H + r1) * a.W;
        const float *row2 = a.in + ((long long)k * a.H + r2) * a.W;
        const float dv1 = (float)r1 - v0, dv2 = (float)r2 - v0;
        for (int m = threadIdx.x; m < N; m += NT) {
            float x = 0.0f, y = 0.0f;
            if (m < a.W) {
                const float du = (float)m - u0;
                x = row1[m] * f * rsqrtf(f2 + du * du + dv1 * dv1);
                if (r2 < a.H) y = row2[m] * f * rsqrtf(f2 + du * du + dv2 * dv2);
            }
            b0[m] = make_float2(x, y);
        }
        __syncthreads();
        float2 *X = stockham<NT>(b0, b1, tw, N, false);
        float2 *Y = (X == b0) ? b1 : b0;
        for (int m = threadIdx.x; m < N; m += NT) {
            const float h = __ldg(a.spec + m) * a.scale;
            X[m] = make_float2(X[m].x * h, X[m].y * h);
        }
        __syncthreads();
        float2 *R = stockham<NT>(X, Y, tw, N, true);
        float *o1 = a.out + ((long long)k * a.H + r1) * a.W;
        float *o2 = a.out + ((long long)k * a.H + r2) * a.W;
        for (int m = threadIdx.x; m < a.W; m += NT) {
            const float2 v = R[m];
            o1[m] = v.x;
            if (r2 < a.H) o2[m] = v.y;
        }
        __syncthreads();   // before the next pair overwrites the buffers
    }
}

// ---------------------------------------------------------------------------
// N = 4096 = 16^3 (detector rows of 1025..2048 pixels): three radix-16
// Stockham passes per transform with the 16 points of each thread in
// registers.  Pass p (stride Ns = 16^p) takes a_m = in[j + 256 m] times
// exp(-+2 pi i m (j mod Ns) / (16 Ns)), forms their 16-point DFT y_q and
// stores it at (j - j mod Ns) 16 + j mod Ns + q Ns.  The first pass reads
// the weighted rows straight from global memory, and the last forward pass
// leaves thread j holding X[j + 256 q] -- exactly the inputs of the first
// inverse pass -- so the spectrum multiply happens in registers; the last
// inverse pass leaves result[j + 256 q] for the coalesced row stores.  Four
// shared-memory exchanges per row pair, padded one float2 per 16 so every
// exchange runs at the minimum of two wavefronts per warp access.
constexpr int kF16N = 4096;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// In-place 4-point DFT; INV uses exp(+2 pi i nk/4).
template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
    // forward: -i d13; inverse: +i d13
    const float2 r = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
    a0 = cadd(s02, s13);
    a1 = cadd(d02, r);
    a2 = csub(s02, s13);
    a3 = csub(d02, r);
}

// x[n] -> x[q] = sum_n x[n] exp(-+2 pi i n q / 16), as 4 x 4 with n = 4 n1 + n2,
// q = k1 + 4 k2 and the twiddles exp(-+2 pi i n2 k1 / 16) in between.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&x)[16])
{
    // cos and sin of 2 pi j / 16 for the twiddle exponents j = n2 k1
    constexpr float C1 = 0.92387953251128676f, S1 = 0.38268343236508977f, H = 0.70710678118654752f;
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
    // x[4 k1 + n2] now holds the n2-th inner DFT at k1
    const float sg = INV ? 1.0f : -1.0f;
    const float2 w1 = make_float2(C1, sg * S1), w2 = make_float2(H, sg * H), w3 = make_float2(S1, sg * C1);
    const float2 w6 = make_float2(-H, sg * H), w9 = make_float2(-C1, -sg * S1);
    x[5] = cmul(x[5], w1);
    x[6] = cmul(x[6], w2);
    x[7] = cmul(x[7], w3);
    x[9] = cmul(x[9], w2);
    x[10] = make_float2(-sg * x[10].y, sg * x[10].x);   // times exp(-+i pi/2)
    x[11] = cmul(x[11], w6);
    x[13] = cmul(x[13], w3);
    x[14] = cmul(x[14], w6);
    x[15] = cmul(x[15], w9);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
    // x[4 k1 + k2] holds X[k1 + 4 k2]: transpose into natural order
    float2 y[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) y[q] = x[4 * (q & 3) + (q >> 2)];
#pragma unroll
    for (int q = 0; q < 16; ++q) x[q] = y[q];
}

// Pass with stride Ns (16 or 256) reading from the shared buffer.  The
// twiddles w^m, w = exp(-+2 pi i kk tstep / N), come from four table values
// (w, w^2, w^4, w^8) and at most two products each.
template <bool INV>
__device__ __forceinline__ void pass_in(float2 (&x)[16], const float2 *buf, const float2 *__restrict__ tw,
                                        int j, int kk, int tstep)
{
#pragma unroll
    for (int m = 0; m < 16; ++m) x[m] = buf[pad16(j + 256 * m)];
    const int t1 = kk * tstep;
    float2 w1 = __ldg(tw + t1), w2 = __ldg(tw + 2 * t1), w4 = __ldg(tw + 4 * t1), w8 = __ldg(tw + 8 * t1);
    if (INV) {
        w1.y = -w1.y;
        w2.y = -w2.y;
        w4.y = -w4.y;
        w8.y = -w8.y;
    }
    const float2 w3 = cmul(w1, w2);
    x[1] = cmul(x[1], w1);
    x[2] = cmul(x[2], w2);
    x[3] = cmul(x[3], w3);
    x[4] = cmul(x[4], w4);
    x[5] = cmul(x[5], cmul(w4, w1));
    x[6] = cmul(x[6], cmul(w4, w2));
    x[7] = cmul(x[7], cmul(w4, w3));
    x[8] = cmul(x[8], w8);
    x[9] = cmul(x[9], cmul(w8, w1));
    x[10] = cmul(x[10], cmul(w8, w2));
    x[11] = cmul(x[11], cmul(w8, w3));
    const float2 w12 = cmul(w8, w4);
    x[12] = cmul(x[12], w12);
    x[13] = cmul(x[13], cmul(w12, w1));
    x[14] = cmul(x[14], cmul(w12, w2));
    x[15] = cmul(x[15], cmul(w12, w3));
    dft16<INV>(x);
}

__device__ __forceinline__ uint32_t fsmem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bounded wait for the phase with the given parity of the mbarrier at bar:
// at most `limit` polls.
__device__ __forceinline__ bool fmbar_wait(uint32_t bar, uint32_t parity, long long limit)
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

// Copy the rows of row pair rp into a stage (rows rowoff floats apart) with
// bulk copies completing on the mbarrier at bar.  Called by one thread.
__device__ __forceinline__ void filter_issue(const FilterArgs &a, long long rp, int pairs, float *stage,
                                             uint32_t bar, int rowoff = kF16N / 2)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // after the stage's last reads
    const int k = (int)(rp / pairs), p = (int)(rp % pairs);
    const int r1 = 2 * p, r2 = 2 * p + 1;
    const uint32_t rowbytes = (uint32_t)a.W * 4u;
    const uint32_t bytes = r2 < a.H ? 2u * rowbytes : rowbytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
    const float *row1 = a.in + ((long long)k * a.H + r1) * a.W;
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(fsmem(stage)), "l"(row1), "r"(rowbytes), "r"(bar) : "memory");
    if (r2 < a.H)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(fsmem(stage + rowoff)), "l"(row1 + a.W), "r"(rowbytes), "r"(bar) : "memory");
}

// STAGED: the rows (W % 4 == 0, 16-byte aligned) of the row pair after next
// are copied into one of two shared-memory stages while this one is
// transformed, so the first pass reads its inputs from shared memory.
template <bool STAGED>
__global__ void __launch_bounds__(256, 2)
fdk_filter4096_kernel(const __grid_constant__ FilterArgs a)
{
    extern __shared__ __align__(128) float2 fsm[];
    float2 *buf = fsm;                                               // padded transform buffer
    float *stages = reinterpret_cast<float *>(fsm + kF16N + kF16N / 16);   // 2 x (2 rows of 2048)
    __shared__ __align__(8) unsigned long long full[2];
    const int j = threadIdx.x;
    const int pairs = (a.H + 1) / 2;
    const long long total = (long long)pairs * a.n_views;
    const long long stride = gridDim.x;
    const uint32_t full0 = fsmem(full);
    unsigned nis[2] = {0u, 0u};   // copies issued into each stage (thread 0)
    if (STAGED) {
        if (j == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(full0) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(full0 + 8u) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (j == 0) {
            for (int q = 0; q < 2; ++q) {
                const long long rq = blockIdx.x + q * stride;
                if (rq < total) {
                    filter_issue(a, rq, pairs, stages + q * kF16N, full0 + 8u * q);
                    ++nis[q];
                }
            }
        }
    }
    int it = 0;
    for (long long rp = blockIdx.x; rp < total; rp += stride, ++it) {
        const int k = (int)(rp / pairs), p = (int)(rp % pairs);
        const int r1 = 2 * p, r2 = 2 * p + 1;
        // camera of view k from M M^T
        float P[9];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                P[3 * q + c] = a.mats_dev ? __ldg(a.mats_dev + 12 * k + 4 * q + c) : a.mats[12 * k + 4 * q + c];
        const float s2 = P[6] * P[6] + P[7] * P[7] + P[8] * P[8];
        const float u0 = (P[0] * P[6] + P[1] * P[7] + P[2] * P[8]) / s2;
        const float v0 = (P[3] * P[6] + P[4] * P[7] + P[5] * P[8]) / s2;
        const float f2v = (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / s2 - u0 * u0;
        const float f = sqrtf(f2v);
        const float *row1, *row2;
        const int st = it & 1;
        bool ok = true;
        if (STAGED) {
            row1 = stages + st * kF16N;
            row2 = row1 + kF16N / 2;
            ok = fmbar_wait(full0 + 8u * st, (unsigned)(it >> 1) & 1u, a.wait_limit);
        } else {
            row1 = a.in + ((long long)k * a.H + r1) * a.W;
            row2 = a.in + ((long long)k * a.H + r2) * a.W;
        }
        const float dv1 = (float)r1 - v0, dv2 = (float)r2 - v0;
        const bool has2 = r2 < a.H;

        float2 x[16];
        // forward pass 1 (Ns = 1) from the weighted rows, zero past the row
        // (W <= 2048 = N / 2, so points 2048.. are zero padding)
#pragma unroll
        for (int m = 8; m < 16; ++m) x[m] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int col = j + 256 * m;
            float vx = 0.0f, vy = 0.0f;
            if (col < a.W) {
                const float du = (float)col - u0;
                vx = row1[col] * f * rsqrtf(f2v + du * du + dv1 * dv1);
                if (has2) vy = row2[col] * f * rsqrtf(f2v + du * du + dv2 * dv2);
            }
            x[m] = make_float2(vx, vy);
        }
        dft16<false>(x);
        // the previous row pair's last reads of buf, and this one's reads of
        // its stage, are done
        if (STAGED) {
            if (!__syncthreads_and(ok)) {
                if (j == 0) {
                    atomicOr(a.err, 1u);
                    // drain with the full limit: no copy may still be
                    // writing this CTA's shared memory when it exits
                    for (int q = 0; q < 2; ++q)
                        if (nis[q] > 0) fmbar_wait(full0 + 8u * q, (nis[q] - 1) & 1u, kWaitLimit);
                }
                return;
            }
            if (j == 0 && rp + 2 * stride < total) {
                filter_issue(a, rp + 2 * stride, pairs, stages + st * kF16N, full0 + 8u * st);
                ++nis[st];
            }
        } else {
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) buf[pad16(16 * j + q)] = x[q];
        __syncthreads();
        // forward pass 2 (Ns = 16)
        pass_in<false>(x, buf, a.tw, j, j & 15, 16);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) buf[pad16((j & ~15) * 16 + (j & 15) + 16 * q)] = x[q];
        __syncthreads();
        // forward pass 3 (Ns = 256): thread j ends with X[j + 256 q]
        pass_in<false>(x, buf, a.tw, j, j, 1);
        // the kernel's spectrum (real, 1/N folded in) and the caller's scale
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float hq = __ldg(a.spec + j + 256 * q) * a.scale;
            x[q] = make_float2(x[q].x * hq, x[q].y * hq);
        }
        // inverse pass 1 (Ns = 1) on the registers
        dft16<true>(x);
        __syncthreads();   // everyone's pass-3 reads are done
#pragma unroll
        for (int q = 0; q < 16; ++q) buf[pad16(16 * j + q)] = x[q];
        __syncthreads();
        pass_in<true>(x, buf, a.tw, j, j & 15, 16);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) buf[pad16((j & ~15) * 16 + (j & 15) + 16 * q)] = x[q];
        __syncthreads();
        // inverse pass 3: thread j ends with result[j + 256 q]
        pass_in<true>(x, buf, a.tw, j, j, 1);
        float *o1 = a.out + ((long long)k * a.H + r1) * a.W;
        float *o2 = a.out + ((long long)k * a.H + r2) * a.W;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int col = j + 256 * q;
            if (col < a.W) {
                o1[col] = x[q].x;
                if (has2) o2[col] = x[q].y;
            }
        }
    }
}

// N = 2560 (rows of 1025..1280 pixels, where the power-of-two length would
// be 4096): 2560 = 10 x 16 x 16, about 60% of the 4096-point work.  Stockham
// passes as in the 4096-point kernel -- the pass with radix R and stride Ns
// has butterfly j read x[j + (N / R) m], scale it by w^m with
// w = exp(-+2 pi i (j mod Ns) / (Ns R)), transform, and write output q to
// (j - j mod Ns) R + j mod Ns + q Ns -- with radices 10, 16, 16 forward
// (strides 1, 10, 160) and 16, 16, 10 inverse (strides 1, 16, 256).  A CTA
// has 160 threads, one per butterfly of the radix-16 passes; the radix-10
// passes' 256 butterflies are j and j + 160.  (With 256 threads, three
// warps idled through the radix-16 passes: 14% slower.)  The last forward
// pass leaves thread j with X[j + 160 q], the inputs of the first inverse
// pass, so the spectrum multiply happens in registers; the last inverse
// pass leaves result[j + 256 q].  The first exchange is unpadded (writes at stride 10:
// two wavefronts per half-warp, reads conflict-free); the others are padded
// one float2 per 16 (conflict-free both ways).
constexpr int kF25N = 2560;

// 5-point DFT, exp(-+2 pi i nk / 5).
template <bool INV>
__device__ __forceinline__ void dft5(float2 &x0, float2 &x1, float2 &x2, float2 &x3, float2 &x4)
{
    // cos and sin of 2 pi / 5 and 4 pi / 5
    constexpr float C1 = 0.30901699437494742f, C2 = -0.80901699437494742f;
    constexpr float S1 = 0.95105651629515357f, S2 = 0.58778525229247313f;
    const float2 t1 = cadd(x1, x4), t2 = cadd(x2, x3), t3 = csub(x1, x4), t4 = csub(x2, x3);
    const float2 b1 = make_float2(x0.x + C1 * t1.x + C2 * t2.x, x0.y + C1 * t1.y + C2 * t2.y);
    const float2 b2 = make_float2(x0.x + C2 * t1.x + C1 * t2.x, x0.y + C2 * t1.y + C1 * t2.y);
    const float2 d1 = make_float2(S1 * t3.x + S2 * t4.x, S1 * t3.y + S2 * t4.y);
    const float2 d2 = make_float2(S2 * t3.x - S1 * t4.x, S2 * t3.y - S1 * t4.y);
    x0 = cadd(x0, cadd(t1, t2));
    // forward: X1 = b1 - i d1, X4 = b1 + i d1, X2 = b2 - i d2, X3 = b2 + i d2
    const float2 e1 = INV ? make_float2(-d1.y, d1.x) : make_float2(d1.y, -d1.x);   // -+ i d1
    const float2 e2 = INV ? make_float2(-d2.y, d2.x) : make_float2(d2.y, -d2.x);
    x1 = cadd(b1, e1);
    x4 = csub(b1, e1);
    x2 = cadd(b2, e2);
    x3 = csub(b2, e2);
}

// 10-point DFT as 2 x 5: the pairs (x[n2], x[n2 + 5]), the twiddles
// exp(-+2 pi i n2 k1 / 10), then 5-point DFTs over n2 giving X[k1 + 2 k2];
// the result in natural order.
template <bool INV>
__device__ __forceinline__ void dft10(float2 (&x)[10])
{
    // cos and sin of pi j / 5, j = 1..4
    constexpr float CA = 0.80901699437494742f, SA = 0.58778525229247313f;
    constexpr float CB = 0.30901699437494742f, SB = 0.95105651629515357f;
    const float sg = INV ? 1.0f : -1.0f;
    float2 a[5], b[5];
#pragma unroll
    for (int n = 0; n < 5; ++n) {
        a[n] = cadd(x[n], x[n + 5]);
        b[n] = csub(x[n], x[n + 5]);
    }
    b[1] = cmul(b[1], make_float2(CA, sg * SA));
    b[2] = cmul(b[2], make_float2(CB, sg * SB));
    b[3] = cmul(b[3], make_float2(-CB, sg * SB));
    b[4] = cmul(b[4], make_float2(-CA, sg * SA));
    dft5<INV>(a[0], a[1], a[2], a[3], a[4]);
    dft5<INV>(b[0], b[1], b[2], b[3], b[4]);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        x[2 * k] = a[k];
        x[2 * k + 1] = b[k];
    }
}

// Scale x[m] by w^m, w = tw[t1] (conjugated for the inverse), from the table
// values w, w^2, w^4, w^8 and products, for m < R.
template <int R, bool INV>
__device__ __forceinline__ void twiddle_by(float2 (&x)[R], const float2 *__restrict__ tw, int t1)
{
    float2 w1 = __ldg(tw + t1), w2 = __ldg(tw + 2 * t1), w4 = __ldg(tw + 4 * t1), w8 = __ldg(tw + 8 * t1);
    if (INV) {
        w1.y = -w1.y;
        w2.y = -w2.y;
        w4.y = -w4.y;
        w8.y = -w8.y;
    }
    const float2 w3 = cmul(w1, w2);
    x[1] = cmul(x[1], w1);
    x[2] = cmul(x[2], w2);
    x[3] = cmul(x[3], w3);
    x[4] = cmul(x[4], w4);
    x[5] = cmul(x[5], cmul(w4, w1));
    x[6] = cmul(x[6], cmul(w4, w2));
    x[7] = cmul(x[7], cmul(w4, w3));
    x[8] = cmul(x[8], w8);
    x[9] = cmul(x[9], cmul(w8, w1));
    if constexpr (R == 16) {
        x[10] = cmul(x[10], cmul(w8, w2));
        x[11] = cmul(x[11], cmul(w8, w3));
        const float2 w12 = cmul(w8, w4);
        x[12] = cmul(x[12], w12);
        x[13] = cmul(x[13], cmul(w12, w1));
        x[14] = cmul(x[14], cmul(w12, w2));
        x[15] = cmul(x[15], cmul(w12, w3));
    }
}

template <bool STAGED>
__global__ void __launch_bounds__(160, 3)
fdk_filter2560_kernel(const __grid_constant__ FilterArgs a)
{
    constexpr int N = kF25N, ROW = N / 2;
    extern __shared__ __align__(128) float2 fsm[];
    float2 *buf = fsm;                                             // N + N / 16 float2
    float *stages = reinterpret_cast<float *>(fsm + N + N / 16);   // 2 x (2 rows of ROW)
    __shared__ __align__(8) unsigned long long full[2];
    const int j = threadIdx.x;
    const int pairs = (a.H + 1) / 2;
    const long long total = (long long)pairs * a.n_views;
    const long long stride = gridDim.x;
    const uint32_t full0 = fsmem(full);
    unsigned nis[2] = {0u, 0u};   // copies issued into each stage (thread 0)
    if (STAGED) {
        if (j == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(full0) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(full0 + 8u) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (j == 0) {
            for (int q = 0; q < 2; ++q) {
                const long long rq = blockIdx.x + q * stride;
                if (rq < total) {
                    filter_issue(a, rq, pairs, stages + q * N, full0 + 8u * q, ROW);
                    ++nis[q];
                }
            }
        }
    }
    int it = 0;
    for (long long rp = blockIdx.x; rp < total; rp += stride, ++it) {
        const int k = (int)(rp / pairs), p = (int)(rp % pairs);
        const int r1 = 2 * p, r2 = 2 * p + 1;
        // camera of view k from M M^T
        float P[9];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                P[3 * q + c] = a.mats_dev ? __ldg(a.mats_dev + 12 * k + 4 * q + c) : a.mats[12 * k + 4 * q + c];
        const float s2 = P[6] * P[6] + P[7] * P[7] + P[8] * P[8];
        const float u0 = (P[0] * P[6] + P[1] * P[7] + P[2] * P[8]) / s2;
        const float v0 = (P[3] * P[6] + P[4] * P[7] + P[5] * P[8]) / s2;
        const float f2v = (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / s2 - u0 * u0;
        const float f = sqrtf(f2v);
        const float *row1, *row2;
        const int st = it & 1;
        bool ok = true;
        if (STAGED) {
            row1 = stages + st * N;
            row2 = row1 + ROW;
            ok = fmbar_wait(full0 + 8u * st, (unsigned)(it >> 1) & 1u, a.wait_limit);
        } else {
            row1 = a.in + ((long long)k * a.H + r1) * a.W;
            row2 = a.in + ((long long)k * a.H + r2) * a.W;
        }
        const float dv1 = (float)r1 - v0, dv2 = (float)r2 - v0;
        const bool has2 = r2 < a.H;

        // forward pass 1 (radix 10, Ns = 1) from the weighted rows, zero past
        // the row (W <= 1280 = N / 2, so points 1280.. are zero padding);
        // butterflies j and j + 160 (< 256)
        float2 y[10], y2[10];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jb = j + 160 * h;
            float2 (&yy)[10] = h ? y2 : y;
#pragma unroll
            for (int m = 5; m < 10; ++m) yy[m] = make_float2(0.0f, 0.0f);
            if (jb < 256) {
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    const int col = jb + 256 * m;
                    float vx = 0.0f, vy = 0.0f;
                    if (col < a.W) {
                        const float du = (float)col - u0;
                        vx = row1[col] * f * rsqrtf(f2v + du * du + dv1 * dv1);
                        if (has2) vy = row2[col] * f * rsqrtf(f2v + du * du + dv2 * dv2);
                    }
                    yy[m] = make_float2(vx, vy);
                }
                dft10<false>(yy);
            }
        }
        // the previous row pair's last reads of buf, and this one's reads of
        // its stage, are done
        if (STAGED) {
            if (!__syncthreads_and(ok)) {
                if (j == 0) {
                    atomicOr(a.err, 1u);
                    // drain with the full limit: no copy may still be
                    // writing this CTA's shared memory when it exits
                    for (int q = 0; q < 2; ++q)
                        if (nis[q] > 0) fmbar_wait(full0 + 8u * q, (nis[q] - 1) & 1u, kWaitLimit);
                }
                return;
            }
            if (j == 0 && rp + 2 * stride < total) {
                filter_issue(a, rp + 2 * stride, pairs, stages + st * N, full0 + 8u * st, ROW);
                ++nis[st];
            }
        } else {
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) buf[10 * j + q] = y[q];
        if (j + 160 < 256) {
#pragma unroll
            for (int q = 0; q < 10; ++q) buf[10 * (j + 160) + q] = y2[q];
        }
        __syncthreads();
        float2 x[16];
        // forward pass 2 (radix 16, Ns = 10)
        {
#pragma unroll
            for (int m = 0; m < 16; ++m) x[m] = buf[j + 160 * m];
            twiddle_by<16, false>(x, a.tw, (j % 10) * 16);
            dft16<false>(x);
        }
        __syncthreads();
        {
#pragma unroll
            for (int q = 0; q < 16; ++q) buf[pad16((j / 10) * 160 + j % 10 + 10 * q)] = x[q];
        }
        __syncthreads();
        {
            // forward pass 3 (radix 16, Ns = 160): thread j ends with X[j + 160 q]
#pragma unroll
            for (int m = 0; m < 16; ++m) x[m] = buf[pad16(j + 160 * m)];
            twiddle_by<16, false>(x, a.tw, j);
            dft16<false>(x);
            // the kernel's spectrum (real, 1/N folded in) and the caller's scale
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float hq = __ldg(a.spec + j + 160 * q) * a.scale;
                x[q] = make_float2(x[q].x * hq, x[q].y * hq);
            }
            // inverse pass 1 (radix 16, Ns = 1) on the registers
            dft16<true>(x);
        }
        __syncthreads();   // everyone's pass-3 reads are done
        {
#pragma unroll
            for (int q = 0; q < 16; ++q) buf[pad16(16 * j + q)] = x[q];
        }
        __syncthreads();
        // inverse pass 2 (radix 16, Ns = 16)
        {
#pragma unroll
            for (int m = 0; m < 16; ++m) x[m] = buf[pad16(j + 160 * m)];
            twiddle_by<16, true>(x, a.tw, (j % 16) * 10);
            dft16<true>(x);
        }
        __syncthreads();
        {
#pragma unroll
            for (int q = 0; q < 16; ++q) buf[pad16((j / 16) * 256 + j % 16 + 16 * q)] = x[q];
        }
        __syncthreads();
        // inverse pass 3 (radix 10, Ns = 256): butterfly jb ends with result[jb + 256 q]
        float *o1 = a.out + ((long long)k * a.H + r1) * a.W;
        float *o2 = a.out + ((long long)k * a.H + r2) * a.W;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jb = j + 160 * h;
            if (jb < 256) {
#pragma unroll
                for (int m = 0; m < 10; ++m) y[m] = buf[pad16(jb + 256 * m)];
                twiddle_by<10, true>(y, a.tw, jb);
                dft10<true>(y);
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    const int col = jb + 256 * q;
                    if (col < a.W) {
                        o1[col] = y[q].x;
                        if (has2) o2[col] = y[q].y;
                    }
                }
            }
        }
    }
}

fdk_status launch_twiddles(float2 *tw, int N, cudaStream_t s)
{
    fdk_twiddle_kernel<<<(N + 255) / 256, 256, 0, s>>>(tw, N);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("filter twiddle launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

fdk_status launch_ramlak_spectrum(float *spec, int N, cudaStream_t s)
{
    fdk_ramlak_spectrum_kernel<<<(N + 255) / 256, 256, 0, s>>>(spec, N);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("filter spectrum launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

fdk_status launch_filter(float *out, const float *in, const float *spec, const float2 *tw, float scale,
                         const float *mats_host, const float *mats_dev, int W, int H, int n_views,
                         int N, unsigned *err, cudaStream_t s)
{
    static thread_local FilterArgs a;
    a.out = out;
    a.in = in;
    a.spec = spec;
    a.tw = tw;
    a.err = err;
    a.wait_limit = consumer_wait_limit();
    a.scale = scale;
    a.mats_dev = mats_dev;
    a.W = W;
    a.H = H;
    a.n_views = n_views;
    a.N = N;
    if (!mats_dev) memcpy(a.mats, mats_host, sizeof(float) * 12 * n_views);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long total = (long long)((H + 1) / 2) * n_views;
    if (N == kF25N && tw) {
        const bool staged = err && W % 4 == 0 && ((uintptr_t)in % 16) == 0;
        auto k = staged ? fdk_filter2560_kernel<true> : fdk_filter2560_kernel<false>;
        const int smem = (int)(sizeof(float2) * (kF25N + kF25N / 16) + (staged ? sizeof(float) * 2 * kF25N : 0));
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("filter: shared-memory opt-in failed: %s", cudaGetErrorString(e));
            return FDK_ERR_CUDA;
        }
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 160, smem) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        long long grid = (long long)sms * per_sm;
        if (grid > total) grid = total;
        if (grid < 1) return FDK_OK;
        k<<<(unsigned)grid, 160, smem, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("filter launch failed: %s", cudaGetErrorString(e));
            return FDK_ERR_CUDA;
        }
        return FDK_OK;
    }
    if (N == kF16N && tw) {
        // rows staged by bulk copies when each row is a whole number of
        // 16-byte units starting on a 16-byte boundary
        const bool staged = err && W % 4 == 0 && ((uintptr_t)in % 16) == 0;
        auto k = staged ? fdk_filter4096_kernel<true> : fdk_filter4096_kernel<false>;
        const int smem = (int)(sizeof(float2) * (kF16N + kF16N / 16) + (staged ? sizeof(float) * 2 * kF16N : 0));
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("filter: shared-memory opt-in failed: %s", cudaGetErrorString(e));
            return FDK_ERR_CUDA;
        }
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        long long grid = (long long)sms * per_sm;
        if (grid > total) grid = total;
        if (grid < 1) return FDK_OK;
        k<<<(unsigned)grid, 256, smem, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("filter launch failed: %s", cudaGetErrorString(e));
            return FDK_ERR_CUDA;
        }
        return FDK_OK;
    }
    constexpr int NT = 256;
    const size_t smem = sizeof(float2) * (size_t)(2 * N + 3 * N / 4);
    cudaError_t e = cudaFuncSetAttribute(fdk_filter_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("filter: shared-memory opt-in failed: %s", cudaGetErrorString(e));
        return FDK_ERR_CUDA;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fdk_filter_kernel<NT>, NT, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    long long grid = (long long)sms * per_sm;
    if (grid > total) grid = total;
    if (grid < 1) return FDK_OK;
    fdk_filter_kernel<NT><<<(unsigned)grid, NT, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("filter launch failed: %s", cudaGetErrorString(e));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

}  // namespace fdk
