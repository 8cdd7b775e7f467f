// FDK pre-processing on the device: cosine pre-weighting and Ram-Lak row
// filtering (the data of the paper arrives in this form, Sec. IV).
//
//   out[k][n][m] = scale * sum_{m'} h(m - m') c_k(m', n) in[k][n][m']
//   h(0) = 1/4, h(d) = -1/(pi^2 d^2) for odd d, 0 for even d != 0
//   c_k(m, n) = f / sqrt(f^2 + (m - u0)^2 + (n - v0)^2)
//
// with (f, u0, v0) read off view k's matrix through M M^T (square pixels, no
// skew).  The linear convolution along a row is evaluated as a circular one
// of length N = 2^ceil(log2(2W)) >= 2W (so every lag |m - m'| < W is within
// N/2 and nothing wraps): two rows are packed as the real and imaginary
// parts of one complex signal, transformed by a radix-4 Stockham FFT in
// shared memory, multiplied by the kernel's spectrum (real, since h is
// even) and transformed back.
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

struct FilterArgs {
    float *out;
    const float *in;
    const float *spec;      // N spectrum values (1/N folded in)
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

fdk_status launch_filter(float *out, const float *in, const float *spec, float scale,
                         const float *mats_host, const float *mats_dev, int W, int H, int n_views,
                         int N, cudaStream_t s)
{
    static thread_local FilterArgs a;
    a.out = out;
    a.in = in;
    a.spec = spec;
    a.scale = scale;
    a.mats_dev = mats_dev;
    a.W = W;
    a.H = H;
    a.n_views = n_views;
    a.N = N;
    if (!mats_dev) memcpy(a.mats, mats_host, sizeof(float) * 12 * n_views);
    constexpr int NT = 256;
    const size_t smem = sizeof(float2) * (size_t)(2 * N + 3 * N / 4);
    cudaError_t err = cudaFuncSetAttribute(fdk_filter_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) {
        cudaGetLastError();
        set_error("filter: shared-memory opt-in failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fdk_filter_kernel<NT>, NT, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long long total = (long long)((H + 1) / 2) * n_views;
    long long grid = (long long)sms * per_sm;
    if (grid > total) grid = total;
    if (grid < 1) return FDK_OK;
    fdk_filter_kernel<NT><<<(unsigned)grid, NT, smem, s>>>(a);
    err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("filter launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

}  // namespace fdk
