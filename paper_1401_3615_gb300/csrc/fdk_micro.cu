// Gather micro-benchmarks: the GB300 counterpart of the paper's gather
// measurements on the Xeon Phi (Sec. V, Table II), which explain where the
// back-projection's time goes.
//
//   FDK_MICRO_LDG    warp-wide 4-byte loads from L1-resident data whose 32
//                    lanes touch `param` distinct 128-byte lines (1..32)
//   FDK_MICRO_LDS    warp-wide 4-byte shared-memory loads with a `param`-way
//                    bank conflict (1..32)
//   FDK_MICRO_TLD4   2x2 texture gathers (tex2Dgather) at random texels of a
//                    `param` x `param` texture
//   FDK_MICRO_RCP    reciprocal approximations (rcp.approx.ftz.f32)
//   FDK_MICRO_CHASE  dependent loads (pointer chase) over a `param`-KiB ring:
//                    the latency of L1, L2 or HBM hits
//
// Throughput kernels keep 16 independent operations per thread in flight
// (for shared memory and reciprocals each is a dependent chain, so the
// compiler can neither hoist nor fold them) on every SM; a launch is timed
// with CUDA events and converted to operations per SM per cycle with the SM
// clock measured by a clock64 spin of known length.  The chase runs one
// thread and reports cycles per load (clock64).
#include <string.h>

#include "fdk_internal.cuh"

namespace fdk {

constexpr int kMicroIters = 256;
constexpr int kMicroUnroll = 16;

__global__ void __launch_bounds__(256, 8) micro_ldg_kernel(const float *__restrict__ buf, int lines, float *sink)
{
    const int lane = threadIdx.x & 31;
    // lanes spread over `lines` distinct 128-byte lines, distinct words within a line
    const int line = lane % lines;
    const int word = (lane / lines) % 32;
    // 64 lines of 128 bytes (8 KB) from one of 8 bases 4 KB apart (40 KB in
    // all, resident in L1), rotated per unrolled load
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const float *base = buf + (warp & 7) * 1024;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int rot = 0;
    for (int it = 0; it < kMicroIters; ++it) {
#pragma unroll
        for (int u = 0; u < kMicroUnroll; ++u) {
            const int l = (line * 2 + u + rot) & 63;
            acc[u & 3] += __ldg(base + l * 32 + word);
        }
        rot += 17;
    }
    if (acc[0] + acc[1] + acc[2] + acc[3] == -1.0f) sink[0] = acc[0];   // never true; keeps the loads
}

// Each lane walks its row of a 32 x 32 table (next word = s[current]);
// lanes with equal lane % (32 / conflict) are in the same bank at every
// step, in `conflict` different rows.
__global__ void __launch_bounds__(256, 8) micro_lds_kernel(int conflict, float *sink)
{
    __shared__ int s[32 * 32];
    for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) s[i] = (i & ~31) | ((i + 1) & 31);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int per = 32 / conflict;
    const int row = lane / per;
    int p[kMicroUnroll];
#pragma unroll
    for (int u = 0; u < kMicroUnroll; ++u) p[u] = row * 32 + (((lane % per) + 2 * u) & 31);
    for (int it = 0; it < kMicroIters; ++it) {
#pragma unroll
        for (int u = 0; u < kMicroUnroll; ++u) p[u] = s[p[u]];
    }
    int acc = 0;
#pragma unroll
    for (int u = 0; u < kMicroUnroll; ++u) acc += p[u];
    if (acc == -1) sink[0] = (float)acc;
}

__global__ void __launch_bounds__(256, 8) micro_tld4_kernel(cudaTextureObject_t tex, int size, float *sink)
{
    unsigned h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u;
    float acc = 0.0f;
    for (int it = 0; it < kMicroIters; ++it) {
#pragma unroll
        for (int u = 0; u < kMicroUnroll; ++u) {
            h = h * 1664525u + 1013904223u;
            const float x = (float)((h >> 8) % (unsigned)size) + 0.5f;
            const float y = (float)((h >> 20) % (unsigned)size) + 0.5f;
            const float4 g = tex2Dgather<float4>(tex, x, y, 0);
            acc += g.x + g.w;
        }
    }
    if (acc == -1.0f) sink[0] = acc;
}

// x <- 1 / (x + 1) per chain (converges to 0.618...), one add and one
// reciprocal approximation per step.
__global__ void __launch_bounds__(256, 8) micro_rcp_kernel(float seed, float *sink)
{
    float x[kMicroUnroll];
#pragma unroll
    for (int u = 0; u < kMicroUnroll; ++u) x[u] = seed + (float)(threadIdx.x + u);
    for (int it = 0; it < kMicroIters; ++it) {
#pragma unroll
        for (int u = 0; u < kMicroUnroll; ++u) {
            float r;
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[u] + 1.0f));
            x[u] = r;
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int u = 0; u < kMicroUnroll; ++u) acc += x[u];
    if (acc == -1.0f) sink[0] = acc;
}

// One thread follows next = ring[next] for `steps` loads.
__global__ void micro_chase_kernel(const unsigned *__restrict__ ring, int steps, unsigned long long *cycles,
                                   unsigned *sink)
{
    unsigned p = 0;
    for (int i = 0; i < 64; ++i) p = ring[p];   // warm the path
    const unsigned long long t0 = clock64();
    for (int i = 0; i < steps; ++i) p = ring[p];
    const unsigned long long t1 = clock64();
    cycles[0] = t1 - t0;
    sink[0] = p;
}

// Spin for `spin` SM cycles (clock64 always advances, so this ends).
__global__ void micro_clock_kernel(unsigned long long *out, long long spin)
{
    const unsigned long long t0 = clock64();
    while ((long long)(clock64() - t0) < spin) {
    }
    out[0] = clock64() - t0;
}

// Ring next(i) = (i + 4 KB + 128 B) mod size: consecutive loads fall in
// different 128-byte lines and 4 KB pages.
__global__ void micro_ring_kernel(unsigned *ring, unsigned words)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= words) return;
    const unsigned stride = 1056;   // 4 KB + 128 B in words
    ring[i] = (unsigned)(((unsigned long long)i + stride) % words);
}

}  // namespace fdk

using namespace fdk;

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() { cudaEventCreate(&a); cudaEventCreate(&b); }
    ~Timer() { cudaEventDestroy(a); cudaEventDestroy(b); }
    double ms()
    {
        cudaEventSynchronize(b);
        float v = 0.0f;
        cudaEventElapsedTime(&v, a, b);
        return v;
    }
};

// SM clock in MHz: a spin of a known number of clock64 cycles timed with events.
double sm_mhz(cudaStream_t s, unsigned long long *dcyc)
{
    Timer t;
    const long long spin = 20000000;
    micro_clock_kernel<<<1, 1, 0, s>>>(dcyc, spin);
    cudaEventRecord(t.a, s);
    micro_clock_kernel<<<1, 1, 0, s>>>(dcyc, spin);
    cudaEventRecord(t.b, s);
    const double ms = t.ms();
    unsigned long long cyc = 0;
    cudaMemcpy(&cyc, dcyc, sizeof cyc, cudaMemcpyDeviceToHost);
    return ms > 0.0 ? (double)cyc / (ms * 1e3) : 0.0;
}

}  // namespace

extern "C" {

fdk_status fdk_microbench(int32_t which, int32_t param, double *result)
{
    if (!result) { set_error("result is null"); return FDK_ERR_INVALID_ARG; }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t bytes = 1 << 20;
    if (which == FDK_MICRO_CHASE) {
        if (param < 1 || param > (1 << 22)) {
            set_error("chase ring must be 1 KiB .. 4 GiB");
            return FDK_ERR_INVALID_ARG;
        }
        bytes = (size_t)param * 1024;
    } else if (which == FDK_MICRO_LDG || which == FDK_MICRO_LDS) {
        if (param < 1 || param > 32 || (32 % param) != 0) {
            set_error("the parameter must divide 32");
            return FDK_ERR_INVALID_ARG;
        }
    } else if (which == FDK_MICRO_TLD4) {
        if (param < 2 || param > 4096) {
            set_error("texture size must be 2..4096");
            return FDK_ERR_INVALID_ARG;
        }
    } else if (which != FDK_MICRO_RCP) {
        set_error("unknown micro-benchmark %d", which);
        return FDK_ERR_INVALID_ARG;
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        set_error("stream creation failed");
        return FDK_ERR_CUDA;
    }
    void *scratch = nullptr;
    if (lib_malloc(&scratch, bytes + 256) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(s);
        set_error("micro-benchmark scratch allocation failed");
        return FDK_ERR_OOM;
    }
    float *sink = reinterpret_cast<float *>(static_cast<char *>(scratch) + bytes);
    unsigned long long *dcyc = reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + bytes + 64);
    fdk_status st = FDK_OK;
    const int threads = 256, blocks = sms * 8;
    const double warp_ops = (double)blocks * (threads / 32) * kMicroIters * kMicroUnroll;
    // one warm-up launch, one timed launch; warp operations per SM per cycle
    auto rate = [&](auto launch) {
        Timer t;
        launch();
        cudaEventRecord(t.a, s);
        launch();
        cudaEventRecord(t.b, s);
        const double ms = t.ms();
        const double mhz = sm_mhz(s, dcyc);
        return (ms > 0.0 && mhz > 0.0) ? warp_ops / ((double)sms * ms * 1e-3 * mhz * 1e6) : 0.0;
    };
    switch (which) {
    case FDK_MICRO_LDG: {
        cudaMemsetAsync(scratch, 0, bytes, s);
        const float *buf = static_cast<const float *>(scratch);
        *result = rate([&] { micro_ldg_kernel<<<blocks, threads, 0, s>>>(buf, param, sink); });
        break;
    }
    case FDK_MICRO_LDS:
        *result = rate([&] { micro_lds_kernel<<<blocks, threads, 0, s>>>(param, sink); });
        break;
    case FDK_MICRO_TLD4: {
        cudaChannelFormatDesc ch = cudaCreateChannelDesc<float>();
        cudaArray_t arr = nullptr;
        if (lib_malloc_array(&arr, &ch, param, param, cudaArrayTextureGather) != cudaSuccess) {
            cudaGetLastError();
            st = FDK_ERR_OOM;
            set_error("texture array allocation failed");
            break;
        }
        cudaResourceDesc rd;
        memset(&rd, 0, sizeof rd);
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = arr;
        cudaTextureDesc td;
        memset(&td, 0, sizeof td);
        td.addressMode[0] = cudaAddressModeBorder;
        td.addressMode[1] = cudaAddressModeBorder;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        cudaTextureObject_t tex = 0;
        if (cudaCreateTextureObject(&tex, &rd, &td, nullptr) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeArray(arr);
            st = FDK_ERR_CUDA;
            set_error("texture object creation failed");
            break;
        }
        *result = rate([&] { micro_tld4_kernel<<<blocks, threads, 0, s>>>(tex, param, sink); });
        cudaDestroyTextureObject(tex);
        cudaFreeArray(arr);
        break;
    }
    case FDK_MICRO_RCP:
        *result = rate([&] { micro_rcp_kernel<<<blocks, threads, 0, s>>>(1.5f, sink); });
        break;
    case FDK_MICRO_CHASE: {
        const unsigned words = (unsigned)(bytes / 4);
        unsigned *ring = static_cast<unsigned *>(scratch);
        micro_ring_kernel<<<(words + 255) / 256, 256, 0, s>>>(ring, words);
        const int steps = 4096;
        micro_chase_kernel<<<1, 1, 0, s>>>(ring, steps, dcyc, reinterpret_cast<unsigned *>(sink));
        unsigned long long cyc = 0;
        cudaMemcpyAsync(&cyc, dcyc, sizeof cyc, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        *result = (double)cyc / steps;   // cycles per dependent load
        break;
    }
    default:
        break;
    }
    if (st == FDK_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("micro-benchmark failed: %s", cudaGetErrorString(e));
            st = FDK_ERR_CUDA;
        }
    }
    cudaFree(scratch);
    cudaStreamDestroy(s);
    return st;
}

}  // extern "C"
