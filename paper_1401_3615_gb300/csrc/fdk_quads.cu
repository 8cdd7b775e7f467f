// Quad images: each projection is re-laid as a grid of 2x2 tap cells so the
// back-projection fetches the four bilinear taps of a voxel with one 16-byte
// (FP32) or 8-byte (FP16/BF16) load.  Cell (i, j) holds
//   (p(i, j), p(i+1, j), p(i, j+1), p(i+1, j+1)),   p = 0 outside the image,
// for i in [-2, W] and j in [-2, H]; the outermost cells are all zero, so any
// detector position clamped into that range reads exactly the bilinear value
// the definition gives (zero off the detector).  This is the GPU form of the
// paper's zero-padding copy (Sec. VI), widened so one load serves all taps.
#include "fdk_internal.cuh"

namespace fdk {

template <typename T> struct QuadOf;
template <> struct QuadOf<float> { using type = float4; };
template <> struct QuadOf<__half> { using type = uint2; };
template <> struct QuadOf<__nv_bfloat16> { using type = uint2; };

template <typename T>
__device__ __forceinline__ T tap(const T *img, int W, int H, int i, int j)
{
    return ((unsigned)i < (unsigned)W && (unsigned)j < (unsigned)H) ? img[(long long)j * W + i] : T(0.0f);
}

__device__ __forceinline__ float4 pack4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }

template <typename T>
__device__ __forceinline__ uint2 pack4(T a, T b, T c, T d)
{
    const unsigned short ua = *reinterpret_cast<unsigned short *>(&a);
    const unsigned short ub = *reinterpret_cast<unsigned short *>(&b);
    const unsigned short uc = *reinterpret_cast<unsigned short *>(&c);
    const unsigned short ud = *reinterpret_cast<unsigned short *>(&d);
    return make_uint2((unsigned)ua | ((unsigned)ub << 16), (unsigned)uc | ((unsigned)ud << 16));
}

// One thread per quad cell; grid-stride over all cells of n images.
template <typename T>
__global__ void fdk_make_quads_kernel(const T *__restrict__ proj, typename QuadOf<T>::type *__restrict__ quads,
                                      int n, int W, int H, int QP, int QH)
{
    const long long per = (long long)QP * QH;
    const long long total = per * n;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(q / per);
        const long long r = q - (long long)k * per;
        const int j = (int)(r / QP) - 2, i = (int)(r % QP) - 2;
        const T *img = proj + (long long)k * W * H;
        quads[q] = pack4(tap(img, W, H, i, j), tap(img, W, H, i + 1, j), tap(img, W, H, i, j + 1),
                         tap(img, W, H, i + 1, j + 1));
    }
}

size_t quad_elem_size(int dtype) { return dtype == FDK_F32 ? 16 : 8; }

fdk_status launch_make_quads(const void *proj, void *quads, int n, int W, int H, int dtype,
                             cudaStream_t s)
{
    const int QP = W + 3, QH = H + 3;
    const long long total = (long long)QP * QH * n;
    if (total == 0) return FDK_OK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    const long long cap = (long long)(sms > 0 ? sms : 152) * 8;
    if (blocks > cap) blocks = cap;
    switch (dtype) {
    case FDK_F32:
        fdk_make_quads_kernel<float><<<(unsigned)blocks, threads, 0, s>>>(
            static_cast<const float *>(proj), static_cast<float4 *>(quads), n, W, H, QP, QH);
        break;
    case FDK_F16:
        fdk_make_quads_kernel<__half><<<(unsigned)blocks, threads, 0, s>>>(
            static_cast<const __half *>(proj), static_cast<uint2 *>(quads), n, W, H, QP, QH);
        break;
    default:
        fdk_make_quads_kernel<__nv_bfloat16><<<(unsigned)blocks, threads, 0, s>>>(
            static_cast<const __nv_bfloat16 *>(proj), static_cast<uint2 *>(quads), n, W, H, QP, QH);
        break;
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("quad staging launch failed: %s", cudaGetErrorString(err));
        return FDK_ERR_CUDA;
    }
    return FDK_OK;
}

}  // namespace fdk
