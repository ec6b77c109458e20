// peak.cu -- arithmetic rate of this GPU, measured: the roofs that the FP64
// kernels (two-link build, APE step) and the FP32 stencil arithmetic are
// judged against.  Not a step of the method (the paper has no counterpart).
//
// Each thread runs 8 independent FMA chains x <- x * b + c with |b| < 1, so
// no value overflows and no chain waits on another; nothing touches memory
// except one conditional store that keeps the compiler from dropping the
// chains.  The rate is 2 flops per FMA (per lane for the packed FP32 pair
// form) over the kernel's CUDA-event time on its own stream.
#include <cuda_runtime.h>

#include "../../include/tls.h"

namespace {

template <typename T> struct Fma;
template <> struct Fma<double> {
    static __device__ __forceinline__ double f(double a, double b, double c) { return fma(a, b, c); }
    static constexpr int lanes = 1;
};
template <> struct Fma<float> {
    static __device__ __forceinline__ float f(float a, float b, float c) { return fmaf(a, b, c); }
    static constexpr int lanes = 1;
};
template <> struct Fma<float2> {
    static __device__ __forceinline__ float2 f(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    static constexpr int lanes = 2;
};

template <typename T> __device__ __forceinline__ T splat(float v);
template <> __device__ __forceinline__ double splat<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ float splat<float>(float v) { return v; }
template <> __device__ __forceinline__ float2 splat<float2>(float v) { return make_float2(v, v * 0.5f); }

template <typename T> __device__ __forceinline__ bool is_magic(T v);
template <> __device__ __forceinline__ bool is_magic<double>(double v) { return v == 1234.5; }
template <> __device__ __forceinline__ bool is_magic<float>(float v) { return v == 1234.5f; }
template <> __device__ __forceinline__ bool is_magic<float2>(float2 v) { return v.x == 1234.5f; }

template <typename T> __device__ __forceinline__ T add(T a, T b) { return a + b; }
template <> __device__ __forceinline__ float2 add<float2>(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, float seed, T *sink)
{
    T x[8];
    const T b = splat<T>(0.999999f), c = splat<T>(1e-7f);
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = splat<T>(seed + 0.01f * k + 1e-6f * threadIdx.x);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = Fma<T>::f(x[k], b, c);
    }
    T s = x[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) s = add(s, x[k]);
    if (is_magic(s)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T> tls_status run(int device, double *tflops)
{
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return TLS_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, 256, 0);
    if (sms <= 0 || per_sm <= 0) return TLS_ERR_CUDA;
    const int grid = sms * per_sm;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return TLS_ERR_CUDA;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // calibrate the loop count to about 100 ms per launch, then time the best of 3
    int iters = 64;
    double best = 0.0;
    tls_status st = TLS_OK;
    for (int rep = 0; rep < 8 && st == TLS_OK; ++rep) {
        cudaEventRecord(a, s);
        k_fma_chains<T><<<grid, 256, 0, s>>>(iters, 0.5f, nullptr);
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            st = TLS_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const double fmas = (double)grid * 256 * iters * 16 * 8 * Fma<T>::lanes;
        if (ms < 50.f && iters < (1 << 24)) {
            iters = (int)(iters * (100.0 / (ms > 0.01f ? ms : 0.01f)));
            if (iters < 64) iters = 64;
            if (iters > (1 << 24)) iters = 1 << 24;
            continue;
        }
        const double r = 2.0 * fmas / (ms * 1e-3) / 1e12;
        if (r > best) best = r;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(s);
    if (st != TLS_OK) return st;
    *tflops = best;
    return TLS_OK;
}

}  // namespace

extern "C" tls_status tls_peak_flops(int device, int kind, double *tflops)
{
    if (!tflops) return TLS_ERR_ARG;
    *tflops = 0.0;
    switch (kind) {
    case TLS_PEAK_F64: return run<double>(device, tflops);
    case TLS_PEAK_F32: return run<float>(device, tflops);
    case TLS_PEAK_F32X2: return run<float2>(device, tflops);
    default: return TLS_ERR_ARG;
    }
}
