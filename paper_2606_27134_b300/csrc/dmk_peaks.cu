// Throughput microbenchmarks of the three arithmetic pipes the DMK kernels are bound by:
// the FP32 FMA pipe (residual sums, Chebyshev and plane-wave contractions of the mixed path),
// the FP64 FMA pipe (the plain path and the root far field) and the MUFU reciprocal square
// root (one per residual pair).  They give the measured denominators of the roofline
// fractions; the GPU's clocks and settings are left as they are.
//
// Every thread runs kChains independent dependency chains so that the pipe, not the latency
// of one chain, sets the rate; the chains converge to finite fixed points (no overflow, no
// denormals), and every thread writes its result so that nothing is eliminated.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;

__global__ void __launch_bounds__(kThreads) k_ffma32(int iters, float b, float c, float* out) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = 0.01f * (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_dfma64(int iters, double b, double c, double* out) {
    double a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = 0.01 * (double)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x -> x^(-1/2) has the fixed point 1; the chains stay within [0.5, 2]
__global__ void __launch_bounds__(kThreads) k_mufu_rsqrt(int iters, float* out) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = 1.0f + 0.05f * (float)i + 1e-6f * (float)threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = rsqrt_approx(a[i]);
    }
    float s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

/* Measured throughput of one pipe on the current device, best of `reps` timed launches
 * (CUDA events on a stream of its own, after one warm-up launch).
 *   which = 0: FP32 FFMA, result in FLOP/s (2 per FMA);
 *   which = 1: FP64 DFMA, FLOP/s (2 per FMA);
 *   which = 2: MUFU rsqrt.approx.f32, operations/s.
 * The grid is 4 blocks of 512 threads per SM (2048 resident threads); `iters` x 16 x 8
 * operations per thread.  *ops_per_s and *ms (the best launch's duration) are written on
 * success.  Returns 0, or the CUDA error code. */
int dmk_peak_measure(int which, int iters, int reps, double* ops_per_s, double* ms) {
    if (!ops_per_s || !ms || which < 0 || which > 2 || iters < 1 || reps < 1) return (int)cudaErrorInvalidValue;
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
    const int blocks = 4 * n_sm;
    const size_t n_out = (size_t)blocks * kThreads;
    void* out = nullptr;
    if ((e = cudaMalloc(&out, n_out * sizeof(double))) != cudaSuccess) return (int)e;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    auto launch = [&]() {
        if (which == 0) k_ffma32<<<blocks, kThreads, 0, st>>>(iters, 0.999999f, 1e-7f, (float*)out);
        else if (which == 1) k_dfma64<<<blocks, kThreads, 0, st>>>(iters, 0.999999, 1e-7, (double*)out);
        else k_mufu_rsqrt<<<blocks, kThreads, 0, st>>>(iters, (float*)out);
    };
    launch();
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a, st);
        launch();
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float t = 0;
        cudaEventElapsedTime(&t, a, b);
        best = std::min(best, t);
    }
    e = cudaGetLastError();
    const double ops = (double)n_out * iters * 16.0 * kChains * (which == 2 ? 1.0 : 2.0);
    *ms = best;
    *ops_per_s = ops / (best * 1e-3);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(st);
    cudaFree(out);
    return (int)e;
}

}  // extern "C"
