// peaks.cu -- FP32 and FP64 FMA throughput of the device (measurement only).
//
// The classification and root-solve kernels are bound by FP32 and FP64
// arithmetic, not by memory, so their roofline needs the device's FMA rate.
// peaks_fma() times a kernel in which every thread runs NCHAIN independent
// FMA chains for `iters` iterations (no memory traffic inside the loop), on a
// grid of blocks_per_sm * SMs blocks, with CUDA events on the given stream.
// One FMA counts as two flops.  The result is stored behind a comparison the
// compiler cannot resolve, so the chains are not removed.
//
// This library is separate from libeses: it is a measuring tool for the
// benchmark, not part of the surface computation.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int NCHAIN = 8;
constexpr int THREADS = 256;

template <class T>
__global__ void __launch_bounds__(THREADS) k_fma(int iters, T a, T b, T *out, T sentinel)
{
    T x[NCHAIN];
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < NCHAIN; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) s += x[c];
    if (s == sentinel) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int time_fma(int blocks_per_sm, int iters, int reps, cudaStream_t st, double *tflops, double *ms_out)
{
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    const int grid = n_sm * blocks_per_sm;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * (size_t)grid * THREADS) != cudaSuccess) return -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = (T)0.999999, b = (T)1e-7;
    k_fma<T><<<grid, THREADS, 0, st>>>(iters, a, b, out, (T)-12345.0);  // warm-up
    double best = 0.0, best_ms = 0.0;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, st);
        k_fma<T><<<grid, THREADS, 0, st>>>(iters, a, b, out, (T)-12345.0);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * NCHAIN * 16.0 * (double)iters * (double)grid * THREADS;
        const double tf = flops / (ms * 1e-3) / 1e12;
        if (tf > best) {
            best = tf;
            best_ms = ms;
        }
    }
    const int rc = cudaGetLastError() == cudaSuccess ? 0 : -1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *tflops = best;
    *ms_out = best_ms;
    return rc;
}

}  // namespace

// out[0] FP32 TFLOP/s, out[1] its kernel ms, out[2] FP64 TFLOP/s, out[3] its
// kernel ms (best of `reps` launches each).  Returns 0, or -1 on a CUDA error.
extern "C" int peaks_fma(int reps, void *stream, double out[4])
{
    cudaStream_t st = (cudaStream_t)stream;
    if (reps < 1) reps = 1;
    // FP32: 8 blocks of 256 threads per SM (full occupancy), ~1e12 FMAs
    if (time_fma<float>(8, 4096, reps, st, &out[0], &out[1]) != 0) return -1;
    // FP64 runs far slower on this part: fewer iterations for a similar time
    if (time_fma<double>(8, 64, reps, st, &out[2], &out[3]) != 0) return -1;
    return 0;
}
