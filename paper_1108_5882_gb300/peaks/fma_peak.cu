// FP32 and FP64 fused multiply-add rates of this GPU's SIMT pipes, measured.
//
// The FP32-bound kernels of the library (the batched event x wave x start contraction, the
// normalisation integral) are reported as a fraction of the FFMA rate this microbenchmark
// measures on the same GPU in the same run; no vendor figure is involved.  It is built into its
// own library (libpwa_peaks.so): measurement support, not part of the likelihood path.
//
// Each thread runs 8 independent FMA chains x = x * a + b (|a| < 1, so the values stay bounded);
// 8 chains per thread and 32 warps per SM cover the FMA latency on every scheduler.  The chains
// are summed and stored under a condition that is never true in practice, so the compiler
// keeps every FMA.
#include <cuda_runtime.h>
#include <stdint.h>

#define PEAK_API extern "C" __attribute__((visibility("default")))

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* __restrict__ out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            x0 = fma(x0, a, b);
            x1 = fma(x1, a, b);
            x2 = fma(x2, a, b);
            x3 = fma(x3, a, b);
            x4 = fma(x4, a, b);
            x5 = fma(x5, a, b);
            x6 = fma(x6, a, b);
            x7 = fma(x7, a, b);
        }
    }
    const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == (T)-1234.5) out[blockIdx.x] = s;
}

}  // namespace

// Times `launches` back-to-back launches of blocks x 256 threads doing `iters` x 256 FMAs per
// thread, on `stream` (NULL: the legacy default stream).  Writes the elapsed milliseconds of
// the whole sequence and the flop count (2 per FMA).  fp64 selects DFMA instead of FFMA.
// Returns 0, or the CUDA error code.
PEAK_API int pwa_peak_fma(int fp64, int blocks, int iters, int launches, float* ms, double* flops, void* stream) {
    if (blocks < 1 || iters < 1 || launches < 1 || !ms || !flops) return (int)cudaErrorInvalidValue;
    cudaStream_t st = (cudaStream_t)stream;
    void* out = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(double) * (size_t)blocks);
    if (e != cudaSuccess) return (int)e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&]() {
        if (fp64)
            k_fma_chains<double><<<blocks, 256, 0, st>>>((double*)out, iters, 0.9999999, 1e-7);
        else
            k_fma_chains<float><<<blocks, 256, 0, st>>>((float*)out, iters, 0.9999f, 1e-4f);
    };
    launch();  // warm-up (module load, clocks)
    cudaEventRecord(e0, st);
    for (int l = 0; l < launches; ++l) launch();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) {
        cudaEventElapsedTime(ms, e0, e1);
        *flops = 2.0 * 8.0 * 32.0 * (double)iters * 256.0 * (double)blocks * (double)launches;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return (int)e;
}
