// FP64 FMA throughput probe: the denominator of the diagram kernels'
// roofline (the FP64 pipe bounds them).
#include <cuda_runtime.h>

#include "mgpu.h"
#include "mgpu_bench.h"

namespace {

__global__ void __launch_bounds__(256) k_dfma(double *out, int iters, double a, double b) {
    double x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = threadIdx.x * 1e-9 + k;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 16; k++) s += x[k];
    if (s == 1234.5678) out[threadIdx.x] = s;  // keeps the chains live
}

}  // namespace

extern "C" int mg_probe_fp64_peak(int blocks, int iters, int reps, double *flops_out) {
    if (!flops_out || iters <= 0 || reps <= 0) return MG_ERR_BAD_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MG_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MG_ERR_CUDA;
    if (blocks <= 0) blocks = 8 * nsm;
    double *d = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = MG_OK;
    float best = 1e30f;
    if (cudaMalloc(&d, 256 * sizeof(double)) != cudaSuccess) return MG_ERR_NO_MEMORY;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = MG_ERR_CUDA;
        goto done;
    }
    k_dfma<<<blocks, 256, 0, s>>>(d, iters, 0.999999, 1e-7);
    for (int r = 0; r < reps && st == MG_OK; r++) {
        cudaEventRecord(e0, s);
        k_dfma<<<blocks, 256, 0, s>>>(d, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = MG_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    if (st == MG_OK && cudaGetLastError() != cudaSuccess) st = MG_ERR_CUDA;
    if (st == MG_OK) *flops_out = 2.0 * 16.0 * iters * 256.0 * blocks / (best * 1e-3);
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(d);
    return st;
}
