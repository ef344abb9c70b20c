// Fused multiply-add throughput of the device, for the arithmetic roofline
// of the kernels that run in FP64 (the FP64 sweep is bound by FP64 issue on
// GB300, not by memory).  Each thread runs eight independent FMA chains;
// the grid holds a few blocks per SM so that every sub-partition issues.
#include <cuda_runtime.h>

#include "../../include/lbib.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T *__restrict__ sink, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == T(-1.25)) sink[0] = s;  // never true; keeps the chains live
}

template <typename T>
int measure(double *flops) {
    int dev = 0, nsm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBIB_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LBIB_ECUDA;
    T *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    int rc = LBIB_OK;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        rc = LBIB_ECUDA;
    const int blocks = 8 * nsm, threads = 256, iters = sizeof(T) == 8 ? 2048 : 65536;
    float best = 1e30f;
    for (int rep = 0; rep < 3 && rc == LBIB_OK; ++rep) {
        cudaEventRecord(e0, s);
        k_fma_chains<T><<<blocks, threads, 0, s>>>(sink, iters, T(0.999999), T(1e-7));
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = LBIB_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // the first launch warms up
    }
    if (rc == LBIB_OK) *flops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3);
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return rc;
}

}  // namespace

extern "C" int lbib_measure_fma(int fp64, double *flops_per_s) {
    if (!flops_per_s) return LBIB_EINVAL;
    return fp64 ? measure<double>(flops_per_s) : measure<float>(flops_per_s);
}
