// k_probe.cu -- FP64 throughput probes.
//
// The rotation passes of this library are bound by the FP64 pipe, not by
// HBM (a pair costs three FMAs on 16 bytes that stay on chip for many
// passes), so the roofline of those kernels is the rate at which the GPU
// retires FP64 fused multiply-adds.  Two probes measure it on the device at
// hand: independent DFMA chains in every thread of a full-occupancy grid, and
// independent chains of the FP64 matrix instruction (8x8x4 per warp), whose
// rate shows whether the tensor path would beat plain DFMA for this work.
#include <cuda_runtime.h>

#include "../../include/stab.h"
#include "launch.h"

namespace stab {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kDfmaChains = 8;
constexpr int kDmmaChains = 4;

// a <- a * b + c on kDfmaChains independent chains; a stays bounded (it
// converges to c / (1 - b)), so no chain overflows or goes subnormal.
__global__ void __launch_bounds__(kProbeThreads) k_probe_dfma(int64_t iters, double b, double c,
                                                              double *sink) {
    double a[kDfmaChains];
#pragma unroll
    for (int k = 0; k < kDfmaChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + 32 * k);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kDfmaChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kDfmaChains; ++k) s += a[k];
    // never true for the arguments the host passes; keeps the chains live
    if (s == -1.0) sink[threadIdx.x] = s;
}

// D <- A B + D with the m8n8k4 FP64 matrix instruction, kDmmaChains
// independent accumulators per warp.
__global__ void __launch_bounds__(kProbeThreads) k_probe_dmma(int64_t iters, double b, double c,
                                                              double *sink) {
    const double av = b, bv = 1e-3 * (1 + (threadIdx.x & 7));
    double d0[kDmmaChains], d1[kDmmaChains];
#pragma unroll
    for (int k = 0; k < kDmmaChains; ++k) {
        d0[k] = c * (k + 1);
        d1[k] = c * (k + 2);
    }
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kDmmaChains; ++k) {
            asm volatile(
                "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                : "+d"(d0[k]), "+d"(d1[k])
                : "d"(av), "d"(bv));
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kDmmaChains; ++k) s += d0[k] + d1[k];
    if (s == -1.0) sink[threadIdx.x] = s;
}

}  // namespace

}  // namespace stab

using namespace stab;

extern "C" int stab_probe_fp64(int kind, int64_t iters, double *tflops, double *ms) {
    if (!tflops || (kind != 0 && kind != 1)) return STAB_E_INVAL;
    if (iters < 1 || iters > ((int64_t)1 << 30)) return STAB_E_RANGE;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = kind == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_probe_dfma,
                                                                      kProbeThreads, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_probe_dmma,
                                                                      kProbeThreads, 0);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return STAB_E_CUDA;
    }
    if (occ < 1) occ = 1;
    const int grid = sms * occ;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double *sink = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&sink, kProbeThreads * sizeof(double), st);
    const double b = 0.999999, c = 1e-6;
    auto launch = [&](int64_t it) {
        if (kind == 0) k_probe_dfma<<<grid, kProbeThreads, 0, st>>>(it, b, c, sink);
        else k_probe_dmma<<<grid, kProbeThreads, 0, st>>>(it, b, c, sink);
        return cudaGetLastError();
    };
    float t = 0.0f;
    if (e == cudaSuccess) e = launch(iters / 8 + 1);   // warm-up: clocks up, code loaded
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch(iters);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (sink) cudaFreeAsync(sink, st);
    if (st) cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return STAB_E_CUDA;
    }
    const double threads = (double)grid * kProbeThreads;
    // DFMA: 2 flops per chain step per thread; DMMA: 8 x 8 x 4 FMAs per warp
    // instruction, i.e. 2 * 256 / 32 = 16 flops per thread and chain step
    const double flops = kind == 0 ? threads * kDfmaChains * 2.0 * (double)iters
                                   : threads * kDmmaChains * 16.0 * (double)iters;
    *tflops = t > 0.0f ? flops / (t * 1e-3) / 1e12 : 0.0;
    if (ms) *ms = t;
    return STAB_OK;
}
