// k_probe.cu -- FP64 throughput probes and a pass-latency probe.
//
// The rotation passes of this library are bound by the FP64 pipe, not by
// HBM (a pair costs three FMAs on 16 bytes that stay on chip for many
// passes), so the roofline of those kernels is the rate at which the GPU
// retires FP64 fused multiply-adds.  Two probes measure it on the device at
// hand: independent DFMA chains in every thread of a full-occupancy grid, and
// independent chains of the FP64 matrix instruction (8x8x4 per warp), whose
// rate shows whether the tensor path would beat plain DFMA for this work.
//
// The pass-latency probe times, on one CTA and with the SM's cycle counter,
// the pieces of the n = 4 register pass loop that bounds a lone vector (the
// first part of a split generator sweep): a wire pass on a wire whose group
// sits in a warp's lanes (three shuffles, then three dependent FP64
// instructions per lane), a switch of the register layout through shared
// memory, and a pull through a four-CNOT ring walked record by record.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/stab.h"
#include "device_ops.cuh"
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

// ---------------------------------------------------------------- pass latency

// The four index bits of lane/thread t in the two layouts of the probe: the
// identity, and the low and high nibbles swapped (the two wire pairs trade
// lane and warp positions, as in the register loop's layouts).
__device__ __forceinline__ uint32_t probe_idx(uint32_t t, int layout) {
    return layout ? (((t & 15u) << 4) | (t >> 4)) : t;
}

__device__ __forceinline__ double probe_row(const double *m, uint32_t slot, double x, double y,
                                            double z) {
    const double *mm = m + 3 * (slot - 1u);
    return fma(mm[2], z, fma(mm[1], y, mm[0] * x));
}

// A wire pass on the lane-bit pair sh, sh + 1 of a warp: slot 0 (I) keeps its
// entry, X, Y and Z get their row of the 3x3 map.
__device__ __forceinline__ void probe_lane_pass(double &v, uint32_t lane, int sh,
                                                const double *m) {
    const uint32_t zb = (lane >> sh) & 1u, xb = (lane >> (sh + 1)) & 1u;
    const uint32_t base = lane & ~(3u << sh);
    const double x = __shfl_sync(0xffffffffu, v, base | (2u << sh));
    const double y = __shfl_sync(0xffffffffu, v, base | (3u << sh));
    const double z = __shfl_sync(0xffffffffu, v, base | (1u << sh));
    if (xb | zb) v = probe_row(m, xb ? (zb ? 2u : 1u) : 3u, x, y, z);
}

// Patterns 0..2: one entry of a 4^4 vector per thread (256 threads; 128 runs
// half a vector), `passes` wire passes alternating between the two lane-bit
// pairs; 1 adds a layout switch (write, barrier, read) before every second
// pass, 2 also walks a four-CNOT ring's pull records before every fourth.
// Pattern 4 (256 threads): two-wire fused passes -- each lane's 16-entry
// block (the (z, x) bits of two wires in lane bits 0..3) goes through
// (1 + M) (x) (1 + M) in one pass: up to nine source lanes and coefficients
// per output (three with one I slot, one for I I), taken warp-uniformly as
// nine shuffles and nine dependent FP64 instructions; `passes` counts wire
// passes, two per fused pass.
// Pattern 3 (128 threads): two entries per thread, so three wires' groups
// lie within a warp (lane bits and the register); per layer three register
// passes, then the fourth wire's pass read through the ring's pull from
// shared memory -- one barrier per layer.  The map is a rotation, so every
// entry stays bounded.  clk[0] = the CTA's cycles over the timed loop.
template <int PATTERN>
__global__ void k_probe_pass(int64_t passes, const double *mtab, double *sink, long long *clk) {
    __shared__ double buf[2][256];
    __shared__ Rec recs[4];
    __shared__ double m[9];
    const uint32_t t = threadIdx.x, lane = t & 31u, w = t >> 5;
    if (t < 9) m[t] = mtab[t];
    if (t < 4) {
        Rec r{};
        r.kind = R_CX;
        r.q = (uint8_t)t;
        r.q1 = (uint8_t)((t + 1) & 3u);
        recs[t] = r;
    }
    for (uint32_t i = t; i < 512u; i += blockDim.x) (&buf[0][0])[i] = 0.0;
    double v = (t == 5u) ? 1.0 : 0.0, v1 = (t == 9u) ? 0.5 : 0.0;
    __syncthreads();
    // pattern 4: per block slot (s0 + 4 s1; slot code 0 I, 1 Z, 2 X, 3 Y by
    // the (z, x) bits), nine (source slot, coefficient) terms, zero-padded
    __shared__ uint32_t fsrc[16][9];
    __shared__ double fcoef[16][9];
    if (PATTERN == 4 && t < 16) {
        const uint32_t s0 = t & 3u, s1 = t >> 2;
        // map row of a slot code: X 1, Y 2, Z 3 (row - 1 indexes m)
        auto row = [](uint32_t sc) { return sc == 2u ? 0u : (sc == 3u ? 1u : 2u); };
        const uint32_t xyz[3] = {2u, 3u, 1u};   // slot codes of X, Y, Z
        int k = 0;
        if (s0 == 0u && s1 == 0u) {
            fsrc[t][k] = t;
            fcoef[t][k++] = 1.0;
        } else if (s0 == 0u) {
            for (int b = 0; b < 3; ++b) {
                fsrc[t][k] = xyz[b] << 2;
                fcoef[t][k++] = m[3 * row(s1) + (uint32_t)b];
            }
        } else if (s1 == 0u) {
            for (int a = 0; a < 3; ++a) {
                fsrc[t][k] = xyz[a];
                fcoef[t][k++] = m[3 * row(s0) + (uint32_t)a];
            }
        } else {
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    fsrc[t][k] = xyz[a] | (xyz[b] << 2);
                    fcoef[t][k++] = m[3 * row(s0) + (uint32_t)a] * m[3 * row(s1) + (uint32_t)b];
                }
        }
        for (; k < 9; ++k) {
            fsrc[t][k] = t;
            fcoef[t][k] = 0.0;
        }
    }
    __syncthreads();
    const long long t0 = clock64();
    if constexpr (PATTERN == 4) {
        const uint32_t slot = lane & 15u, base = lane & 16u;
        for (int64_t it = 0; it < passes; it += 2) {
            double val[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) val[k] = __shfl_sync(0xffffffffu, v, base | fsrc[slot][k]);
            double acc = fcoef[slot][0] * val[0];
#pragma unroll
            for (int k = 1; k < 9; ++k) acc = fma(fcoef[slot][k], val[k], acc);
            v = acc;
        }
    } else if constexpr (PATTERN < 3) {
        int layout = 0;
        for (int64_t it = 0; it < passes; ++it) {
            if (PATTERN >= 1 && (it & 1) == 0) {
                double *b = buf[(it >> 1) & 1];
                b[probe_idx(t, layout)] = v;
                __syncthreads();
                uint32_t j = probe_idx(t, layout ^ 1), neg = 0;
                if (PATTERN == 2 && (it & 3) == 0) j = pull_recs(j, 4, recs, 4, neg);
                v = flip(b[j], neg);
                layout ^= 1;
            }
            probe_lane_pass(v, lane, 2 * (int)(it & 1), m);
        }
    } else {
        const uint32_t i0 = lane | (w << 6), i1 = i0 | 32u;
        for (int64_t it = 0; it < passes; it += 4) {
            probe_lane_pass(v, lane, 0, m);
            probe_lane_pass(v1, lane, 0, m);
            probe_lane_pass(v, lane, 2, m);
            probe_lane_pass(v1, lane, 2, m);
            {   // lane bit 4 = x, the register = z
                const double o0 = __shfl_xor_sync(0xffffffffu, v, 16);
                const double o1 = __shfl_xor_sync(0xffffffffu, v1, 16);
                const bool xl = (lane >> 4) & 1u;
                const double X = xl ? v : o0, Y = xl ? v1 : o1, Z = xl ? o1 : v1;
                if (xl) v = probe_row(m, 1u, X, Y, Z);
                v1 = probe_row(m, xl ? 2u : 3u, X, Y, Z);
            }
            double *b = buf[(it >> 2) & 1];
            b[i0] = v;
            b[i1] = v1;
            __syncthreads();
            uint32_t n0 = 0, n1 = 0;
            const uint32_t j0 = pull_recs(i0, 4, recs, 4, n0), j1 = pull_recs(i1, 4, recs, 4, n1);
            // the fourth wire (bits 6 = z, 7 = x) at the pulled positions
            const uint32_t g0 = j0 & 63u, s0 = (j0 >> 6) & 3u, g1 = j1 & 63u, s1 = (j1 >> 6) & 3u;
            const double x0 = b[g0 | 128u], y0 = b[g0 | 192u], z0 = b[g0 | 64u], e0 = b[g0];
            const double x1 = b[g1 | 128u], y1 = b[g1 | 192u], z1 = b[g1 | 64u], e1 = b[g1];
            // slot code (bit 0 = z, bit 1 = x): 0 I, 1 Z, 2 X, 3 Y -> map row X 1, Y 2, Z 3
            v = flip(s0 ? probe_row(m, s0 == 2u ? 1u : (s0 == 3u ? 2u : 3u), x0, y0, z0) : e0, n0);
            v1 = flip(s1 ? probe_row(m, s1 == 2u ? 1u : (s1 == 3u ? 2u : 3u), x1, y1, z1) : e1, n1);
        }
    }
    const long long t1 = clock64();
    // never true for a rotation's bounded values; keeps the loop live
    if (v + v1 == -1e300) sink[t] = v;
    if (t == 0) clk[0] = t1 - t0;
}

}  // namespace

}  // namespace stab

using namespace stab;

extern "C" int stab_probe_pass(int pattern, int threads, int64_t passes, double *clk_per_pass) {
    if (!clk_per_pass || pattern < 0 || pattern > 4 || (threads != 128 && threads != 256) ||
        (pattern == 3 && threads != 128))
        return STAB_E_INVAL;
    if (passes < 4 || passes > ((int64_t)1 << 24) || passes % 4 != 0) return STAB_E_RANGE;
    cudaStream_t st = nullptr;
    double *dm = nullptr, *sink = nullptr;
    long long *dclk = nullptr;
    long long hclk = 0;
    // a rotation by 0.7 rad about the third axis
    const double c = std::cos(0.7), s = std::sin(0.7);
    const double hm[9] = {c, -s, 0.0, s, c, 0.0, 0.0, 0.0, 1.0};
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dm, sizeof hm, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&sink, 256 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dclk, sizeof(long long), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dm, hm, sizeof hm, cudaMemcpyHostToDevice, st);
    auto launch = [&](int64_t n) {
        switch (pattern) {
        case 0: k_probe_pass<0><<<1, threads, 0, st>>>(n, dm, sink, dclk); break;
        case 1: k_probe_pass<1><<<1, threads, 0, st>>>(n, dm, sink, dclk); break;
        case 2: k_probe_pass<2><<<1, threads, 0, st>>>(n, dm, sink, dclk); break;
        case 3: k_probe_pass<3><<<1, threads, 0, st>>>(n, dm, sink, dclk); break;
        default: k_probe_pass<4><<<1, threads, 0, st>>>(n, dm, sink, dclk); break;
        }
        return cudaGetLastError();
    };
    if (e == cudaSuccess) e = launch(4);        // warm-up: code loaded
    if (e == cudaSuccess) e = launch(passes);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hclk, dclk, sizeof hclk, cudaMemcpyDeviceToHost, st);
    if (dm) cudaFreeAsync(dm, st);
    if (sink) cudaFreeAsync(sink, st);
    if (dclk) cudaFreeAsync(dclk, st);
    const cudaError_t e2 = st ? cudaStreamSynchronize(st) : cudaSuccess;
    if (st) cudaStreamDestroy(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        record_cuda_error(e);
        return STAB_E_CUDA;
    }
    *clk_per_pass = (double)hclk / (double)passes;
    return STAB_OK;
}

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
