// resident.cuh -- building blocks of the shared-memory-resident kernels: a
// CTA holds one 4^n coefficient vector in shared memory and applies passes to
// it in place.
#pragma once

#include <cuda_runtime.h>

#include "device_ops.cuh"
#include "launch.h"

namespace stab {

template <int N>
struct RCfg {
    static constexpr int E = 1 << (2 * N);   // coefficients per vector
    static constexpr int G = E / 4;          // groups of one wire
    static constexpr int T = G < 32 ? 32 : (G > 1024 ? 1024 : G);
    static constexpr int GPT = (G + T - 1) / T;
    static constexpr int EPT = (E + T - 1) / T;
};

// Deterministic block sum (fixed order for a fixed block size).
template <int T>
__device__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double total = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (T + 31) / 32; ++w) total += red[w];
    }
    return total;
}

template <int N>
__device__ void resident_init(double *vec, const ResidentArgs &a) {
    using C = RCfg<N>;
    const int b = blockIdx.x;
    for (int i = threadIdx.x; i < C::E; i += C::T) {
        double v = 0.0;
        if (a.init == INIT_RHO0) v = (i < (1 << N)) ? 1.0 : 0.0;
        else if (a.init == INIT_LOAD) v = a.in[(size_t)b * C::E + i];
        vec[i] = v;
    }
    __syncthreads();
    if (a.init == INIT_GENERATOR) {
        if (threadIdx.x == 0) vec[1u << b] = 1.0;   // Z_b: z bit b set
    } else if (a.init == INIT_TERMS) {
        for (int k = threadIdx.x; k < a.n_terms; k += C::T) vec[a.terms[k].idx] = a.terms[k].coeff;
    }
    __syncthreads();
}

// One P_WIRE pass on a shared-memory vector.
template <int N>
__device__ __forceinline__ void resident_wire(double *vec, const DevPass &p, const DevOp *ops,
                                              const DevMap3 *maps, int inverse) {
    using C = RCfg<N>;
    const int q = p.q;
    double x[C::GPT], y[C::GPT], z[C::GPT];
    uint32_t base[C::GPT];
#pragma unroll
    for (int k = 0; k < C::GPT; ++k) {
        const int g = threadIdx.x + k * C::T;
        base[k] = (uint32_t)group_base((uint64_t)g, N, q);
        if (g < C::G) {
            x[k] = vec[base[k] | (1u << (N + q))];
            y[k] = vec[base[k] | (1u << (N + q)) | (1u << q)];
            z[k] = vec[base[k] | (1u << q)];
        }
    }
    const int n_ops = p.n_ops;
    for (int j = 0; j < n_ops; ++j) {
        const DevOp op = ops[p.first + (inverse ? n_ops - 1 - j : j)];
#pragma unroll
        for (int k = 0; k < C::GPT; ++k) apply_op1(x[k], y[k], z[k], op, maps, inverse);
    }
#pragma unroll
    for (int k = 0; k < C::GPT; ++k) {
        const int g = threadIdx.x + k * C::T;
        if (g < C::G) {
            vec[base[k] | (1u << (N + q))] = x[k];
            vec[base[k] | (1u << (N + q)) | (1u << q)] = y[k];
            vec[base[k] | (1u << q)] = z[k];
        }
    }
}

// One P_CLIFF pass: pull every entry through the pass's signed permutation.
template <int N>
__device__ __forceinline__ void resident_cliff(double *vec, const DevPass &p, const DevOp *ops,
                                               int inverse) {
    using C = RCfg<N>;
    double v[C::EPT];
#pragma unroll
    for (int k = 0; k < C::EPT; ++k) {
        const int i = threadIdx.x + k * C::T;
        if (i < C::E) {
            uint32_t neg = 0;
            uint64_t j = pull_pass((uint64_t)i, N, ops + p.first, p.n_ops, inverse, neg);
            v[k] = flip(vec[j], neg);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < C::EPT; ++k) {
        const int i = threadIdx.x + k * C::T;
        if (i < C::E) vec[i] = v[k];
    }
}

template <int N>
__device__ void resident_run(double *vec, const Program &prog, int inverse) {
    const int np = prog.n_passes;
    for (int s = 0; s < np; ++s) {
        const DevPass p = prog.passes[inverse ? np - 1 - s : s];
        if (p.type == P_WIRE) {
            resident_wire<N>(vec, p, prog.ops, prog.maps, inverse);
        } else {
            resident_cliff<N>(vec, p, prog.ops, inverse);
        }
        __syncthreads();
    }
}

}  // namespace stab
