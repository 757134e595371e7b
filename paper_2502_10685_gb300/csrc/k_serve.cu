// k_serve.cu -- the serving iteration kernel: one persistent launch advances
// every admitted request by a slice of its instruction streams.
//
// A request evaluated by the server is a few units, each a vector (or an
// adjoint pair of vectors) that walks one instruction stream: the observable
// backward through the circuit for <O>; for a gradient, rho_0 forward through
// the first half of the passes and O backward through the second half, then
// the pair (lambda, rho) met at the cut backward through the first half and
// forward through the second, taking each rotation's dot.  Between launches a
// unit's vectors stay in the request's own device memory, so requests join
// and leave at slice boundaries while others are in flight.  Chunk
// boundaries of a stream are valid places to stop: no pass straddles a chunk
// and every chunk carries the pulls of its own passes.
//
// Each CTA takes units from a counter (the host orders them by the work of
// their slices, largest first).  A unit whose buffers fit the launch's shared
// memory loads its vectors there at the start of the slice and stores them
// back at the end; larger ones (with the server's default 32 KiB budget:
// vectors and pairs of n = 6, and n = 7, 8 when the engine takes them) work
// on the request's own buffers in global memory, which stay in L2 while the
// CTA works on them.  The pass code is the one of the resident and batch
// kernels.
#include <cuda_runtime.h>

#include "resident.cuh"

namespace stab {

namespace {

using namespace resident;

constexpr int kServeThreads = 256;

__device__ __forceinline__ void copy_vec(double *dst, const double *src, int E) {
    if (dst == src) return;
    for (int i = threadIdx.x; i < E; i += kServeThreads) dst[i] = src[i];
}

template <int N>
__device__ void serve_vec(const ServeUnit &U, int smem_buf, Stager &st, unsigned char *smem,
                          int32_t *status, bool &ok) {
    constexpr int E = 1 << (2 * N);
    double *red = reinterpret_cast<double *>(smem + kOffRed);
    const bool in_smem = 2 * E * (int)sizeof(double) <= smem_buf;
    double *bufA = in_smem ? reinterpret_cast<double *>(smem + kSmemHeader) : U.state;
    double *bufB = bufA + E;
    if (U.init == INIT_LOAD) {
        copy_vec(bufA, U.src, E);
    } else {
        for (int i = threadIdx.x; i < E; i += kServeThreads)
            bufA[i] = (U.init == INIT_RHO0 && i < (1 << N)) ? 1.0 : 0.0;
        __syncthreads();
        if (U.init == INIT_TERMS)
            for (int k = threadIdx.x; k < U.n_terms; k += kServeThreads)
                bufA[U.terms[k].idx] = U.terms[k].coeff;
    }
    __syncthreads();
    double *res;
    if constexpr (N <= 4) {
        // rows streams (one 3x3 map per wire pass) need the lane-quad loop
        res = (U.flags & SF_ROWS) ? run_stream<N, 4, kServeThreads>(st, 0, U.n_chunks, bufA, bufB,
                                                                    status)
                                  : run_stream<N, 1, kServeThreads>(st, 0, U.n_chunks, bufA, bufB,
                                                                    status);
    } else {
        res = run_stream<N, 1, kServeThreads>(st, 0, U.n_chunks, bufA, bufB, status);
    }
    if (res == nullptr) {
        ok = false;
        return;
    }
    st.advance_phases();
    copy_vec(U.state, res, E);
    if ((U.flags & SF_LAST) && U.xfree_out) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < (1 << N); i += kServeThreads) acc += res[i];
        const double total = block_sum<kServeThreads>(acc, red);
        if (threadIdx.x == 0) *U.xfree_out = total;
    }
    __syncthreads();
}

template <int N>
__device__ void serve_pair(const ServeUnit &U, int smem_buf, Stager &st, unsigned char *smem,
                           int32_t *status, bool &ok) {
    constexpr int E = 1 << (2 * N);
    double *red = reinterpret_cast<double *>(smem + kOffRed);
    const bool in_smem = 4 * E * (int)sizeof(double) <= smem_buf;
    double *lam = in_smem ? reinterpret_cast<double *>(smem + kSmemHeader) : U.state;
    double *rho = lam + E, *lam_n = rho + E, *rho_n = lam_n + E;
    copy_vec(lam, U.src, E);
    copy_vec(rho, U.src2, E);
    __syncthreads();
    if (!adjoint_sweep<N, kServeThreads>(st, 0, U.n_chunks, lam, lam_n, rho, rho_n, U.grad_rot,
                                         status, smem, U.kind == SV_PAIR_FWD)) {
        ok = false;
        return;
    }
    st.advance_phases();
    copy_vec(U.state, lam, E);
    copy_vec(U.state + E, rho, E);
    if ((U.flags & SF_LAST) && U.xfree_out) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < (1 << N); i += kServeThreads) acc += lam[i];
        const double total = block_sum<kServeThreads>(acc, red);
        if (threadIdx.x == 0) *U.xfree_out = total;
    }
    __syncthreads();
}

template <int N>
__device__ void serve_unit(const ServeUnit &U, int smem_buf, Stager &st, unsigned char *smem,
                           int32_t *status, bool &ok) {
    st.s0 = U.stream;
    st.s1 = nullptr;
    st.n0 = U.n_chunks;
    st.n_total = U.n_chunks;
    st.restart();
    if (U.kind == SV_VEC) serve_vec<N>(U, smem_buf, st, smem, status, ok);
    else serve_pair<N>(U, smem_buf, st, smem, status, ok);
}

// Three CTAs per SM: 80 registers, enough for every unit form without
// spilling (at four CTAs per SM the 64-register bound spilled, and the n <= 8
// serving trace ran about 8 % slower).
__global__ void __launch_bounds__(kServeThreads, 3) k_serve(ServeArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_unit;
    Stager st;
    stager_setup(st, smem);
    st.n_total = 0;
    st.start();   // initialises the barriers (no chunk yet)
    bool ok = true;
    while (ok) {
        if (threadIdx.x == 0) s_unit = atomicAdd(a.counter, 1);
        __syncthreads();
        const int u = s_unit;
        __syncthreads();
        if (u >= a.n_units) break;
        const ServeUnit U = a.units[u];
        const long long t0 = clock64();
        switch (U.n) {
        case 1: serve_unit<1>(U, a.smem_buf, st, smem, a.status, ok); break;
        case 2: serve_unit<2>(U, a.smem_buf, st, smem, a.status, ok); break;
        case 3: serve_unit<3>(U, a.smem_buf, st, smem, a.status, ok); break;
        case 4: serve_unit<4>(U, a.smem_buf, st, smem, a.status, ok); break;
        case 5: serve_unit<5>(U, a.smem_buf, st, smem, a.status, ok); break;
        case 6: serve_unit<6>(U, a.smem_buf, st, smem, a.status, ok); break;
        case 7: serve_unit<7>(U, a.smem_buf, st, smem, a.status, ok); break;
        case 8: serve_unit<8>(U, a.smem_buf, st, smem, a.status, ok); break;
        default: break;
        }
        // the slice's length, for the host's estimate of what a chunk of this
        // kind of unit costs (every thread has passed the slice's last barrier)
        if (a.unit_cycles && threadIdx.x == 0) a.unit_cycles[u] = (int64_t)(clock64() - t0);
    }
}

}  // namespace

size_t serve_smem_bytes(int smem_buf) { return kSmemHeader + (size_t)(smem_buf > 0 ? smem_buf : 0); }

cudaError_t serve_occupancy(size_t smem, int *ctas_per_sm) {
    static SmemLimit lim;
    cudaError_t e = raise_smem_limit(k_serve, smem, lim);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_serve, kServeThreads, smem);
}

// serve_occupancy() sets the kernel's shared-memory limit before the first launch.
cudaError_t launch_serve(const ServeArgs &a, int grid, size_t smem, cudaStream_t s) {
    k_serve<<<grid, kServeThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace stab
