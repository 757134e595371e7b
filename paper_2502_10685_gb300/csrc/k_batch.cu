// k_batch.cu -- one persistent launch over many uneven circuits.
//
// Every unit is one vector of one circuit: a generator Z_k of a circuit whose
// generators are wanted, or the observable of a circuit whose <O> is wanted
// (all 2m parameter-shift copies of a circuit are such units).  Each CTA
// takes units from a device counter, longest first (the host sorts them),
// and runs the unit's instruction stream exactly like the single-circuit
// resident kernels: n <= 4 with a lane quad per group, n = 5, 6 with a lane
// per group, the vector in shared memory; n = 7, 8 with the vector pair in
// the CTA's slab of global memory (it stays in L2 while the CTA works on it).
#include <cuda_runtime.h>

#include "resident.cuh"

namespace stab {

namespace {

using namespace resident;

constexpr int kBatchThreads = 256;

template <int N>
__device__ void batch_unit(const BatchUnit &U, int n_chunks, int smem_n, Stager &st,
                           unsigned char *smem, double *slab, int32_t *status, bool &ok) {
    constexpr int E = 1 << (2 * N);
    constexpr int LPG = N <= 4 ? 4 : 1;
    double *red = reinterpret_cast<double *>(smem + kOffRed);
    // the launch's shared memory holds vectors up to smem_n qubits (chosen by
    // the batch's autotuner); larger ones live in the CTA's slab
    double *bufA = (N <= kMaxResidentQubits && N <= smem_n)
                       ? reinterpret_cast<double *>(smem + kSmemHeader)
                       : slab;
    double *bufB = bufA + E;
    st.s0 = U.stream;
    st.s1 = nullptr;
    st.n0 = n_chunks;
    st.n_total = n_chunks;
    st.restart();
    for (int i = threadIdx.x; i < E; i += kBatchThreads) {
        double v = 0.0;
        if (U.init == INIT_RHO0) v = (i < (1 << N)) ? 1.0 : 0.0;
        bufA[i] = v;
    }
    __syncthreads();
    if (U.init == INIT_GENERATOR) {
        if (threadIdx.x == 0) bufA[1u << U.gen] = 1.0;
    } else if (U.init == INIT_TERMS) {
        for (int k = threadIdx.x; k < U.n_terms; k += kBatchThreads)
            bufA[U.terms[k].idx] = U.terms[k].coeff;
    }
    __syncthreads();
    double *res = run_stream<N, LPG, kBatchThreads>(st, 0, n_chunks, bufA, bufB, status);
    if (res == nullptr) {
        ok = false;
        return;
    }
    st.advance_phases();
    if (U.out) {
        for (int i = threadIdx.x; i < E; i += kBatchThreads) U.out[i] = res[i];
    }
    if (U.xfree_out) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < (1 << N); i += kBatchThreads) acc += res[i];
        const double total = block_sum<kBatchThreads>(acc, red);
        if (threadIdx.x == 0) *U.xfree_out = total;
    }
    __syncthreads();
}

// At least four CTAs per SM: with the thread bound alone ptxas settled on 48
// registers and spilled inside the pass loop; 4 gives 62 and no spills.
__global__ void __launch_bounds__(kBatchThreads, 4) k_batch(BatchArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_unit;
    Stager st;
    stager_setup(st, smem);
    st.n_total = 0;
    st.start();   // initialises the barriers (no chunk yet)
    double *slab = a.slab ? a.slab + (size_t)blockIdx.x * a.slab_doubles : nullptr;
    bool ok = true;
    while (ok) {
        if (threadIdx.x == 0) s_unit = atomicAdd(a.counter, 1);
        __syncthreads();
        const int u = s_unit;
        __syncthreads();
        if (u >= a.n_units) break;
        const BatchUnit U = a.units[u];
        const int nc = (a.max_chunks > 0 && U.n_chunks > a.max_chunks) ? a.max_chunks : U.n_chunks;
        const int sn = a.smem_n > 0 ? a.smem_n : kMaxResidentQubits;
        switch (U.n) {
        case 1: batch_unit<1>(U, nc, sn, st, smem, slab, a.status, ok); break;
        case 2: batch_unit<2>(U, nc, sn, st, smem, slab, a.status, ok); break;
        case 3: batch_unit<3>(U, nc, sn, st, smem, slab, a.status, ok); break;
        case 4: batch_unit<4>(U, nc, sn, st, smem, slab, a.status, ok); break;
        case 5: batch_unit<5>(U, nc, sn, st, smem, slab, a.status, ok); break;
        case 6: batch_unit<6>(U, nc, sn, st, smem, slab, a.status, ok); break;
        case 7: batch_unit<7>(U, nc, sn, st, smem, slab, a.status, ok); break;
        case 8: batch_unit<8>(U, nc, sn, st, smem, slab, a.status, ok); break;
        default: break;
        }
    }
}

}  // namespace

size_t batch_smem_bytes(int max_n_in_smem) {
    const int nn = max_n_in_smem < 1 ? 1 : max_n_in_smem;
    return kSmemHeader + 2 * (sizeof(double) << (2 * nn));
}

int batch_threads() { return kBatchThreads; }

cudaError_t batch_occupancy(size_t smem, int *ctas_per_sm) {
    static SmemLimit lim;
    cudaError_t e = raise_smem_limit(k_batch, smem, lim);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_batch, kBatchThreads,
                                                         smem);
}

// batch_occupancy() sets the kernel's shared-memory limit before the first launch.
cudaError_t launch_batch(const BatchArgs &a, int grid, size_t smem, cudaStream_t s) {
    k_batch<<<grid, kBatchThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace stab
