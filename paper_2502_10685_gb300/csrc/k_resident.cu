// k_resident.cu -- propagation with the whole 4^n coefficient vector resident
// in shared memory, one CTA per vector (n <= 7).
//
// The CTA walks the pass list of the loaded circuit (the Map stage of
// Sec. IV-B, sequential by nature) and applies each pass to its vector in
// place: a P_WIRE pass gives each thread whole groups of one wire and runs the
// wire's ops on them in registers (Table I rows, lifting form for rotations);
// a P_CLIFF pass pulls every entry through the pass's two-qubit Clifford
// permutation (map_CX of Sec. III-C and CZ).  Only rotations use the FP64 pipe.
#include <cuda_runtime.h>

#include "resident.cuh"

namespace stab {

template <int N>
__global__ void __launch_bounds__(RCfg<N>::T) k_resident(ResidentArgs a) {
    using C = RCfg<N>;
    extern __shared__ double smem[];
    double *vec = smem;
    double *red = smem + C::E;
    resident_init<N>(vec, a);
    resident_run<N>(vec, a.prog, a.inverse);
    if (a.out) {
        double *o = a.out + (size_t)blockIdx.x * C::E;
        for (int i = threadIdx.x; i < C::E; i += C::T) o[i] = vec[i];
    }
    if (a.xfree_out) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < (1 << N); i += C::T) acc += vec[i];
        double total = block_sum<C::T>(acc, red);
        if (threadIdx.x == 0) a.xfree_out[blockIdx.x] = total;
    }
}

template <int N>
static cudaError_t launch_resident_n(const ResidentArgs &a, cudaStream_t st) {
    using C = RCfg<N>;
    const size_t smem = (size_t)C::E * sizeof(double) + 32 * sizeof(double);
    static bool configured[64] = {};  // the attribute is set once per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(k_resident<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    k_resident<N><<<a.n_vec, C::T, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_resident(int n, const ResidentArgs &a, cudaStream_t st) {
    switch (n) {
    case 1: return launch_resident_n<1>(a, st);
    case 2: return launch_resident_n<2>(a, st);
    case 3: return launch_resident_n<3>(a, st);
    case 4: return launch_resident_n<4>(a, st);
    case 5: return launch_resident_n<5>(a, st);
    case 6: return launch_resident_n<6>(a, st);
    case 7: return launch_resident_n<7>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace stab
