// k_decode.cu -- decoding the Pauli coefficients of a state into its density
// matrix (the paper's toDM() target, Sec. III-D and IV-C, Eq. (3)).
//
// rho = 2^-n sum_P r_P P with r the forward-evolved coefficients of
// 2^n |0><0|.  A string P(x, z) has one nonzero per row (Sec. III-D):
// <a| P |b> = i^{|x & z|} (-1)^{z . b} when a = b ^ x.  Hence, for each x,
//     rho[b ^ x][b] = 2^-n sum_z r(x, z) i^{|x & z|} (-1)^{z . b},
// a Walsh-Hadamard transform over z of the contiguous block r(x, .) (index
// z | x << n).  One CTA per x: phases, an in-place transform in shared memory
// (n butterfly stages of additions), and a scatter into column b of row b ^ x.
#include <cuda_runtime.h>

#include "launch.h"

namespace stab {

namespace {

constexpr int kDecodeThreads = 256;

__global__ void __launch_bounds__(kDecodeThreads) k_decode_rho(const double *__restrict__ r,
                                                               int n, double *__restrict__ rho) {
    extern __shared__ double sm[];
    const uint32_t D = 1u << n;
    double *re = sm, *im = sm + D;
    const uint32_t x = blockIdx.x;
    const double *rx = r + ((size_t)x << n);
    for (uint32_t z = threadIdx.x; z < D; z += blockDim.x) {
        const double v = rx[z];
        const uint32_t k = __popc(x & z) & 3u;   // i^k
        re[z] = (k == 0) ? v : (k == 2 ? -v : 0.0);
        im[z] = (k == 1) ? v : (k == 3 ? -v : 0.0);
    }
    __syncthreads();
    for (uint32_t h = 1; h < D; h <<= 1) {
        for (uint32_t t = threadIdx.x; t < D / 2; t += blockDim.x) {
            const uint32_t j = ((t & ~(h - 1)) << 1) | (t & (h - 1));   // bit h of j clear
            const double ur = re[j], vr = re[j | h], ui = im[j], vi = im[j | h];
            re[j] = ur + vr;
            re[j | h] = ur - vr;
            im[j] = ui + vi;
            im[j | h] = ui - vi;
        }
        __syncthreads();
    }
    const double scale = 1.0 / (double)D;
    for (uint32_t b = threadIdx.x; b < D; b += blockDim.x) {
        const size_t at = ((size_t)(b ^ x) * D + b) * 2;
        rho[at] = scale * re[b];
        rho[at + 1] = scale * im[b];
    }
}

}  // namespace

cudaError_t launch_decode_rho(const double *r, int n, double *rho, cudaStream_t st) {
    const size_t smem = 2 * (sizeof(double) << n);
    static SmemLimit lim;
    cudaError_t e = raise_smem_limit(k_decode_rho, smem, lim);
    if (e != cudaSuccess) return e;
    k_decode_rho<<<1u << n, kDecodeThreads, smem, st>>>(r, n, rho);
    return cudaGetLastError();
}

}  // namespace stab
