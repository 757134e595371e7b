// launch.h -- host-side launch wrappers of the library's kernels.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "stab_internal.h"

namespace stab {

constexpr int kMaxResidentQubits = 7;   // 4^7 doubles = 128 KiB of shared memory
constexpr int kMaxResidentAdjoint = 6;  // two vectors: 2 x 4^6 doubles = 64 KiB
constexpr int kRotPerGradPass = 8;      // rotations per P_WIRE pass in gradient plans

struct ResidentArgs {
    Program prog;
    int32_t inverse;         // 0: forward (U P U^dagger), 1: backward (U^dagger P U)
    int32_t init;            // InitMode
    const DevTerm *terms;    // INIT_TERMS
    int32_t n_terms;
    int32_t n_vec;           // vectors (blocks)
    const double *in;        // INIT_LOAD: block b reads in + b * 4^n
    double *out;             // final vector of block b at out + b * 4^n (may be null)
    double *xfree_out;       // block b: sum of its x-free coefficients (may be null)
};

// Encode kernel: lifting coefficients of every rotation op and composed 3x3
// maps, from the angle array on the device.
cudaError_t launch_encode(DevOp *ops, int n_ops, DevMap3 *maps, int n_maps,
                          const int32_t *map_gate_idx, const RawGate *gates, const double *thetas,
                          cudaStream_t st);

// Shared-memory-resident propagation, one CTA per vector (n <= 7).
cudaError_t launch_resident(int n, const ResidentArgs &a, cudaStream_t st);

// Streamed passes over n_vec vectors of 4^n doubles in global memory.
cudaError_t launch_fill(double *vec, int n, int n_vec, int init, const DevTerm *terms,
                        int n_terms, cudaStream_t st);
cudaError_t launch_stream_wire(double *vec, int n, int n_vec, const DevPass &p, const DevOp *ops,
                               const DevMap3 *maps, int inverse, cudaStream_t st);
cudaError_t launch_stream_cliff(const double *src, double *dst, int n, int n_vec,
                                const DevPass &p, const DevOp *ops, int inverse, cudaStream_t st);
cudaError_t launch_xfree_sum(const double *vec, int n, int n_vec, double *out, cudaStream_t st);

// Adjoint gradient.
struct AdjointArgs {
    Program prog;              // gradient plan: no K_MAP3, <= kRotPerGradPass rotations per pass
    const DevTerm *terms;
    int32_t n_terms;
    double *grad_rot;          // one entry per rotation ordinal
    double *expect_out;        // <O>
};
cudaError_t launch_adjoint_resident(int n, const AdjointArgs &a, cudaStream_t st);

// Streamed adjoint pieces.
int adjoint_stream_blocks(int n);
cudaError_t launch_adjoint_wire(double *lam, double *rho, int n, const DevPass &p,
                                const DevOp *ops, double *partials, int rot_base, int n_rot_total,
                                cudaStream_t st);
cudaError_t launch_reduce_partials(const double *partials, int n_rot, int n_blocks,
                                   double *grad_rot, cudaStream_t st);
cudaError_t launch_gather_grads(const double *grad_rot, const int32_t *param_ptr,
                                const int32_t *param_rot, int n_params, double *grads,
                                cudaStream_t st);

}  // namespace stab
