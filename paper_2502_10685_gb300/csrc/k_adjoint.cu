// k_adjoint.cu -- adjoint (reverse-mode) gradient of <O> in the Pauli basis,
// streamed form (vectors in global memory; the shared-memory form is in
// k_resident.cu).
//
// With rho_0 the coefficient vector of 2^n |0><0| (1 on every string of I and
// Z) and M_j the orthogonal transfer map of gate j, <O> = <o, M_m ... M_1 rho_0>.
// Let r_j = M_j ... M_1 rho_0 and l_j = M_{j+1}^T ... M_m^T o.  For a rotation
// on a pair (u, v), d M_j / d theta = J M_j with J (u, v) = (-v, u), so
//     d<O>/d theta_j = sum over the gate's pairs of  l_u * (-r_v) + l_v * r_u
// evaluated on (l_j, r_j).  One reverse sweep carries l and r backward
// together (r_{j-1} = M_j^T r_j, exact up to rounding because every map is
// orthogonal), so no forward state is stored except r_m.
#include <cuda_runtime.h>

#include "device_ops.cuh"
#include "launch.h"

namespace stab {

namespace {

constexpr int R = kRotPerGradPass;

__device__ __forceinline__ double pair_dot(int axis, double lx, double ly, double lz, double rx,
                                           double ry, double rz) {
    // (u, v) = (Y, Z) for R_x, (Z, X) for R_y, (X, Y) for R_z
    if (axis == AX_X) return fma(lz, ry, -ly * rz);
    if (axis == AX_Y) return fma(lx, rz, -lz * rx);
    return fma(ly, rx, -lx * ry);
}

__device__ __forceinline__ uint64_t deposit_runs(uint64_t v, const BitRuns &r) {
    uint64_t out = 0;
    for (int k = 0; k < r.n; ++k)
        out |= ((v >> r.src[k]) & ((1ull << r.len[k]) - 1ull)) << r.dst[k];
    return out;
}

__device__ __forceinline__ void add_slot(double (&part)[R], int slot, double d) {
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (r == slot) part[r] += d;
}

// Walks one P_WIRE pass backward on a group: accumulates the gradient dot of
// every rotation into part[] (slot = rotation's position within the pass) and
// applies the inverse op to both vectors.
__device__ __forceinline__ void adjoint_group(const DevPass &p, const DevOp *ops,
                                              const DevMap3 *maps, double &lx, double &ly,
                                              double &lz, double &rx, double &ry, double &rz,
                                              double (&part)[R], int n_rot) {
    int slot = n_rot - 1;
    for (int j = p.n_ops - 1; j >= 0; --j) {
        const DevOp op = ops[p.first + j];
        if (op.kind == K_ROT) {
            add_slot(part, slot, pair_dot(op.axis, lx, ly, lz, rx, ry, rz));
            --slot;
        }
        apply_op1(lx, ly, lz, op, maps, 1);
        apply_op1(rx, ry, rz, op, maps, 1);
    }
}

// The same pass forward: each gate on both vectors, then (rotations) the dot
// at the post-gate pair; slots in op order.
__device__ __forceinline__ void adjoint_group_fwd(const DevPass &p, const DevOp *ops,
                                                  double &lx, double &ly, double &lz, double &rx,
                                                  double &ry, double &rz, double (&part)[R]) {
    int slot = 0;
    for (int j = 0; j < p.n_ops; ++j) {
        const DevOp op = ops[p.first + j];
        apply_op1(lx, ly, lz, op, nullptr, 0);
        apply_op1(rx, ry, rz, op, nullptr, 0);
        if (op.kind == K_ROT) {
            add_slot(part, slot, pair_dot(op.axis, lx, ly, lz, rx, ry, rz));
            ++slot;
        }
    }
}

__device__ __forceinline__ int count_rot(const DevPass &p, const DevOp *ops) {
    int c = 0;
    for (int j = 0; j < p.n_ops; ++j) c += ops[p.first + j].kind == K_ROT;
    return c;
}

// Gradient slot of the r-th rotation of a pass.
__device__ __forceinline__ int rot_gate(const DevPass &p, const DevOp *ops, int r) {
    for (int j = 0; j < p.n_ops; ++j) {
        if (ops[p.first + j].kind == K_ROT) {
            if (r == 0) return ops[p.first + j].gate;
            --r;
        }
    }
    return -1;
}

// ---------------------------------------------------------------- streamed

constexpr int kAdjThreads = 256;
constexpr int kAdjStagedOps = 96;   // ops of a tile group staged in shared memory (3 KiB)

__global__ void __launch_bounds__(kAdjThreads) k_adjoint_wire(double *lam, double *rho, int n,
                                                              DevPass p, const DevOp *ops,
                                                              double *partials, int forward) {
    __shared__ double red[(kAdjThreads / 32) * R];
    const int q = p.q;
    const uint64_t G = 1ull << (2 * n - 2);
    const uint64_t bx = 1ull << (n + q), bz = 1ull << q;
    const int n_rot = count_rot(p, ops);
    double part[R];
#pragma unroll
    for (int r = 0; r < R; ++r) part[r] = 0.0;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < G;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = group_base(g, n, q);
        double *L = lam + b, *Rh = rho + b;
        double lx = L[bx], ly = L[bx | bz], lz = L[bz];
        double rx = Rh[bx], ry = Rh[bx | bz], rz = Rh[bz];
        if (forward) adjoint_group_fwd(p, ops, lx, ly, lz, rx, ry, rz, part);
        else adjoint_group(p, ops, nullptr, lx, ly, lz, rx, ry, rz, part, n_rot);
        L[bx] = lx; L[bx | bz] = ly; L[bz] = lz;
        Rh[bx] = rx; Rh[bx | bz] = ry; Rh[bz] = rz;
    }
    if (n_rot == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // only the pass's rotations are reduced (n_rot is uniform over the grid)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r < n_rot) {
            double v = part[r];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp * R + r] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < n_rot) {
        double total = 0.0;
        for (int w = 0; w < kAdjThreads / 32; ++w) total += red[w * R + threadIdx.x];
        partials[(size_t)rot_gate(p, ops, threadIdx.x) * gridDim.x + blockIdx.x] = total;
    }
}

// Rotations of a tile group: the gradient dots a launch accumulates.
int group_rotations(const TileGroup &tg) {
    int n_acc = 0;
    for (int j = 0; j < tg.n_pass; ++j) n_acc += tg.n_rot[j];
    return n_acc;
}

// Tile-fused adjoint sweep: up to kTileMaxPasses wire passes on at most
// kTileWires wires, applied backward (tg.inverse = 1; forward with 0) to the
// pair (lambda, rho) held as two shared-memory tiles (pair[0 .. 4^n) =
// lambda, pair[4^n ..) = rho).  The group's ops are staged in shared memory
// once per launch.  Each thread adds every rotation's gradient dot of its
// group to its own shared-memory accumulator (tile after tile), so the op
// chain carries no reduction; at the end each rotation's accumulators are
// summed over the threads in a fixed order and the result goes to
// partials[gate][block].
__global__ void __launch_bounds__(kAdjThreads) k_adjoint_tile(const double *src, double *pair,
                                                              int n, TileGroup tg,
                                                              const DevOp *ops,
                                                              double *partials) {
    extern __shared__ double sm[];
    const uint32_t T = 1u << tg.tile_bits;
    const int nt = (int)blockDim.x;
    double *tl = sm, *tr = sm + T;
    DevOp *sops = reinterpret_cast<DevOp *>(tr + T);                   // kAdjStagedOps
    uint32_t *offs = reinterpret_cast<uint32_t *>(sops + kAdjStagedOps);
    double *acc = reinterpret_cast<double *>(offs + T);                // rotations x threads
    __shared__ int s_first[kTileMaxPasses], s_nrot[kTileMaxPasses], s_rbase[kTileMaxPasses];
    __shared__ int s_staged, s_nacc;
    for (uint32_t e = threadIdx.x; e < T; e += blockDim.x)
        offs[e] = (uint32_t)deposit_runs(e, tg.tile_runs);
    if (threadIdx.x == 0) {
        int total = 0;
        for (int j = 0; j < tg.n_pass; ++j) total += tg.n_ops[j];
        s_staged = total <= kAdjStagedOps;
        int at = 0, rb = 0;
        for (int j = 0; j < tg.n_pass; ++j) {
            s_first[j] = s_staged ? at : (int)tg.first[j];
            at += tg.n_ops[j];
            s_nrot[j] = tg.n_rot[j];
            s_rbase[j] = rb;
            rb += tg.n_rot[j];
        }
        s_nacc = rb;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < s_nacc * nt; k += blockDim.x) acc[k] = 0.0;
    __syncthreads();
    const bool staged = s_staged != 0;
    if (staged) {
        int at = 0;
        for (int j = 0; j < tg.n_pass; ++j) {
            for (int k = threadIdx.x; k < (int)tg.n_ops[j]; k += blockDim.x)
                sops[at + k] = ops[tg.first[j] + k];
            at += tg.n_ops[j];
        }
    }
    __syncthreads();
    const DevOp *pops = staged ? sops : ops;
    const uint64_t E = 1ull << (2 * n);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t tiles = 1ull << tg.rest_bits;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t base = deposit_runs(t, tg.rest_runs);
        if (tg.pull_n == 0) {
            for (uint32_t e = threadIdx.x; e < T; e += blockDim.x) {
                tl[e] = src[base + offs[e]];
                tr[e] = src[E + base + offs[e]];
            }
        } else {
            // the Clifford gather that precedes the group, on both vectors
            for (uint32_t e = threadIdx.x; e < T; e += blockDim.x) {
                uint32_t neg = 0;
                const uint64_t j = pull_pass(base + offs[e], n, ops + tg.pull_first, tg.pull_n,
                                             tg.pull_inverse, neg);
                tl[e] = flip(src[j], neg);
                tr[e] = flip(src[E + j], neg);
            }
        }
        __syncthreads();
        for (int j = 0; j < tg.n_pass; ++j) {
            const int lz = tg.lz[j], lx = tg.lx[j];
            const int lo = lz < lx ? lz : lx, hi = lz < lx ? lx : lz;
            const uint32_t bz = 1u << lz, bx = 1u << lx;
            const int n_ops = tg.n_ops[j];
            const DevOp *po = pops + s_first[j];
            const int n_rot = s_nrot[j];
            double *my_acc = acc + (size_t)s_rbase[j] * nt + threadIdx.x;
            // one group per thread (the launch has T / 4 threads): each
            // rotation's dot is added to this thread's own shared-memory
            // accumulator (my_acc); every rotation is summed over the threads
            // once, in a fixed order, at the end of the launch
            const uint32_t g = threadIdx.x;
            const bool live = g < T / 4;
            uint32_t b = ((g >> lo) << (lo + 1)) | (g & ((1u << lo) - 1u));
            b = ((b >> hi) << (hi + 1)) | (b & ((1u << hi) - 1u));
            double lx_ = 0.0, ly_ = 0.0, lz_ = 0.0, rx_ = 0.0, ry_ = 0.0, rz_ = 0.0;
            if (live) {
                lx_ = tl[b | bx]; ly_ = tl[b | bx | bz]; lz_ = tl[b | bz];
                rx_ = tr[b | bx]; ry_ = tr[b | bx | bz]; rz_ = tr[b | bz];
            }
            if (tg.inverse) {
                // reverse sweep: the dot at the post-gate pair, then the inverse gate
                int slot = n_rot - 1;
                for (int k = n_ops - 1; k >= 0; --k) {
                    const DevOp op = po[k];
                    if (op.kind == K_ROT) {
                        my_acc[slot * nt] += pair_dot(op.axis, lx_, ly_, lz_, rx_, ry_, rz_);
                        --slot;
                    }
                    apply_op1(lx_, ly_, lz_, op, nullptr, 1);
                    apply_op1(rx_, ry_, rz_, op, nullptr, 1);
                }
            } else {
                // forward sweep (both vectors carried forward, the maps being
                // orthogonal): the gate, then the dot at the post-gate pair
                int slot = 0;
                for (int k = 0; k < n_ops; ++k) {
                    const DevOp op = po[k];
                    apply_op1(lx_, ly_, lz_, op, nullptr, 0);
                    apply_op1(rx_, ry_, rz_, op, nullptr, 0);
                    if (op.kind == K_ROT) {
                        my_acc[slot * nt] += pair_dot(op.axis, lx_, ly_, lz_, rx_, ry_, rz_);
                        ++slot;
                    }
                }
            }
            if (live) {
                tl[b | bx] = lx_; tl[b | bx | bz] = ly_; tl[b | bz] = lz_;
                tr[b | bx] = rx_; tr[b | bx | bz] = ry_; tr[b | bz] = rz_;
            }
            __syncthreads();
        }
        for (uint32_t e = threadIdx.x; e < T; e += blockDim.x) {
            pair[base + offs[e]] = tl[e];
            pair[E + base + offs[e]] = tr[e];
        }
        __syncthreads();
    }
    // rotation r (pass j, slot r - s_rbase[j]) by warp r mod warps: each lane
    // sums its threads' accumulators in order, then a fixed shuffle tree
    const int nw = nt >> 5;
    for (int r = warp; r < s_nacc; r += nw) {
        double total = 0.0;
        for (int t = lane; t < nt; t += 32) total += acc[(size_t)r * nt + t];
        for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
        if (lane == 0) {
            int j = 0;
            while (j + 1 < tg.n_pass && s_rbase[j + 1] <= r) ++j;
            DevPass p{};
            p.n_ops = tg.n_ops[j];
            p.first = s_first[j];
            partials[(size_t)rot_gate(p, pops, r - s_rbase[j]) * gridDim.x + blockIdx.x] = total;
        }
    }
}

__global__ void k_reduce_partials(const double *partials, int n_rot, int n_blocks,
                                  double *grad_rot) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rot) return;
    double acc = 0.0;
    for (int b = 0; b < n_blocks; ++b) acc += partials[(size_t)r * n_blocks + b];
    grad_rot[r] = acc;
}

__global__ void k_gather_grads(const double *grad_rot, const int32_t *param_ptr,
                               const int32_t *param_rot, int n_params, double *grads) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_params) return;
    double acc = 0.0;
    for (int k = param_ptr[p]; k < param_ptr[p + 1]; ++k) acc += grad_rot[param_rot[k]];
    grads[p] = acc;
}

}  // namespace

int adjoint_stream_blocks(int n) {
    if (n <= kAdjTileMaxN) {
        // tile-fused sweep: one tile of 2^kAdjTileBits entries per CTA
        const int bits = 2 * n - kAdjTileBits;
        return bits > 0 ? 1 << bits : 1;
    }
    const long long G = 1ll << (2 * n - 2);
    long long b = (G + kAdjThreads - 1) / kAdjThreads;
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_adjoint_wire(double *lam, double *rho, int n, const DevPass &p,
                                const DevOp *ops, double *partials, int forward,
                                cudaStream_t st) {
    k_adjoint_wire<<<adjoint_stream_blocks(n), kAdjThreads, 0, st>>>(lam, rho, n, p, ops,
                                                                      partials, forward);
    return cudaGetLastError();
}

namespace {

int adjoint_tile_threads(int tile_bits) {
    int threads = (int)((1u << tile_bits) / 4);
    if (threads > kAdjThreads) threads = kAdjThreads;
    if (threads < 32) threads = 32;
    return threads;
}

}  // namespace

size_t adjoint_tile_smem(int tile_bits, int n_rot) {
    const size_t T = (size_t)1 << tile_bits;
    return 2 * T * sizeof(double) + kAdjStagedOps * sizeof(DevOp) + T * sizeof(uint32_t) +
           (size_t)n_rot * adjoint_tile_threads(tile_bits) * sizeof(double);
}

cudaError_t launch_adjoint_tile(const double *src_pair, double *dst_pair, int n,
                                const TileGroup &tg, const DevOp *ops, double *partials,
                                cudaStream_t st) {
    static SmemLimit lim;
    const size_t smem = adjoint_tile_smem(tg.tile_bits, group_rotations(tg));
    cudaError_t e = raise_smem_limit(k_adjoint_tile, smem, lim);
    if (e != cudaSuccess) return e;
    k_adjoint_tile<<<adjoint_stream_blocks(n), adjoint_tile_threads(tg.tile_bits), smem, st>>>(
        src_pair, dst_pair, n, tg, ops, partials);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double *partials, int n_rot, int n_blocks,
                                   double *grad_rot, cudaStream_t st) {
    if (n_rot == 0) return cudaSuccess;
    k_reduce_partials<<<(n_rot + 127) / 128, 128, 0, st>>>(partials, n_rot, n_blocks, grad_rot);
    return cudaGetLastError();
}

cudaError_t launch_gather_grads(const double *grad_rot, const int32_t *param_ptr,
                                const int32_t *param_rot, int n_params, double *grads,
                                cudaStream_t st) {
    if (n_params == 0) return cudaSuccess;
    k_gather_grads<<<(n_params + 127) / 128, 128, 0, st>>>(grad_rot, param_ptr, param_rot,
                                                           n_params, grads);
    return cudaGetLastError();
}

}  // namespace stab
