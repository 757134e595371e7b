// k_stream.cu -- angle encoding and the streamed (HBM-resident) passes.
//
// Streamed passes keep the vectors in global memory and apply one fused pass
// per launch to every vector of the batch: a P_WIRE pass reads each group of
// the pass's wire once, runs all of the wire's ops on it in registers and
// writes it back in place; a P_CLIFF pass gathers every entry through the
// pass's signed permutation into a second buffer.
#include <cuda_runtime.h>

#include "device_ops.cuh"
#include "launch.h"
#include "tma.cuh"

namespace stab {

namespace {

constexpr int kThreads = 256;

int grid_for(uint64_t work, int threads) {
    uint64_t b = (work + threads - 1) / threads;
    const uint64_t cap = 152ull * 16ull;  // grid-stride beyond 16 CTAs per SM
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// 3x3 maps on the (X, Y, Z) coefficients of one wire (new = M old), Table I
// rows; Clifford gates as signed permutation matrices.
__device__ void gate_matrix3(const RawGate &g, const double *thetas, double M[9]) {
    for (int k = 0; k < 9; ++k) M[k] = 0.0;
    double c = 1.0, s = 0.0;
    if (g.op >= 8) sincos(thetas[g.param], &s, &c);
    switch (g.op) {
    case 0:  // H: X <- Z, Y <- -Y, Z <- X
        M[2] = 1.0; M[4] = -1.0; M[6] = 1.0; break;
    case 1:  // S: X <- -Y, Y <- X
        M[1] = -1.0; M[3] = 1.0; M[8] = 1.0; break;
    case 2:  // Sdg: X <- Y, Y <- -X
        M[1] = 1.0; M[3] = -1.0; M[8] = 1.0; break;
    case 3:  // X: Y, Z negated
        M[0] = 1.0; M[4] = -1.0; M[8] = -1.0; break;
    case 4:  // Y: X, Z negated
        M[0] = -1.0; M[4] = 1.0; M[8] = -1.0; break;
    case 5:  // Z: X, Y negated
        M[0] = -1.0; M[4] = -1.0; M[8] = 1.0; break;
    case 8:  // RX: Y' = cY - sZ, Z' = sY + cZ
        M[0] = 1.0; M[4] = c; M[5] = -s; M[7] = s; M[8] = c; break;
    case 9:  // RY: X' = cX + sZ, Z' = -sX + cZ
        M[0] = c; M[2] = s; M[4] = 1.0; M[6] = -s; M[8] = c; break;
    case 10: // RZ: X' = cX - sY, Y' = sX + cY
        M[0] = c; M[1] = -s; M[3] = s; M[4] = c; M[8] = 1.0; break;
    default:
        M[0] = M[4] = M[8] = 1.0; break;
    }
}

// Shear coefficients of an angle: theta is reduced to phi in [-pi/2, pi/2] up
// to a factor R(pi) = -1 on the pair (neg), so that t = -tan(phi/2) stays in
// [-1, 1].
__device__ void shear_coeffs(double theta, double &t, double &s, uint16_t &neg) {
    const double two_pi = 6.283185307179586476925286766559;
    const double pi = 3.1415926535897932384626433832795;
    double phi = remainder(theta, two_pi);
    neg = 0;
    if (phi > 0.5 * pi) { phi -= pi; neg = 1; }
    else if (phi < -0.5 * pi) { phi += pi; neg = 1; }
    t = -tan(0.5 * phi);
    s = sin(phi);
}

// 3x3 product C = A B (row-major).
__device__ __forceinline__ void mul3(const double A[9], const double B[9], double C[9]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            C[3 * r + c] = fma(A[3 * r + 2], B[6 + c], fma(A[3 * r + 1], B[3 + c], A[3 * r] * B[c]));
}

// Composed map of every run, one warp per map: lane l composes a contiguous
// chunk of the run's gates in order (the lanes evaluate their gates' sin/cos
// at once), then the 32 partial products are multiplied in order by a
// shuffle tree (later chunk times earlier chunk), log2(32) steps instead of a
// sequential walk over the whole run.
__global__ void k_compose_maps(DevMap3 *maps, int n_maps, const int32_t *map_gate_idx,
                               const RawGate *gates, const double *thetas) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = (int)(threadIdx.x & 31u);
    if (w >= n_maps) return;   // whole warps
    const DevMap3 mp = maps[w];
    const int per = (mp.count + 31) / 32;
    const int k0 = min(lane * per, mp.count), k1 = min(k0 + per, mp.count);
    double M[9] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0};
    for (int k = k0; k < k1; ++k) {
        double G[9], R[9];
        gate_matrix3(gates[map_gate_idx[mp.first + k]], thetas, G);
        mul3(G, M, R);
#pragma unroll
        for (int j = 0; j < 9; ++j) M[j] = R[j];
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        double O[9], R[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) O[j] = __shfl_down_sync(0xffffffffu, M[j], d);
        if ((lane & (2 * d - 1)) == 0) {
            mul3(O, M, R);
#pragma unroll
            for (int j = 0; j < 9; ++j) M[j] = R[j];
        }
    }
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < 9; ++j) maps[w].m[j] = M[j];
}

// Composed map of every run, one thread per map walking its gates in order:
// the form for plans of short runs (a warp per map would idle most lanes).
__global__ void k_compose_maps_seq(DevMap3 *maps, int n_maps, const int32_t *map_gate_idx,
                                   const RawGate *gates, const double *thetas) {
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n_maps) return;
    const DevMap3 mp = maps[i];
    double M[9] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0};
    for (int k = 0; k < mp.count; ++k) {
        double G[9], R[9];
        gate_matrix3(gates[map_gate_idx[mp.first + k]], thetas, G);
        mul3(G, M, R);
#pragma unroll
        for (int j = 0; j < 9; ++j) M[j] = R[j];
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) maps[i].m[j] = M[j];
}

// Angles -> stream records: shear coefficients of rotations, and the composed
// maps (from k_compose_maps) copied into the R_MAP3 data records, transposed
// (the inverse) in backward streams.
__global__ void k_encode_stream(Rec *recs, const int32_t *enc, int n_enc, const DevMap3 *maps,
                                const double *thetas) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_enc) return;
    Rec &r = recs[enc[k]];
    if (r.kind == R_ROT) {
        double t, s;
        uint16_t neg;
        shear_coeffs(thetas[r.param], t, s, neg);
        r.t = r.inv ? -t : t;
        r.s = r.inv ? -s : s;
        r.code = neg;
    } else if (r.kind == R_MAP3) {
        const double *M = maps[r.param].m;
        double *dst = reinterpret_cast<double *>(&r + 1);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) dst[3 * i + j] = r.inv ? M[3 * j + i] : M[3 * i + j];
    }
}

__global__ void k_encode(DevOp *ops, int n_ops, const double *thetas) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_ops && ops[i].kind == K_ROT) {
        double t, s;
        uint16_t neg;
        shear_coeffs(thetas[ops[i].param], t, s, neg);
        ops[i].t = t;
        ops[i].s = s;
        ops[i].perm = neg;
    }
}

__global__ void k_fill(double *vec, int n, int n_vec, int init) {
    const uint64_t E = 1ull << (2 * n);
    const uint64_t total = E * (uint64_t)n_vec;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = t >> (2 * n), i = t & (E - 1);
        double val = 0.0;
        if (init == INIT_RHO0) val = i < (1ull << n) ? 1.0 : 0.0;
        else if (init == INIT_GENERATOR) val = (i == (1ull << v)) ? 1.0 : 0.0;
        vec[t] = val;
    }
}

__global__ void k_scatter_terms(double *vec, const DevTerm *terms, int n_terms) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_terms) vec[terms[k].idx] = terms[k].coeff;
}

__global__ void __launch_bounds__(kThreads) k_stream_wire(double *vec, int n, int n_vec, DevPass p,
                                                          const DevOp *ops, const DevMap3 *maps,
                                                          int inverse) {
    const int q = p.q;
    const uint64_t E = 1ull << (2 * n);
    const uint64_t G = E >> 2;
    const uint64_t total = G * (uint64_t)n_vec;
    const uint64_t bx = 1ull << (n + q), bz = 1ull << q;
    const int n_ops = p.n_ops;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = t >> (2 * n - 2), g = t & (G - 1);
        double *base = vec + v * E + group_base(g, n, q);
        double x = base[bx], y = base[bx | bz], z = base[bz];
        for (int j = 0; j < n_ops; ++j) {
            const DevOp op = ops[p.first + (inverse ? n_ops - 1 - j : j)];
            apply_op1(x, y, z, op, maps, inverse);
        }
        base[bx] = x;
        base[bx | bz] = y;
        base[bz] = z;
    }
}

__global__ void __launch_bounds__(kThreads) k_stream_cliff(const double *__restrict__ src,
                                                           double *__restrict__ dst, int n,
                                                           int n_vec, DevPass p, const DevOp *ops,
                                                           int inverse) {
    const uint64_t E = 1ull << (2 * n);
    const uint64_t total = E * (uint64_t)n_vec;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = t >> (2 * n), i = t & (E - 1);
        uint32_t neg = 0;
        const uint64_t j = pull_pass(i, n, ops + p.first, p.n_ops, inverse, neg);
        dst[t] = flip(src[v * E + j], neg);
    }
}

// Exponent c (mod 4) of P(a) P(b) = i^c P(a xor b) for Hermitian Pauli strings
// given by x / z masks: per qubit, with a = Y: z_b - x_b; a = X: z_b (2 x_b - 1);
// a = Z: x_b (1 - 2 z_b) (the phase function of Aaronson and Gottesman's
// tableau algorithm), summed with population counts.
__device__ __forceinline__ uint32_t tab_mul_phase(uint32_t ax, uint32_t az, uint32_t bx,
                                                  uint32_t bz) {
    const uint32_t A = ax & az, B = ax & ~az, C = ~ax & az;
    const uint32_t plus = (A & bz & ~bx) | (B & bz & bx) | (C & bx & ~bz);
    const uint32_t minus = (A & bx & ~bz) | (B & bz & ~bx) | (C & bx & bz);
    return (uint32_t)(__popc(plus) - __popc(minus)) & 3u;
}

// A Clifford run as one signed gather: dst[i] = sign * src[j] with
// V P_i V^dagger = sign P_j for the map V whose tableau is given (the run's
// inverse for a forward application).  V P(x, z) V^dagger is i^{|x & z|} times
// the product of the generator images (X_q images for x, Z_q images for z, q
// ascending, Y = i X Z), each factor adding its phase and sign.
__global__ void __launch_bounds__(kThreads) k_stream_tab(const double *__restrict__ src,
                                                         double *__restrict__ dst, int n,
                                                         int n_vec, const DevTab *tab) {
    // The tableau regrouped by chunks of 4 qubits: entry (c, t) is the ordered
    // product of the generator images that subset t of chunk c selects (bit j:
    // X of qubit 4c + j, bit 4 + j: its Z), built by every block in shared
    // memory; an index then takes ceil(n / 4) lookups and string products
    // instead of one product per set bit.
    constexpr int kChunkQ = 4;
    __shared__ uint32_t cx[3 * 256], cz[3 * 256], ce[3 * 256];
    const int n_ch = (n + kChunkQ - 1) / kChunkQ;
    for (int k = threadIdx.x; k < n_ch * 256; k += blockDim.x) {
        const int c = k >> 8, t = k & 255;
        uint32_t rx = 0, rz = 0, e = 0;
        for (int j = 0; j < kChunkQ; ++j) {
            const int q = kChunkQ * c + j;
            if (q >= n) break;
            for (int part = 0; part < 2; ++part) {   // X_q, then Z_q
                if (!((t >> (part * kChunkQ + j)) & 1)) continue;
                const int g = part ? n + q : q;
                e += tab_mul_phase(rx, rz, tab->x[g], tab->z[g]) +
                     (((tab->neg >> g) & 1u) ? 2u : 0u);
                rx ^= tab->x[g];
                rz ^= tab->z[g];
            }
        }
        cx[k] = rx;
        cz[k] = rz;
        ce[k] = e & 3u;
    }
    __syncthreads();
    const uint64_t E = 1ull << (2 * n);
    const uint64_t total = E * (uint64_t)n_vec;
    const uint32_t zmask = (1u << n) - 1u;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = t >> (2 * n);
        const uint32_t i = (uint32_t)(t & (E - 1));
        const uint32_t x = i >> n, z = i & zmask;
        uint32_t rx = 0, rz = 0, e = (uint32_t)__popc(x & z);
        for (int c = 0; c < n_ch; ++c) {
            const uint32_t sh = (uint32_t)(kChunkQ * c);
            const int k = (c << 8) | (int)(((x >> sh) & 15u) | (((z >> sh) & 15u) << 4));
            e += ce[k] + tab_mul_phase(rx, rz, cx[k], cz[k]);
            rx ^= cx[k];
            rz ^= cz[k];
        }
        const double val = src[v * E + (((uint64_t)rx << n) | rz)];
        dst[t] = (e & 2u) ? -val : val;
    }
}

__device__ __forceinline__ uint64_t deposit_runs(uint64_t v, const BitRuns &r) {
    uint64_t out = 0;
    for (int k = 0; k < r.n; ++k)
        out |= ((v >> r.src[k]) & ((1ull << r.len[k]) - 1ull)) << r.dst[k];
    return out;
}

__global__ void __launch_bounds__(kThreads) k_stream_tile(const double *src, double *dst, int n,
                                                          int n_vec, TileGroup tg,
                                                          const DevOp *ops,
                                                          const DevMap3 *maps) {
    extern __shared__ double tile[];
    const uint32_t T = 1u << tg.tile_bits;
    // the group's ops, staged once (when they fit), then the tile-local entry
    // -> offset table, the same for every tile
    DevOp *sops = reinterpret_cast<DevOp *>(tile + T);
    uint32_t *offs = reinterpret_cast<uint32_t *>(sops + kTileStagedOps);
    int total_ops = 0;
    for (int j = 0; j < tg.n_pass; ++j) total_ops += tg.n_ops[j];
    const bool staged = total_ops <= kTileStagedOps;
    if (staged) {
        int at = 0;
        for (int j = 0; j < tg.n_pass; ++j) {
            for (int k = threadIdx.x; k < (int)tg.n_ops[j]; k += blockDim.x)
                sops[at + k] = ops[tg.first[j] + k];
            at += tg.n_ops[j];
        }
    }
    for (uint32_t e = threadIdx.x; e < T; e += blockDim.x)
        offs[e] = (uint32_t)deposit_runs(e, tg.tile_runs);
    __syncthreads();
    const uint64_t E = 1ull << (2 * n);
    const uint64_t tiles = (uint64_t)n_vec << tg.rest_bits;
    for (uint64_t tb = blockIdx.x; tb < tiles; tb += gridDim.x) {
        const uint64_t v = tb >> tg.rest_bits, t = tb & ((1ull << tg.rest_bits) - 1ull);
        const uint64_t base = deposit_runs(t, tg.rest_runs);
        const double *S = src + v * E;
        double *V = dst + v * E + base;
        if (tg.pull_n == 0) {
            for (uint32_t e = threadIdx.x; e < T; e += blockDim.x) tile[e] = S[base + offs[e]];
        } else {
            for (uint32_t e = threadIdx.x; e < T; e += blockDim.x) {
                uint32_t neg = 0;
                const uint64_t j = pull_pass(base + offs[e], n, ops + tg.pull_first, tg.pull_n,
                                             tg.pull_inverse, neg);
                tile[e] = flip(S[j], neg);
            }
        }
        __syncthreads();
        int at = 0;
        for (int j = 0; j < tg.n_pass; ++j) {
            const int lz = tg.lz[j], lx = tg.lx[j];
            const int lo = lz < lx ? lz : lx, hi = lz < lx ? lx : lz;
            const uint32_t bz = 1u << lz, bx = 1u << lx;
            const int n_ops = tg.n_ops[j];
            const DevOp *pops = staged ? sops + at : ops + tg.first[j];
            at += n_ops;
            for (uint32_t g = threadIdx.x; g < T / 4; g += blockDim.x) {
                uint32_t b = ((g >> lo) << (lo + 1)) | (g & ((1u << lo) - 1u));
                b = ((b >> hi) << (hi + 1)) | (b & ((1u << hi) - 1u));
                double x = tile[b | bx], y = tile[b | bx | bz], z = tile[b | bz];
                for (int k = 0; k < n_ops; ++k) {
                    const DevOp op = pops[tg.inverse ? n_ops - 1 - k : k];
                    apply_op1(x, y, z, op, maps, tg.inverse);
                }
                tile[b | bx] = x;
                tile[b | bx | bz] = y;
                tile[b | bz] = z;
            }
            __syncthreads();
        }
        for (uint32_t e = threadIdx.x; e < T; e += blockDim.x) V[offs[e]] = tile[e];
        __syncthreads();
    }
}

// Deterministic sum of the 2^n x-free coefficients of each vector (one CTA
// per vector, fixed order).
__global__ void __launch_bounds__(kThreads) k_xfree_sum(const double *vec, int n, double *out) {
    __shared__ double red[kThreads / 32];
    const uint64_t E = 1ull << (2 * n);
    const double *v = vec + blockIdx.x * E;
    double acc = 0.0;
    for (int i = threadIdx.x; i < (1 << n); i += blockDim.x) acc += v[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double total = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) total += red[w];
        out[blockIdx.x] = total;
    }
}

// Inner product <a, b> of two coefficient vectors in a fixed order: block b
// sums a contiguous slice (strided by the block's threads, then a shuffle
// tree), the last kernel the kDotBlocks partials in order.
constexpr int kDotBlocks = 256;

__global__ void __launch_bounds__(kThreads) k_dot_partial(const double *a, const double *b,
                                                          int n, double *partial) {
    __shared__ double red[kThreads / 32];
    const uint64_t E = 1ull << (2 * n);
    const uint64_t per = (E + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = blockIdx.x * per, hi = lo + per < E ? lo + per : E;
    double acc = 0.0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc = fma(a[i], b[i], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double total = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) total += red[w];
        partial[blockIdx.x] = total;
    }
}

__global__ void k_dot_final(const double *partial, int nblk, double *out) {
    const int lane = threadIdx.x;
    const int per = (nblk + 31) / 32;
    double t = 0.0;
    for (int k = lane * per; k < nblk && k < (lane + 1) * per; ++k) t += partial[k];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) *out = t;
}

// Waits on a barrier nothing completes, with a poll bound; records a timeout.
__global__ void k_bounded_wait(int64_t polls, int32_t *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        bool ok = polls == 0;
        for (int64_t i = 0; i < polls && !ok; ++i) ok = mbar_try_wait(&bar, 0);
        *status = ok ? 0 : STAB_KSTATUS_TIMEOUT;
    }
}

}  // namespace

cudaError_t launch_bounded_wait(int64_t polls, int32_t *status, cudaStream_t st) {
    k_bounded_wait<<<1, 32, 0, st>>>(polls, status);
    return cudaGetLastError();
}

int max_map_count(const DevMap3 *maps, size_t n_maps) {
    int m = 0;
    for (size_t i = 0; i < n_maps; ++i) m = maps[i].count > m ? maps[i].count : m;
    return m;
}

cudaError_t launch_compose_maps(DevMap3 *maps, int n_maps, int max_count,
                                const int32_t *map_gate_idx, const RawGate *gates,
                                const double *thetas, cudaStream_t st) {
    if (n_maps == 0) return cudaSuccess;
    if (max_count <= kSeqMapGates)
        k_compose_maps_seq<<<(n_maps + 127) / 128, 128, 0, st>>>(maps, n_maps, map_gate_idx, gates,
                                                                 thetas);
    else
        k_compose_maps<<<(n_maps + 3) / 4, 128, 0, st>>>(maps, n_maps, map_gate_idx, gates,
                                                         thetas);
    return cudaGetLastError();
}

cudaError_t launch_encode(DevOp *ops, int n_ops, DevMap3 *maps, int n_maps, int max_count,
                          const int32_t *map_gate_idx, const RawGate *gates, const double *thetas,
                          cudaStream_t st) {
    cudaError_t e = launch_compose_maps(maps, n_maps, max_count, map_gate_idx, gates, thetas, st);
    if (e != cudaSuccess || n_ops == 0) return e;
    k_encode<<<(n_ops + 127) / 128, 128, 0, st>>>(ops, n_ops, thetas);
    return cudaGetLastError();
}

cudaError_t launch_encode_stream(Rec *recs, const int32_t *enc, int n_enc, const DevMap3 *maps,
                                 const double *thetas, cudaStream_t st) {
    if (n_enc == 0) return cudaSuccess;
    k_encode_stream<<<(n_enc + 127) / 128, 128, 0, st>>>(recs, enc, n_enc, maps, thetas);
    return cudaGetLastError();
}

cudaError_t launch_fill(double *vec, int n, int n_vec, int init, const DevTerm *terms,
                        int n_terms, cudaStream_t st) {
    const uint64_t total = (1ull << (2 * n)) * (uint64_t)n_vec;
    k_fill<<<grid_for(total, kThreads), kThreads, 0, st>>>(vec, n, n_vec, init);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || init != INIT_TERMS || n_terms == 0) return e;
    k_scatter_terms<<<(n_terms + 127) / 128, 128, 0, st>>>(vec, terms, n_terms);
    return cudaGetLastError();
}

cudaError_t launch_stream_wire(double *vec, int n, int n_vec, const DevPass &p, const DevOp *ops,
                               const DevMap3 *maps, int inverse, cudaStream_t st) {
    const uint64_t total = (1ull << (2 * n - 2)) * (uint64_t)n_vec;
    k_stream_wire<<<grid_for(total, kThreads), kThreads, 0, st>>>(vec, n, n_vec, p, ops, maps,
                                                                   inverse);
    return cudaGetLastError();
}

cudaError_t launch_stream_tab(const double *src, double *dst, int n, int n_vec,
                              const DevTab *tab, cudaStream_t st) {
    const uint64_t total = (1ull << (2 * n)) * (uint64_t)n_vec;
    k_stream_tab<<<grid_for(total, kThreads), kThreads, 0, st>>>(src, dst, n, n_vec, tab);
    return cudaGetLastError();
}

cudaError_t launch_stream_cliff(const double *src, double *dst, int n, int n_vec,
                                const DevPass &p, const DevOp *ops, int inverse, cudaStream_t st) {
    const uint64_t total = (1ull << (2 * n)) * (uint64_t)n_vec;
    k_stream_cliff<<<grid_for(total, kThreads), kThreads, 0, st>>>(src, dst, n, n_vec, p, ops,
                                                                    inverse);
    return cudaGetLastError();
}

cudaError_t launch_stream_tile(const double *src, double *dst, int n, int n_vec,
                               const TileGroup &tg, const DevOp *ops, const DevMap3 *maps,
                               cudaStream_t st) {
    const uint32_t T = 1u << tg.tile_bits;
    const uint64_t tiles = (uint64_t)n_vec << tg.rest_bits;
    int threads = (int)(T / 4);
    if (threads > kThreads) threads = kThreads;
    if (threads < 32) threads = 32;
    uint64_t grid = tiles;
    if (grid > 152ull * 8ull) grid = 152ull * 8ull;
    const size_t smem = T * (sizeof(double) + sizeof(uint32_t)) + kTileStagedOps * sizeof(DevOp);
    static SmemLimit lim;
    cudaError_t e = raise_smem_limit(k_stream_tile, smem, lim);
    if (e != cudaSuccess) return e;
    k_stream_tile<<<(int)grid, threads, smem, st>>>(src, dst, n, n_vec, tg, ops, maps);
    return cudaGetLastError();
}

cudaError_t launch_dot(const double *a, const double *b, int n, double *partial, double *out,
                       cudaStream_t st) {
    k_dot_partial<<<kDotBlocks, kThreads, 0, st>>>(a, b, n, partial);
    k_dot_final<<<1, 32, 0, st>>>(partial, kDotBlocks, out);
    return cudaGetLastError();
}

cudaError_t launch_xfree_sum(const double *vec, int n, int n_vec, double *out, cudaStream_t st) {
    k_xfree_sum<<<n_vec, kThreads, 0, st>>>(vec, n, out);
    return cudaGetLastError();
}

}  // namespace stab
