// resident.cuh -- device building blocks of the shared-memory-resident
// kernels (k_resident.cu) and the persistent batch kernel (k_batch.cu): pass
// loops over a staged instruction stream on one vector held by one CTA.  The
// vector buffers may live in shared memory or, for larger n, in a per-CTA
// slab of global memory; the code is the same.
#pragma once

#include <cuda_runtime.h>

#include "device_ops.cuh"
#include "launch.h"
#include "tma.cuh"

namespace stab {
namespace resident {

template <int N, int LPG>
struct SCfg {
    static constexpr int E = 1 << (2 * N);   // coefficients per vector
    static constexpr int G = E / 4;          // groups of one wire
    static constexpr int L = G * LPG;        // working lanes
    static constexpr int T = L < 32 ? 32 : (L > 1024 ? 1024 : ((L + 31) / 32) * 32);
    static constexpr int GPT = (G + T - 1) / T;   // groups per thread (LPG = 1)
    static constexpr int W = T / 32;
};

constexpr int R = kRotPerGradPass;

// Shared memory: [chunks 2 x 4 KiB][mbarriers 16 B | flag | gradient slots][reduction][vectors]
constexpr int kOffBar = 2 * kChunkRecs * (int)sizeof(Rec);
constexpr int kOffFlag = kOffBar + 16;
constexpr int kOffSlot = kOffBar + 32;
constexpr int kOffRed = kOffBar + 128;
constexpr int kSmemHeader = kOffRed + 32 * 8 * R;

template <int N>
__device__ __forceinline__ void group_idx(uint32_t g, int q, uint32_t &ii, uint32_t &ix,
                                          uint32_t &iy, uint32_t &iz) {
    ii = group_base32(g, N, q);
    iz = ii | (1u << q);
    ix = ii | (1u << (N + q));
    iy = ix | (1u << q);
}

template <int N>
__device__ __forceinline__ double pulled(const double *src, uint32_t i, const Rec *pulls,
                                         int n_pull) {
    uint32_t neg = 0;
    const uint32_t j = pull_recs(i, N, pulls, n_pull, neg);
    return flip(src[j], neg);
}

// One wire pass, LPG = 1: cur -> nxt, T threads, groups strided by T.
template <int N, int T = SCfg<N, 1>::T>
__device__ __forceinline__ void pass_groups(const double *cur, double *nxt, int q,
                                            const Rec *pulls, int n_pull, const Rec *ops,
                                            int n_ops) {
    constexpr int G = (1 << (2 * N)) / 4;
    constexpr int GPT = (G + T - 1) / T;
#pragma unroll(GPT <= 8 ? GPT : 1)
    for (int k = 0; k < GPT; ++k) {
        const uint32_t g = threadIdx.x + k * T;
        if (g < (uint32_t)G) {
            uint32_t ii, ix, iy, iz;
            group_idx<N>(g, q, ii, ix, iy, iz);
            const double vi = pulled<N>(cur, ii, pulls, n_pull);
            double x = pulled<N>(cur, ix, pulls, n_pull);
            double y = pulled<N>(cur, iy, pulls, n_pull);
            double z = pulled<N>(cur, iz, pulls, n_pull);
            apply_recs(x, y, z, ops, n_ops);
            nxt[ii] = vi;
            nxt[ix] = x;
            nxt[iy] = y;
            nxt[iz] = z;
        }
    }
}

// Slot index of lane (g, slot) for a pass on wire q, and its pulled source.
template <int N>
__device__ __forceinline__ void quad_index(uint32_t g, uint32_t slot, int q, const Rec *pulls,
                                           int n_pull, uint32_t &i, uint32_t &j, uint32_t &neg) {
    const uint32_t b = group_base32(g, N, q);
    // slot 0 = I, 1 = X, 2 = Y, 3 = Z
    const uint32_t xb = (slot == 1u || slot == 2u) ? (1u << (N + q)) : 0u;
    const uint32_t zb = (slot >= 2u) ? (1u << q) : 0u;
    i = b | xb | zb;
    neg = 0;
    j = pull_recs(i, N, pulls, n_pull, neg);
}

template <int T>
__device__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double total = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < T / 32; ++w) total += red[w];
    return total;
}

__device__ __forceinline__ void stager_setup(Stager &st, unsigned char *smem) {
    st.buf = reinterpret_cast<Rec *>(smem);
    st.bar = reinterpret_cast<uint64_t *>(smem + kOffBar);
    st.flag = reinterpret_cast<int *>(smem + kOffFlag);
}

// Runs the passes of chunks [c0, c1) on one vector; returns the buffer that
// holds the result, or nullptr when a staging wait gave up.
// LPG = 4 pass loop (see the file comment).
template <int N>
__device__ double *run_stream_quads(Stager &st, int c0, int c1, double *cur, double *nxt,
                                    int32_t *status) {
    constexpr int L = (1 << (2 * N));   // 4 lanes per group of 4 entries
    const uint32_t l = threadIdx.x;
    const bool active = l < (uint32_t)L;
    const uint32_t g = l >> 2, slot = l & 3u;
    const uint32_t lane = l & 31u, qbase = lane & ~3u;
    for (int c = c0; c < c1; ++c) {
        if (!st.wait(c, status)) return nullptr;
        const Rec *Rr = st.chunk(c);
        int r = 0;
        Rec h = Rr[0];
        uint32_t i = 0, j = 0, neg = 0;
        if (h.kind == R_PASS && active) quad_index<N>(g, slot, h.q, Rr + 1, h.param, i, j, neg);
        while (h.kind == R_PASS) {
            const int r_next = r + 1 + h.param + h.gate;
            const Rec hn = Rr[r_next];
            double v = 0.0;
            if (active) v = flip(cur[j], neg);
            const double x = __shfl_sync(0xffffffffu, v, qbase + 1);
            const double y = __shfl_sync(0xffffffffu, v, qbase + 2);
            const double z = __shfl_sync(0xffffffffu, v, qbase + 3);
            double out = v;
            if (h.gate != 0 && slot != 0u) {
                const double *m =
                    reinterpret_cast<const double *>(Rr + r + 2 + h.param) + 3 * (slot - 1u);
                out = fma(m[2], z, fma(m[1], y, m[0] * x));
            }
            // source of the next pass, computed while the FP64 chain above runs
            uint32_t i2 = 0, j2 = 0, neg2 = 0;
            if (hn.kind == R_PASS && active)
                quad_index<N>(g, slot, hn.q, Rr + r_next + 1, hn.param, i2, j2, neg2);
            if (active) nxt[i] = out;
            double *t = cur;
            cur = nxt;
            nxt = t;
            __syncthreads();
            h = hn;
            r = r_next;
            i = i2;
            j = j2;
            neg = neg2;
        }
        st.release(c);
    }
    return cur;
}

// n = 4, LPG = 4, with the vector held in registers between passes: each of
// the 256 lanes keeps one entry.  In layout A a warp's 32 lanes span the
// (z, x) bits of wires 0 and 1 (plus z_2), in layout B those of wires 2 and 3
// (plus z_0); the warp index holds the other three bits.  A pass on a wire
// of the current layout gathers its group from the quad's lanes by shuffles
// and needs no shared memory and no barrier; a pass that pulls through a
// Clifford run, or whose wire is in the other layout, first goes through
// shared memory (write, one barrier, pulled read in the wanted layout).  The
// two buffers alternate, so a write never meets a read still in flight.
__device__ __forceinline__ uint32_t reg4_index(uint32_t t, int layout) {
    // index bits: z_q = bit q, x_q = bit 4 + q.  Lane/warp bit k -> index bit.
    const uint32_t pa[8] = {0, 4, 1, 5, 2, 6, 3, 7};
    const uint32_t pb[8] = {2, 6, 3, 7, 0, 4, 1, 5};
    uint32_t i = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) i |= ((t >> k) & 1u) << (layout ? pb[k] : pa[k]);
    return i;
}

inline __device__ double *run_stream_reg4(Stager &st, int c0, int c1, double *cur, double *nxt,
                                   int32_t *status) {
    const uint32_t t = threadIdx.x;
    const uint32_t lane = t & 31u;
    const uint32_t iA = reg4_index(t, 0), iB = reg4_index(t, 1);
    int layout = 0;
    double v = cur[iA];
    double *rd = cur, *wr = nxt;   // last buffer read; the one the next write goes to
    // this thread's source index and sign through the last pull records it
    // walked, and the layout they were taken in (-1: none yet in this call)
    uint32_t pj = 0, pneg = 0;
    int play = -1;
    for (int c = c0; c < c1; ++c) {
        if (!st.wait(c, status)) return nullptr;
        const Rec *Rr = st.chunk(c);
        int r = 0;
        Rec h = Rr[0];
        while (h.kind == R_PASS) {
            const int q = h.q, n_pull = h.param;
            const int r_next = r + 1 + n_pull + h.gate;
            const int want = q < 2 ? 0 : 1;
            if (n_pull > 0 || want != layout) {
                wr[layout ? iB : iA] = v;
                __syncthreads();
                uint32_t neg = 0, j;
                if (n_pull > 0 && h.code == kPullRepeat && play == want) {
                    j = pj;   // the same Clifford run as the last pull, same layout
                    neg = pneg;
                } else {
                    j = pull_recs(want ? iB : iA, 4, Rr + r + 1, n_pull, neg);
                    if (n_pull > 0) {
                        pj = j;
                        pneg = neg;
                        play = want;
                    }
                }
                v = flip(wr[j], neg);
                double *tmp = rd;
                rd = wr;
                wr = tmp;
                layout = want;
            }
            if (h.gate != 0) {
                const int sh = 2 * (q & 1);                // the wire's lane-bit pair
                const uint32_t zb = (lane >> sh) & 1u, xb = (lane >> (sh + 1)) & 1u;
                const uint32_t base = lane & ~(3u << sh);
                const double x = __shfl_sync(0xffffffffu, v, base | (2u << sh));
                const double y = __shfl_sync(0xffffffffu, v, base | (3u << sh));
                const double z = __shfl_sync(0xffffffffu, v, base | (1u << sh));
                if (xb | zb) {
                    // slot 1 = X (x), 2 = Y (x, z), 3 = Z (z): row slot - 1 of the map
                    const uint32_t slot = xb ? (zb ? 2u : 1u) : 3u;
                    const double *m =
                        reinterpret_cast<const double *>(Rr + r + 2 + n_pull) + 3 * (slot - 1u);
                    v = fma(m[2], z, fma(m[1], y, m[0] * x));
                }
            }
            r = r_next;
            h = Rr[r];
        }
        st.release(c);
    }
    wr[layout ? iB : iA] = v;
    __syncthreads();
    return wr;
}

// ---------------------------------------------------------------- adjoint

__device__ __forceinline__ double pair_dot(int axis, double lx, double ly, double lz, double rx,
                                           double ry, double rz) {
    // d<O>/d theta on the pair (u, v): l_v r_u - l_u r_v; (u, v) = (Y, Z) for
    // R_x, (Z, X) for R_y, (X, Y) for R_z
    if (axis == AX_X) return fma(lz, ry, -ly * rz);
    if (axis == AX_Y) return fma(lx, rz, -lz * rx);
    return fma(ly, rx, -lx * ry);
}

// One rotation record on the same pair slots of both vectors (lambda and
// rho), as apply_rot does on one.
__device__ __forceinline__ void rot_pair(const Rec &op, double &lx, double &ly, double &lz,
                                         double &rx, double &ry, double &rz) {
    const double t = op.t, s = op.s;
    const uint32_t neg = op.code;
    if (op.axis == AX_X) {
        lift(ly, lz, t, s, neg);
        lift(ry, rz, t, s, neg);
    } else if (op.axis == AX_Y) {
        lift(lz, lx, t, s, neg);
        lift(rz, rx, t, s, neg);
    } else {
        lift(lx, ly, t, s, neg);
        lift(rx, ry, t, s, neg);
    }
}

// The pair (lambda, rho) through chunks [c0, c1) of a gradient stream, with
// each rotation's dot <lambda_j, G_j rho_j> taken at its post-gate pair (G_j
// the generator of the rotation on its pairs) and written to grad_rot at the
// rotation's ordinal.  fwd = false: a backward stream -- the pair holds the
// post-gate values when an inverse op comes up, so dot, then apply; fwd =
// true: a forward stream (lambda_j = M_j lambda_{j-1} because every map is
// orthogonal) -- apply, then dot.  On return lam / rho point at the results;
// false when a staging wait gave up.  The block has T threads (a multiple
// of 32), each taking groups threadIdx.x, + T, ...; each rotation's dot is
// summed over a warp by shuffles, then over the warps in warp order -- or,
// with part_out, each thread stores its own share at part_out[ordinal * T +
// thread] and the sweep does no reduction and no barrier for it (the caller
// sums every rotation over the threads afterwards, in thread order).
// REUSE: with part_out and one group per thread, a pass whose Clifford run
// repeats the last pull on the same wire takes the group's pulled sources
// and signs from registers (eight more registers a thread).
template <int N, int T = SCfg<N, 1>::T, bool REUSE = (N <= 5)>
__device__ __forceinline__ bool adjoint_sweep(Stager &st, int c0, int c1, double *&lam,
                                              double *&lam_n, double *&rho, double *&rho_n,
                                              double *grad_rot, int32_t *status,
                                              unsigned char *smem, const bool fwd,
                                              double *part_out = nullptr) {
    constexpr int G = SCfg<N, 1>::G;
    constexpr int GPT = (G + T - 1) / T;
    constexpr int W = T / 32;
    int *gslot = reinterpret_cast<int *>(smem + kOffSlot);
    double *red = reinterpret_cast<double *>(smem + kOffRed);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // fast path: the group's four pulled sources and signs through the last
    // pull records walked, and the wire of that pass (-1: none yet)
    constexpr bool kReuse = REUSE;
    uint32_t cj[4] = {0, 0, 0, 0}, cn[4] = {0, 0, 0, 0};
    int cq = -1;
    for (int c = c0; c < c1; ++c) {
        if (!st.wait(c, status)) return false;
        const Rec *Rr = st.chunk(c);
        int r = 0;
        while (true) {
            const Rec h = Rr[r];
            if (h.kind != R_PASS) break;
            const Rec *pulls = Rr + r + 1;
            const Rec *ops = pulls + h.param;
            const int n_pull = h.param, n_ops = h.gate, q = h.q;
            if (GPT == 1 && part_out) {
                // one group per thread, each dot's share stored as it comes:
                // every op decoded once for both vectors, the group's four
                // sources pulled once for both
                const uint32_t g = threadIdx.x;
                if (g < (uint32_t)G) {
                    uint32_t ii, ix, iy, iz;
                    group_idx<N>(g, q, ii, ix, iy, iz);
                    uint32_t ji = ii, jx = ix, jy = iy, jz = iz;
                    uint32_t ni = 0, nx = 0, ny = 0, nz = 0;
                    if (kReuse && n_pull > 0 && h.code == kPullRepeat && cq == q) {
                        // the same Clifford run as the last pull, on the same wire
                        ji = cj[0]; jx = cj[1]; jy = cj[2]; jz = cj[3];
                        ni = cn[0]; nx = cn[1]; ny = cn[2]; nz = cn[3];
                    } else if (n_pull > 0) {
                        ji = pull_recs(ii, N, pulls, n_pull, ni);
                        jx = pull_recs(ix, N, pulls, n_pull, nx);
                        jy = pull_recs(iy, N, pulls, n_pull, ny);
                        jz = pull_recs(iz, N, pulls, n_pull, nz);
                        if (kReuse) {
                            cj[0] = ji; cj[1] = jx; cj[2] = jy; cj[3] = jz;
                            cn[0] = ni; cn[1] = nx; cn[2] = ny; cn[3] = nz;
                            cq = q;
                        }
                    }
                    const double li = flip(lam[ji], ni), ri = flip(rho[ji], ni);
                    double lx = flip(lam[jx], nx), ly = flip(lam[jy], ny), lz = flip(lam[jz], nz);
                    double rx = flip(rho[jx], nx), ry = flip(rho[jy], ny), rz = flip(rho[jz], nz);
                    for (int j = 0; j < n_ops; ++j) {
                        const Rec op = ops[j];
                        if (op.kind == R_ROT) {
                            double *share = part_out + (size_t)op.gate * T + threadIdx.x;
                            if (!fwd) *share = pair_dot(op.axis, lx, ly, lz, rx, ry, rz);
                            rot_pair(op, lx, ly, lz, rx, ry, rz);
                            if (fwd) *share = pair_dot(op.axis, lx, ly, lz, rx, ry, rz);
                        } else {
                            apply_recs(lx, ly, lz, ops + j, 1);
                            apply_recs(rx, ry, rz, ops + j, 1);
                        }
                    }
                    lam_n[ii] = li; lam_n[ix] = lx; lam_n[iy] = ly; lam_n[iz] = lz;
                    rho_n[ii] = ri; rho_n[ix] = rx; rho_n[iy] = ry; rho_n[iz] = rz;
                } else {
                    // a thread without a group (n <= 3): zero shares
                    for (int j = 0; j < n_ops; ++j)
                        if (ops[j].kind == R_ROT)
                            part_out[(size_t)ops[j].gate * T + threadIdx.x] = 0.0;
                }
                double *t = lam;
                lam = lam_n;
                lam_n = t;
                t = rho;
                rho = rho_n;
                rho_n = t;
                __syncthreads();
                r += 1 + n_pull + n_ops;
                continue;
            }
            double part[R];
#pragma unroll
            for (int k = 0; k < R; ++k) part[k] = 0.0;
#pragma unroll(GPT <= 4 ? GPT : 1)
            for (int k = 0; k < GPT; ++k) {
                const uint32_t g = threadIdx.x + k * T;
                if (g < (uint32_t)G) {
                    uint32_t ii, ix, iy, iz;
                    group_idx<N>(g, q, ii, ix, iy, iz);
                    const double li = pulled<N>(lam, ii, pulls, n_pull);
                    const double ri = pulled<N>(rho, ii, pulls, n_pull);
                    double lx = pulled<N>(lam, ix, pulls, n_pull);
                    double ly = pulled<N>(lam, iy, pulls, n_pull);
                    double lz = pulled<N>(lam, iz, pulls, n_pull);
                    double rx = pulled<N>(rho, ix, pulls, n_pull);
                    double ry = pulled<N>(rho, iy, pulls, n_pull);
                    double rz = pulled<N>(rho, iz, pulls, n_pull);
                    int slot = 0;
                    for (int j = 0; j < n_ops; ++j) {
                        if (fwd) {
                            apply_recs(lx, ly, lz, ops + j, 1);
                            apply_recs(rx, ry, rz, ops + j, 1);
                        }
                        if (ops[j].kind == R_ROT) {
                            const double d = pair_dot(ops[j].axis, lx, ly, lz, rx, ry, rz);
#pragma unroll
                            for (int s = 0; s < R; ++s)
                                if (s == slot) part[s] += d;
                            ++slot;
                        }
                        if (!fwd) {
                            apply_recs(lx, ly, lz, ops + j, 1);
                            apply_recs(rx, ry, rz, ops + j, 1);
                        }
                    }
                    lam_n[ii] = li; lam_n[ix] = lx; lam_n[iy] = ly; lam_n[iz] = lz;
                    rho_n[ii] = ri; rho_n[ix] = rx; rho_n[iy] = ry; rho_n[iz] = rz;
                }
            }
            if (part_out) {
                // this thread's share of each of the pass's rotations
                int slot = 0;
                for (int j = 0; j < n_ops; ++j) {
                    if (ops[j].kind == R_ROT) {
                        double v = 0.0;
#pragma unroll
                        for (int s = 0; s < R; ++s)
                            if (s == slot) v = part[s];
                        part_out[(size_t)ops[j].gate * T + threadIdx.x] = v;
                        ++slot;
                    }
                }
            } else {
                int n_rot = 0;
                for (int j = 0; j < n_ops; ++j) {
                    if (ops[j].kind == R_ROT) {
                        if (threadIdx.x == 0) gslot[n_rot] = ops[j].gate;
                        ++n_rot;
                    }
                }
                // only the pass's rotations are reduced (n_rot is uniform over the CTA)
#pragma unroll
                for (int s = 0; s < R; ++s) {
                    if (s < n_rot) {
                        double v = part[s];
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                        if (lane == 0) red[warp * R + s] = v;
                    }
                }
                __syncthreads();
                if (threadIdx.x < n_rot) {
                    double total = 0.0;
                    for (int w = 0; w < W; ++w) total += red[w * R + threadIdx.x];
                    grad_rot[gslot[threadIdx.x]] = total;
                }
            }
            double *t = lam;
            lam = lam_n;
            lam_n = t;
            t = rho;
            rho = rho_n;
            rho_n = t;
            __syncthreads();
            r += 1 + n_pull + n_ops;
        }
        st.release(c);
    }
    return true;
}

// The block must have at least 4^n threads for LPG = 4.
template <int N, int LPG, int T = SCfg<N, LPG>::T>
__device__ double *run_stream(Stager &st, int c0, int c1, double *cur, double *nxt,
                              int32_t *status) {
    if constexpr (LPG == 4 && N == 4 && T == 256) {
        return run_stream_reg4(st, c0, c1, cur, nxt, status);
    } else if constexpr (LPG == 4) {
        return run_stream_quads<N>(st, c0, c1, cur, nxt, status);
    } else {
        for (int c = c0; c < c1; ++c) {
            if (!st.wait(c, status)) return nullptr;
            const Rec *Rr = st.chunk(c);
            int r = 0;
            while (true) {
                const Rec h = Rr[r];
                if (h.kind != R_PASS) break;   // R_NEXT or R_END
                const Rec *pulls = Rr + r + 1;
                const Rec *ops = pulls + h.param;
                // Without pulls a thread reads and writes only its own groups, so
                // the pass runs in place; a pull pass permutes and needs the
                // second buffer.  (In place keeps one vector hot in L2 when the
                // buffers are in global memory.)
                if (h.param == 0) {
                    pass_groups<N, T>(cur, cur, h.q, pulls, 0, ops, h.gate);
                } else {
                    pass_groups<N, T>(cur, nxt, h.q, pulls, h.param, ops, h.gate);
                    double *t = cur;
                    cur = nxt;
                    nxt = t;
                }
                __syncthreads();
                r += 1 + h.param + h.gate;
            }
            st.release(c);
        }
        return cur;
    }
}

}  // namespace resident
}  // namespace stab
