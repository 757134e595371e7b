// k_resident.cu -- propagation with the whole 4^n coefficient vector resident
// in shared memory, one CTA per vector (n <= 6), reading an instruction stream
// staged chunk by chunk with bulk copies (see tma.cuh).
//
// The CTA walks the passes of the loaded circuit (the sequential Map stage of
// Sec. IV-B).  Each pass reads its wire's groups from one shared buffer --
// pulling every entry through the preceding run of two-qubit Clifford gates
// (map_CX of Sec. III-C, and CZ) -- applies the wire's ops and writes the
// other buffer; the buffers then swap.  Two thread mappings:
//   LPG = 4 (n <= 4): the wire run is one composed 3x3 map and a quad of
//     lanes holds a group (slots I, X, Y, Z); each lane pulls its own entry,
//     gets the other two through warp shuffles and computes its output row:
//     three dependent FP64 instructions per pass.  An FP64 instruction costs
//     ~68 cycles per warp on this GPU whatever the active-lane mask, so this is
//     the shortest pass; the next pass's source index is computed while the
//     current pass's FP64 chain is in flight.
//   LPG = 1 (n = 5, 6): one lane per group running the ops in registers
//     (lifting rotations, 3 FMAs per rotation): the fewest FP64 instructions.
// The adjoint kernel carries the cotangent and the forward vector backward
// together and reduces each rotation's gradient dot at the end of its pass.
#include <cuda_runtime.h>

#include "resident.cuh"

namespace stab {

namespace {

using namespace resident;

template <int N, int LPG>
__global__ void __launch_bounds__(SCfg<N, LPG>::T) k_resident_stream(StreamArgs a) {
    using C = SCfg<N, LPG>;
    extern __shared__ __align__(128) unsigned char smem[];
    Stager st;
    st.s0 = a.stream;
    st.s1 = nullptr;
    st.n0 = a.n_chunks;
    st.n_total = a.n_chunks;
    stager_setup(st, smem);
    double *red = reinterpret_cast<double *>(smem + kOffRed);
    double *bufA = reinterpret_cast<double *>(smem + kSmemHeader);
    double *bufB = bufA + C::E;
    st.start();

    const int b = blockIdx.x;
    for (int i = threadIdx.x; i < C::E; i += C::T) {
        double v = 0.0;
        if (a.init == INIT_RHO0) v = (i < (1 << N)) ? 1.0 : 0.0;
        else if (a.init == INIT_LOAD) v = a.in[(size_t)b * C::E + i];
        bufA[i] = v;
    }
    __syncthreads();
    if (a.init == INIT_GENERATOR) {
        if (threadIdx.x == 0) bufA[1u << b] = 1.0;   // Z_b: z bit b set
    } else if (a.init == INIT_TERMS) {
        for (int k = threadIdx.x; k < a.n_terms; k += C::T) bufA[a.terms[k].idx] = a.terms[k].coeff;
    }
    __syncthreads();

    double *res = run_stream<N, LPG>(st, 0, a.n_chunks, bufA, bufB, a.status);
    if (res == nullptr) return;
    if (a.out) {
        double *o = a.out + (size_t)b * C::E;
        for (int i = threadIdx.x; i < C::E; i += C::T) o[i] = res[i];
    }
    if (a.xfree_out) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < (1 << N); i += C::T) acc += res[i];
        const double total = block_sum<C::T>(acc, red);
        if (threadIdx.x == 0) a.xfree_out[b] = total;
    }
}

// Generators through a transfer matrix: out[k] = T a[k] for k < n_vec, with
// column j of T (T + j E) the image of the basis string j.  One CTA per vector,
// one output entry per thread, the sum over j in order.
// out_k = T a_k.  One CTA per 32 consecutive outputs i of one vector k: lane
// = output (each row j of T is read coalesced), warp w sums the rows j = w,
// w + 8, ...; the eight partial sums are added in a fixed order.
__global__ void __launch_bounds__(256) k_apply_transfer(const double *T, const double *a,
                                                        double *out, int E) {
    __shared__ double sa[256];
    __shared__ double part[8][32];
    const int k = blockIdx.y, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double *ak = a + (size_t)k * E;
    for (int j = threadIdx.x; j < E; j += blockDim.x) sa[j] = ak[j];
    __syncthreads();
    const int i = blockIdx.x * 32 + lane;
    double acc = 0.0;
    if (i < E)
        for (int j = w; j < E; j += 8) acc = fma(T[(size_t)j * E + i], sa[j], acc);
    part[w][lane] = acc;
    __syncthreads();
    if (w == 0 && i < E) {
        double t = part[0][lane];
        for (int r = 1; r < 8; ++r) t += part[r][lane];
        out[(size_t)k * E + i] = t;
    }
}

// v_k <- T_{S-1} ... T_1 T_0 v_k for small vectors (E = 4^n <= 64): one CTA
// per vector, the vector in shared memory.  For each matrix, thread t sums
// the columns j = t / E, t / E + 256 / E, ... of output row i = t % E, and the
// 256 / E shares of a row are added in a fixed order.  With terms (one
// vector), dot_out receives sum_k coeff_k v[idx_k], summed in term order.
__global__ void __launch_bounds__(256) k_apply_chain(const double *T, int n_mats,
                                                     const double *in, double *out, int E,
                                                     const DevTerm *terms, int n_terms,
                                                     double *dot_out) {
    __shared__ double v[64];
    __shared__ double part[256];
    const int t = threadIdx.x;
    const int groups = 256 / E;
    const int i = t % E, p = t / E;
    const size_t at = (size_t)blockIdx.x * E;
    if (t < E) v[t] = in[at + t];
    __syncthreads();
    for (int s = 0; s < n_mats; ++s) {
        const double *M = T + (size_t)s * E * E;
        double acc = 0.0;
        for (int j = p; j < E; j += groups) acc = fma(M[(size_t)j * E + i], v[j], acc);
        part[t] = acc;
        __syncthreads();
        if (t < E) {
            double tot = 0.0;
            for (int g = 0; g < groups; ++g) tot += part[g * E + t];
            v[t] = tot;
        }
        __syncthreads();
    }
    if (out && t < E) out[at + t] = v[t];
    if (dot_out && t == 0) {
        double acc = 0.0;
        for (int k = 0; k < n_terms; ++k) acc = fma(terms[k].coeff, v[terms[k].idx], acc);
        *dot_out = acc;
    }
}

// ---------------------------------------------------------------- transfer columns
//
// Columns of the transfer matrix T of a stream at n = 4: column j is the
// basis string j carried through the stream's passes.  One CTA of 8 H warps
// carries H columns; each half (8 warps) owns one column, its own copy of
// the staged stream and a named barrier, so the halves run independently and
// one's loads and barriers overlap the others' FP64 work, as separate CTAs on
// an SM would.  For a pass on wire q the warp index holds the wire's (x_q, z_q)
// bits and the lane plus warp bit 0 the other six index bits, so the two warps
// of the I slot do no FP64 work (those entries do not change) and the other
// six compute one output row each from the group's X, Y, Z entries.  Pairs of
// halves use mirrored slot maps: warp w = 8v + 4 b2 + 2 b1 + b0 runs on SMSP
// w % 4 and holds slot (x, z) = (b1 ^ (v & 1), b2), so each SMSP has three
// working warps per pair of halves -- nine warp-wide FP64 instructions per
// pass for two columns, where two CTAs of the lane-per-entry form issue
// twelve.  H = 2: the 255 columns of one transfer matrix on 128 CTAs; H = 4:
// those of two matrices (two parts of a plan) on 128 CTAs, one per SM, with
// every SM's FP64 pipe shared by four columns.
constexpr int kColN = 4;
constexpr int kColE = 1 << (2 * kColN);
constexpr int kColHalf = (kOffRed + 127) / 128 * 128;   // one half's chunks + barriers

template <int H>
__global__ void __launch_bounds__(256 * H, 1) k_transfer_cols(ColArgs a) {
    constexpr int N = kColN, E = kColE;
    extern __shared__ __align__(128) unsigned char smem[];
    const int w = threadIdx.x >> 5;
    const int v = w >> 3;                             // this half
    // slot s of 256 per transfer matrix: the matrix s / 256, column 1 + s % 256
    const int slot = H * (int)blockIdx.x + v;
    const int part = slot / E;
    const int col = 1 + slot % E;
    if (part >= a.n_parts || col >= E) return;       // the 256th slot of a matrix idles
    const uint32_t tid = threadIdx.x & 255u;
    const uint32_t bar = 1u + (uint32_t)v;
    Stager st;
    stager_setup(st, smem + v * kColHalf);
    st.lead = (uint32_t)v * 256u;
    st.bar_id = bar;
    st.bar_n = 256;
    // (selects, not an indexed read: the kernel parameters stay out of local memory)
    const int n_chunks = part ? a.n_chunks[1] : a.n_chunks[0];
    st.s0 = part ? a.stream[1] : a.stream[0];
    st.s1 = nullptr;
    st.n0 = n_chunks;
    st.n_total = n_chunks;
    double *tmat = a.tmat + (size_t)part * E * E;
    double *cur = reinterpret_cast<double *>(smem + H * kColHalf) + v * 2 * E;
    double *nxt = cur + E;
    for (uint32_t i = tid; i < (uint32_t)E; i += 256u) cur[i] = (i == (uint32_t)col) ? 1.0 : 0.0;
    st.start();   // barrier of the half inside
    const uint32_t sx = (uint32_t)(((w >> 1) & 1) ^ (v & 1)), sz = (uint32_t)((w >> 2) & 1);
    const uint32_t g = (threadIdx.x & 31u) | ((uint32_t)(w & 1) << 5);
    const bool work = (sx | sz) != 0u;
    // slot 1 = X, 2 = Y, 3 = Z: row slot - 1 of the composed map
    const uint32_t row = sx ? (sz ? 2u : 1u) : 3u;
    // source index and sign through the last pull records walked, and the
    // wire of the pass they preceded (-1: none yet)
    uint32_t pj = 0, pneg = 0;
    int pq = -1;
    for (int c = 0; c < n_chunks; ++c) {
        if (!st.wait(c, a.status)) return;
        const Rec *Rr = st.chunk(c);
        int r = 0;
        Rec h = Rr[0];
        while (h.kind == R_PASS) {
            const int q = h.q, n_pull = h.param;
            const uint32_t base = group_base32(g, N, q);
            const uint32_t i = base | (sz << q) | (sx << (N + q));
            if (n_pull > 0) {
                // the pass's reads go through the preceding Clifford run (the
                // last one's index again when the run repeats on the same wire)
                uint32_t neg = 0, j;
                if (h.code == kPullRepeat && pq == q) {
                    j = pj;
                    neg = pneg;
                } else {
                    j = pull_recs(i, N, Rr + r + 1, n_pull, neg);
                    pj = j;
                    pneg = neg;
                    pq = q;
                }
                nxt[i] = flip(cur[j], neg);
                double *t = cur;
                cur = nxt;
                nxt = t;
                named_sync(bar, 256);
            }
            if (h.gate != 0) {
                double out;
                if (work) {
                    const double x = cur[base | (1u << (N + q))];
                    const double y = cur[base | (1u << q) | (1u << (N + q))];
                    const double z = cur[base | (1u << q)];
                    const double *m =
                        reinterpret_cast<const double *>(Rr + r + 2 + n_pull) + 3 * (row - 1u);
                    out = fma(m[2], z, fma(m[1], y, m[0] * x));
                } else {
                    out = cur[i];
                }
                nxt[i] = out;
                double *t = cur;
                cur = nxt;
                nxt = t;
                named_sync(bar, 256);
            }
            r += 1 + n_pull + h.gate;
            h = Rr[r];
        }
        st.release(c);
    }
    for (uint32_t i = tid; i < (uint32_t)E; i += 256u) tmat[(size_t)col * E + i] = cur[i];
}

// ---------------------------------------------------------------- adjoint

template <int N>
__global__ void __launch_bounds__(SCfg<N, 1>::T) k_adjoint_stream(AdjointStreamArgs a) {
    using C = SCfg<N, 1>;
    extern __shared__ __align__(128) unsigned char smem[];
    Stager st;
    st.s0 = a.fwd;
    st.s1 = a.bwd;
    st.n0 = a.n_fwd_chunks;
    st.n_total = a.n_fwd_chunks + a.n_bwd_chunks;
    stager_setup(st, smem);
    double *red = reinterpret_cast<double *>(smem + kOffRed);
    double *rA = reinterpret_cast<double *>(smem + kSmemHeader);
    double *rB = rA + C::E, *lA = rB + C::E, *lB = lA + C::E;
    st.start();
    for (int i = threadIdx.x; i < C::E; i += C::T) {
        rA[i] = i < (1 << N) ? 1.0 : 0.0;
        lA[i] = 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < a.n_terms; k += C::T) lA[a.terms[k].idx] = a.terms[k].coeff;
    __syncthreads();

    // forward: r_m = M_m ... M_1 rho_0
    double *rho = run_stream<N, 1>(st, 0, a.n_fwd_chunks, rA, rB, a.status);
    if (rho == nullptr) return;
    double *rho_n = rho == rA ? rB : rA;
    double *lam = lA, *lam_n = lB;
    // no pull reuse at n = 5 here: with the forward sweep in the same kernel
    // the eight cached registers spill
    if (!adjoint_sweep<N, C::T, (N <= 4)>(st, a.n_fwd_chunks, st.n_total, lam, lam_n, rho,
                                          rho_n, a.grad_rot, a.status, smem, false, a.partials))
        return;
    double acc = 0.0;
    for (int i = threadIdx.x; i < (1 << N); i += C::T) acc += lam[i];
    const double total = block_sum<C::T>(acc, red);
    if (threadIdx.x == 0 && a.expect_out) *a.expect_out = total;
}

// Split adjoint, two CTAs, two launches (phase 0, then phase 1):
//   phase 0: CTA 0 carries rho_0 forward through the first part (stream 0)
//     into rmid, CTA 1 carries O backward through the second part (stream 1)
//     into lmid;
//   phase 1: both CTAs start from the pair (lmid, rmid) at the cut: CTA 0
//     sweeps it backward through the first part (stream 0) and also writes
//     <O> (x-free sum of lambda_0), CTA 1 forward through the second part
//     (stream 1); each rotation's dot lands in the part that holds it.
//   with parts (phase 1 only): CTA b walks part b's stream from the part's
//     own pair -- part 0 backward from its end, every later part forward
//     from its start; CTA 0 writes <O>.
template <int N>
__global__ void __launch_bounds__(SCfg<N, 1>::T) k_adjoint_split(AdjointSplitArgs a) {
    using C = SCfg<N, 1>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int b = blockIdx.x;
    Stager st;
    const double *rmid = a.rmid, *lmid = a.lmid;
    bool fwd = b == 1;
    if (a.parts) {
        const AdjPart P = a.parts[b];
        st.s0 = P.stream;
        st.n0 = P.n_chunks;
        rmid = P.rho;
        lmid = P.lam;
        fwd = P.forward != 0;
    } else {
        st.s0 = b == 0 ? a.stream[0] : a.stream[1];
        st.n0 = b == 0 ? a.n_chunks[0] : a.n_chunks[1];
    }
    st.s1 = nullptr;
    st.n_total = st.n0;
    stager_setup(st, smem);
    double *red = reinterpret_cast<double *>(smem + kOffRed);
    double *rA = reinterpret_cast<double *>(smem + kSmemHeader);
    double *rB = rA + C::E, *lA = rB + C::E, *lB = lA + C::E;
    st.start();
    if (a.phase == 0) {
        for (int i = threadIdx.x; i < C::E; i += C::T)
            rA[i] = (b == 0 && i < (1 << N)) ? 1.0 : 0.0;
        __syncthreads();
        if (b == 1)
            for (int k = threadIdx.x; k < a.n_terms; k += C::T) rA[a.terms[k].idx] = a.terms[k].coeff;
        __syncthreads();
        const double *v = run_stream<N, 1>(st, 0, st.n_total, rA, rB, a.status);
        if (v == nullptr) return;
        double *out = b == 0 ? a.rmid : a.lmid;
        for (int i = threadIdx.x; i < C::E; i += C::T) out[i] = v[i];
        return;
    }
    for (int i = threadIdx.x; i < C::E; i += C::T) {
        rA[i] = rmid[i];
        lA[i] = lmid[i];
    }
    __syncthreads();
    double *rho = rA, *rho_n = rB, *lam = lA, *lam_n = lB;
    const bool ok = adjoint_sweep<N>(st, 0, st.n_total, lam, lam_n, rho, rho_n, a.grad_rot,
                                     a.status, smem, fwd, a.partials);
    if (!ok || b != 0) return;
    double acc = 0.0;
    for (int i = threadIdx.x; i < (1 << N); i += C::T) acc += lam[i];
    const double total = block_sum<C::T>(acc, red);
    if (threadIdx.x == 0 && a.expect_out) *a.expect_out = total;
}

template <int N, int LPG>
cudaError_t launch_stream_n(const StreamArgs &a, cudaStream_t s) {
    using C = SCfg<N, LPG>;
    const size_t smem = kSmemHeader + 2 * (size_t)C::E * sizeof(double);
    static SmemLimit lim;
    cudaError_t e = raise_smem_limit(k_resident_stream<N, LPG>, smem, lim);
    if (e != cudaSuccess) return e;
    k_resident_stream<N, LPG><<<a.n_vec, C::T, smem, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_adjoint_split_n(const AdjointSplitArgs &a, cudaStream_t s) {
    using C = SCfg<N, 1>;
    const size_t smem = kSmemHeader + 4 * (size_t)C::E * sizeof(double);
    static SmemLimit lim;
    cudaError_t e = raise_smem_limit(k_adjoint_split<N>, smem, lim);
    if (e != cudaSuccess) return e;
    k_adjoint_split<N><<<a.parts ? a.n_parts : 2, C::T, smem, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_adjoint_stream_n(const AdjointStreamArgs &a, cudaStream_t s) {
    using C = SCfg<N, 1>;
    const size_t smem = kSmemHeader + 4 * (size_t)C::E * sizeof(double);
    static SmemLimit lim;
    cudaError_t e = raise_smem_limit(k_adjoint_stream<N>, smem, lim);
    if (e != cudaSuccess) return e;
    k_adjoint_stream<N><<<1, C::T, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

int resident_lanes_per_group(int n) { return n <= 4 ? 4 : 1; }

cudaError_t launch_resident_stream(int n, const StreamArgs &a, cudaStream_t s) {
    switch (n) {
    case 1: return launch_stream_n<1, 4>(a, s);
    case 2: return launch_stream_n<2, 4>(a, s);
    case 3: return launch_stream_n<3, 4>(a, s);
    case 4: return launch_stream_n<4, 4>(a, s);
    case 5: return launch_stream_n<5, 1>(a, s);
    case 6: return launch_stream_n<6, 1>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjoint_stream(int n, const AdjointStreamArgs &a, cudaStream_t s) {
    switch (n) {
    case 1: return launch_adjoint_stream_n<1>(a, s);
    case 2: return launch_adjoint_stream_n<2>(a, s);
    case 3: return launch_adjoint_stream_n<3>(a, s);
    case 4: return launch_adjoint_stream_n<4>(a, s);
    case 5: return launch_adjoint_stream_n<5>(a, s);
    case 6: return launch_adjoint_stream_n<6>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjoint_split(int n, const AdjointSplitArgs &a, cudaStream_t s) {
    switch (n) {
    case 1: return launch_adjoint_split_n<1>(a, s);
    case 2: return launch_adjoint_split_n<2>(a, s);
    case 3: return launch_adjoint_split_n<3>(a, s);
    case 4: return launch_adjoint_split_n<4>(a, s);
    case 5: return launch_adjoint_split_n<5>(a, s);
    case 6: return launch_adjoint_split_n<6>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_apply_chain(const double *T, int n_mats, const double *in, double *out,
                               int n_vec, int n, const DevTerm *terms, int n_terms,
                               double *dot_out, cudaStream_t st) {
    const int E = 1 << (2 * n);
    if (n < 1 || n > 3 || n_vec < 1 || (dot_out && n_vec != 1)) return cudaErrorInvalidValue;
    k_apply_chain<<<n_vec, 256, 0, st>>>(T, n_mats, in, out, E, terms, n_terms, dot_out);
    return cudaGetLastError();
}

// out = T^T in at n = 4 (T stored by columns, column j at T + j 4^n): output
// j is column j dotted with in -- the backward step through a part whose
// forward transfer matrix is T, the maps being orthogonal.  A warp per
// output, lanes over the column (coalesced), a fixed shuffle tree.
__global__ void __launch_bounds__(256) k_apply_transfer_t(const double *T, const double *in,
                                                          double *out) {
    constexpr int E = kColE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * 8 + warp;
    const double *col = T + (size_t)j * E;
    double acc = 0.0;
    for (int i = lane; i < E; i += 32) acc = fma(col[i], in[i], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[j] = acc;
}

// <O> = sum of the terms' coeff x v[idx], in term order (one thread: an
// observable has few terms).
__global__ void k_terms_dot(const double *v, const DevTerm *terms, int n_terms, double *out) {
    if (threadIdx.x != 0) return;
    double acc = 0.0;
    for (int k = 0; k < n_terms; ++k) acc += terms[k].coeff * v[terms[k].idx];
    *out = acc;
}

cudaError_t launch_apply_transfer_chain(const double *T, int n_mats, const double *in,
                                        double *out, double *tmp, int n_vec, int n,
                                        const DevTerm *terms, int n_terms, double *dot_out,
                                        cudaStream_t st) {
    const int E = 1 << (2 * n);
    if (n != kColN || n_mats < 1 || n_vec < 1 || (dot_out && n_vec != 1))
        return cudaErrorInvalidValue;
    // matrix s maps the previous vector into tmp (ping-pong between its two
    // halves); the last one writes out (or the free half when out is null)
    const size_t V = (size_t)n_vec * E;
    const double *src = in;
    double *dst = nullptr;
    for (int s = 0; s < n_mats; ++s) {
        const bool last = s == n_mats - 1;
        dst = (last && out) ? out : tmp + (size_t)(s & 1) * V;
        cudaError_t e = launch_apply_transfer(T + (size_t)s * E * E, src, dst, n_vec, n, st);
        if (e != cudaSuccess) return e;
        src = dst;
    }
    if (dot_out) {
        k_terms_dot<<<1, 32, 0, st>>>(src, terms, n_terms, dot_out);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

int resident_adjoint_threads(int n) {
    switch (n) {
    case 1: return SCfg<1, 1>::T;
    case 2: return SCfg<2, 1>::T;
    case 3: return SCfg<3, 1>::T;
    case 4: return SCfg<4, 1>::T;
    case 5: return SCfg<5, 1>::T;
    case 6: return SCfg<6, 1>::T;
    default: return 0;
    }
}

// The pairs at the cuts of a K-part split, n <= 3 (see launch.h): thread i
// computes entry i of every product, summing in index order; the CTA syncs
// between the steps of each chain.
__global__ void __launch_bounds__(64) k_adjoint_pairs(const double *T, int K, int E,
                                                      const double *r1, const double *o,
                                                      double *pairs) {
    const int i = threadIdx.x;
    const size_t EE = (size_t)E * E;
    auto lam = [&](int k) { return pairs + (size_t)(k - 1) * 2 * E; };
    auto rho = [&](int k) { return pairs + (size_t)(k - 1) * 2 * E + E; };
    if (i < E) rho(1)[i] = r1[i];
    __syncthreads();
    for (int k = 1; k + 1 <= K - 1; ++k) {
        // rho_{k+1} = T_k rho_k: row i of T_k is entry i of every column
        const double *Tk = T + (size_t)(k - 1) * EE;
        if (i < E) {
            double acc = 0.0;
            for (int j = 0; j < E; ++j) acc = fma(Tk[(size_t)j * E + i], rho(k)[j], acc);
            rho(k + 1)[i] = acc;
        }
        __syncthreads();
    }
    for (int k = K - 1; k >= 1; --k) {
        // lambda_k = T_k^T lambda_{k+1} (lambda_K = o): column i of T_k
        const double *Tk = T + (size_t)(k - 1) * EE;
        const double *src = k == K - 1 ? o : lam(k + 1);
        if (i < E) {
            double acc = 0.0;
            for (int j = 0; j < E; ++j) acc = fma(Tk[(size_t)i * E + j], src[j], acc);
            lam(k)[i] = acc;
        }
        __syncthreads();
    }
}

cudaError_t launch_adjoint_pairs(const double *T, int K, int n, const double *r1,
                                 const double *o, double *pairs, cudaStream_t st) {
    const int E = 1 << (2 * n);
    if (n < 1 || n > 3 || K < 2) return cudaErrorInvalidValue;
    k_adjoint_pairs<<<1, 64, 0, st>>>(T, K, E, r1, o, pairs);
    return cudaGetLastError();
}

cudaError_t launch_apply_transfer_t(const double *T, const double *in, double *out, int n,
                                    cudaStream_t st) {
    if (n != kColN) return cudaErrorInvalidValue;
    k_apply_transfer_t<<<kColE / 8, 256, 0, st>>>(T, in, out);
    return cudaGetLastError();
}

int transfer_cols_ctas(int n) { return n == kColN ? kColE / 2 : 0; }

// more than half an SM's shared memory, so two of these CTAs never share an
// SM (the kernel needs H halves' chunks and barriers + 4 KiB per half)
constexpr size_t kColSmem = 116 * 1024;
size_t transfer_cols_smem() { return kColSmem; }

cudaError_t launch_transfer_cols(const ColArgs &a, int n, cudaStream_t st) {
    if (n != kColN || a.n_parts < 1 || a.n_parts > 2) return cudaErrorInvalidValue;
    const size_t smem = kColSmem;
    static_assert(4 * kColHalf + 8 * kColE * sizeof(double) <= kColSmem, "column buffers");
    static SmemLimit lim2, lim4;
    cudaError_t e;
    if (a.n_parts == 1) {
        e = raise_smem_limit(k_transfer_cols<2>, smem, lim2);
        if (e != cudaSuccess) return e;
        k_transfer_cols<2><<<kColE / 2, 512, smem, st>>>(a);
    } else {
        e = raise_smem_limit(k_transfer_cols<4>, smem, lim4);
        if (e != cudaSuccess) return e;
        k_transfer_cols<4><<<kColE / 2, 1024, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_apply_transfer(const double *T, const double *a, double *out, int n_vec,
                                  int n, cudaStream_t st) {
    const int E = 1 << (2 * n);
    if (E > 256) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((E + 31) / 32), (unsigned)n_vec);
    k_apply_transfer<<<grid, 256, 0, st>>>(T, a, out, E);
    return cudaGetLastError();
}

}  // namespace stab
