// launch.h -- host-side launch wrappers of the library's kernels.
#pragma once

#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "stab_internal.h"

namespace stab {

constexpr int kMaxResidentQubits = 6;   // two buffers of 4^6 doubles = 64 KiB of shared memory
constexpr int kMaxResidentAdjoint = 6;  // four buffers of 4^6 doubles = 128 KiB
constexpr int kRotPerGradPass = 8;      // rotations per P_WIRE pass in gradient plans

// A kernel's dynamic shared-memory limit belongs to the function, not to a
// launch: every thread and context of the process sees the same value.  It is
// only ever raised here, under a lock, so that one thread lowering it cannot
// fail another thread's larger launch.  One SmemLimit per kernel.
struct SmemLimit {
    std::mutex mu;
    size_t set[64] = {};   // per device: the limit set so far
};

template <typename K>
cudaError_t raise_smem_limit(K kernel, size_t smem, SmemLimit &lim) {
    if (smem <= 48 * 1024) return cudaSuccess;   // the default limit
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(lim.mu);
    const bool tracked = dev >= 0 && dev < 64;
    if (tracked && lim.set[dev] >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && tracked) lim.set[dev] = smem;
    return e;
}

struct StreamArgs {
    const Rec *stream;       // instruction stream (device), n_chunks x kChunkRecs records
    int32_t n_chunks;
    int32_t init;            // InitMode
    const DevTerm *terms;    // INIT_TERMS
    int32_t n_terms;
    int32_t n_vec;           // vectors (blocks); block b starts as Z_b for INIT_GENERATOR
    const double *in;        // INIT_LOAD: block b reads in + b * 4^n
    double *out;             // final vector of block b at out + b * 4^n (may be null)
    double *xfree_out;       // block b: sum of its x-free coefficients (may be null)
    int32_t *status;         // set to a nonzero code when a bounded wait gives up
};

// One part of a many-part resident adjoint sweep (phase 1 of k_adjoint_split
// with parts): the part's gradient stream, walked backward (the first part,
// from its end) or forward (every later part, from its start), and the pair
// (lambda, rho) where the walk starts.
struct AdjPart {
    const Rec *stream;
    int32_t n_chunks;
    int32_t forward;
    const double *lam, *rho;
};

// Split resident adjoint (two CTAs, two launches; see k_adjoint_split).
struct AdjointSplitArgs {
    const Rec *stream[2];    // phase 0: forward [0, cut), backward [cut, P); phase 1: backward
                             // [0, cut), forward [cut, P) -- all of the gradient plan
    int32_t n_chunks[2];
    int32_t phase;           // 0 or 1
    const DevTerm *terms;    // phase 0, CTA 1: O
    int32_t n_terms;
    double *rmid, *lmid;     // rho and lambda at the cut: phase 0 writes, phase 1 reads
    double *grad_rot;        // phase 1: one entry per rotation ordinal
    double *partials;        // phase 1, optional: per-thread dots [rotation ordinal][threads]
                             // (summed afterwards by k_reduce_partials); null: each pass
                             // reduces its rotations' dots over the CTA into grad_rot
    const AdjPart *parts;    // phase 1, optional (device array): one CTA per part, in place
    int32_t n_parts;         // of stream[] and the pair (lmid, rmid); CTA 0 writes <O>
    double *expect_out;      // phase 1: <O>
    int32_t *status;
};

struct AdjointStreamArgs {
    const Rec *fwd;          // forward stream of the gradient plan
    const Rec *bwd;          // backward stream of the gradient plan
    int32_t n_fwd_chunks;
    int32_t n_bwd_chunks;
    const DevTerm *terms;
    int32_t n_terms;
    double *grad_rot;        // one entry per rotation ordinal
    double *partials;        // optional, as in AdjointSplitArgs
    double *expect_out;      // <O>
    int32_t *status;
};
// Threads of the resident adjoint kernels' CTA at n qubits (the row length
// of their per-thread partials).
int resident_adjoint_threads(int n);
// The pairs at the cuts of a K-part split at n <= 3, one CTA: rho_1 = r1,
// rho_{k+1} = T_k rho_k, lambda_{K-1} = T_{K-1}^T o, lambda_k = T_k^T
// lambda_{k+1}, with T_k (k = 1 .. K-1) at T + (k - 1) 16^n (by columns);
// pairs = [lambda_1, rho_1, ..., lambda_{K-1}, rho_{K-1}], 4^n doubles each.
cudaError_t launch_adjoint_pairs(const double *T, int K, int n, const double *r1,
                                 const double *o, double *pairs, cudaStream_t st);
// Bytes of the resident adjoint's per-thread dot shares for n_rot rotations
// at n qubits, or 0 where the sweeps reduce each pass's dots themselves.
size_t resident_partial_bytes(int n, int64_t n_rot);

// One unit of the persistent batch kernel: one vector of one circuit.
struct BatchUnit {             // 64 bytes
    const Rec *stream;         // the circuit's forward (generators) or backward (<O>) stream
    int32_t n_chunks;
    int8_t n;                  // qubits (1 .. 8)
    int8_t init;               // INIT_GENERATOR or INIT_TERMS
    int16_t gen;               // generator index for INIT_GENERATOR
    const DevTerm *terms;      // INIT_TERMS
    int32_t n_terms;
    int32_t pad;
    double *out;               // final vector (may be null)
    double *xfree_out;         // <O> (may be null)
    int64_t cost;              // host-side ordering key
    int64_t reserved;
};
static_assert(sizeof(BatchUnit) == 64, "BatchUnit layout");

struct BatchArgs {
    const BatchUnit *units;
    int32_t n_units;
    int32_t *counter;          // next unit to take (zeroed before the launch)
    int32_t *status;
    double *slab;              // per-CTA global vectors for n > kMaxResidentQubits (may be null)
    size_t slab_doubles;       // doubles per CTA slab
    int32_t max_chunks;        // > 0: each unit runs only its first max_chunks chunks (timing
                               // samples; the outputs are then partial); 0: whole streams
    int32_t smem_n;            // units of n <= smem_n keep their vectors in shared memory, the
                               // others in the slab (0: kMaxResidentQubits)
};

// One slice of one unit of the serving iteration kernel (k_serve): a vector
// (or an adjoint pair) of one admitted request carried through a contiguous
// range of chunks of one of its instruction streams.  The request's state
// vectors live in its own device memory between launches; a slice starts
// from them (or from its initial value) and writes them back.
enum ServeKind : int8_t {
    SV_VEC = 0,        // one vector through a stream (forward or backward)
    SV_PAIR_BWD = 1,   // (lambda, rho) through a backward gradient stream, dots then ops
    SV_PAIR_FWD = 2,   // (lambda, rho) through a forward gradient stream, ops then dots
};

struct ServeUnit {             // 80 bytes
    const Rec *stream;         // first chunk of the slice
    int32_t n_chunks;          // chunks of the slice
    int8_t n;                  // qubits (1 .. kServeMaxQubits)
    int8_t kind;               // ServeKind
    int8_t init;               // INIT_RHO0 / INIT_TERMS (first slice of a vector), INIT_LOAD
    int8_t flags;              // SF_LAST | SF_ROWS
    const DevTerm *terms;      // INIT_TERMS
    int32_t n_terms;
    int32_t pad;
    const double *src;         // INIT_LOAD: the vector (SV_VEC) or lambda (pairs)
    const double *src2;        // INIT_LOAD, pairs: rho
    double *state;             // persistent state: SV_VEC [v | spare] (2 x 4^n doubles),
                               // pairs [lambda | rho | spare | spare] (4 x 4^n)
    double *grad_rot;          // pairs: the dots, by rotation ordinal
    double *xfree_out;         // SF_LAST: x-free sum of the vector (SV_VEC) or of lambda
    int64_t reserved;
};
static_assert(sizeof(ServeUnit) == 80, "ServeUnit layout");

constexpr int kServeMaxQubits = 8;
constexpr int SF_LAST = 1;     // the slice ends the unit's stream
constexpr int SF_ROWS = 2;     // SV_VEC at n <= 4: every wire pass one 3x3 map (lane quads)

struct ServeArgs {
    const ServeUnit *units;
    int32_t n_units;
    int32_t *counter;          // next unit to take (zeroed before the launch)
    int32_t *status;
    int32_t smem_buf;          // bytes of shared memory for state buffers: a unit whose
                               // buffers (2 or 4 x 4^n doubles) fit runs in shared memory
    int64_t *unit_cycles;      // per unit: SM clock cycles its slice took (may be null)
};

size_t serve_smem_bytes(int smem_buf);
cudaError_t serve_occupancy(size_t smem, int *ctas_per_sm);
cudaError_t launch_serve(const ServeArgs &a, int grid, size_t smem, cudaStream_t s);

size_t batch_smem_bytes(int max_n_in_smem);
int batch_threads();
cudaError_t batch_occupancy(size_t smem, int *ctas_per_sm);
cudaError_t launch_batch(const BatchArgs &a, int grid, size_t smem, cudaStream_t s);

}  // namespace stab

typedef struct stab_ctx stab_ctx;

namespace stab {

// The context's main stream (work queued by the asynchronous entry points is
// complete once this stream is).
cudaStream_t ctx_stream(stab_ctx *ctx);
// Marks the context's split generator sweep as not made for its current
// angles, so the next call that needs it runs it again (timing probes that
// call the same entry point repeatedly).
void ctx_forget_sweep(stab_ctx *ctx);

// Density matrix from the forward-evolved coefficients of 2^n |0><0|:
// rho (device, 2 x 4^n doubles, interleaved complex, row-major).
cudaError_t launch_decode_rho(const double *r, int n, double *rho, cudaStream_t st);

// Kernel that waits on a barrier nothing completes (bounded), for the self-test.
cudaError_t launch_bounded_wait(int64_t polls, int32_t *status, cudaStream_t st);

// Records the CUDA error behind a STAB_E_CUDA status (stab_last_cuda_error).
void record_cuda_error(cudaError_t e);

// Composed 3x3 map of every run (maps[i].m), from the angle array on the
// device: one thread per map when no run is longer than kSeqMapGates gates
// (max_count, the longest run), else one warp per map.
constexpr int kSeqMapGates = 32;
cudaError_t launch_compose_maps(DevMap3 *maps, int n_maps, int max_count,
                                const int32_t *map_gate_idx, const RawGate *gates,
                                const double *thetas, cudaStream_t st);
int max_map_count(const DevMap3 *maps, size_t n_maps);   // host: the longest run

// Encode: the composed maps, then the lifting coefficients of every rotation op.
cudaError_t launch_encode(DevOp *ops, int n_ops, DevMap3 *maps, int n_maps, int max_count,
                          const int32_t *map_gate_idx, const RawGate *gates, const double *thetas,
                          cudaStream_t st);

// Stream encode: shear coefficients of the R_ROT records and the matrices of
// the R_MAP3 records listed in enc (indices into recs), copied from maps
// (composed before by launch_compose_maps).
cudaError_t launch_encode_stream(Rec *recs, const int32_t *enc, int n_enc, const DevMap3 *maps,
                                 const double *thetas, cudaStream_t st);

// Shared-memory-resident propagation, one CTA per vector (n <= kMaxResidentQubits).
cudaError_t launch_resident_stream(int n, const StreamArgs &a, cudaStream_t st);
// out[k] = T a[k] (k < n_vec) for 4^n x 4^n T stored by columns; n <= 4.
// Columns 1 .. 4^n - 1 of the transfer matrix of a stream (column j = basis
// string j through its passes) into tmat (column j at tmat + j * 4^n), two
// columns per CTA; n = 4 only.  transfer_cols_ctas(n): its grid (0: n unsupported).
int transfer_cols_ctas(int n);
// out_k = T_{n_mats-1} ... T_0 in_k for n <= 3 (matrices of 4^n x 4^n, column
// j of matrix s at T + s 16^n + j 4^n); with dot_out (n_vec = 1) also
// <O> = sum of terms' coeff x out[idx].  out may be null.
cudaError_t launch_apply_chain(const double *T, int n_mats, const double *in, double *out,
                               int n_vec, int n, const DevTerm *terms, int n_terms,
                               double *dot_out, cudaStream_t st);
// The columns of one or two transfer matrices (n_parts streams) at n = 4:
// matrix p at tmat + p 16^n, column j at + j 4^n (column 0 is not written);
// 128 CTAs of two (one matrix) or four (two matrices) columns each.
struct ColArgs {
    const Rec *stream[2];
    int32_t n_chunks[2];
    int32_t n_parts;
    double *tmat;
    int32_t *status;
};
cudaError_t launch_transfer_cols(const ColArgs &a, int n, cudaStream_t st);
// Dynamic shared memory of a k_transfer_cols CTA (more than half an SM's).
size_t transfer_cols_smem();
// out = T^T in for one n = 4 transfer matrix (the backward step through its
// part): 4^n outputs, each a column of T dotted with in.
cudaError_t launch_apply_transfer_t(const double *T, const double *in, double *out, int n,
                                    cudaStream_t st);
// out_k = T_{n_mats-1} ... T_0 in_k at n = 4 (one k_apply_transfer per matrix,
// tmp: 2 x n_vec x 4^n doubles between them); with dot_out (n_vec = 1) also
// <O> = sum of terms' coeff x the result[idx], in term order.  out may be null.
cudaError_t launch_apply_transfer_chain(const double *T, int n_mats, const double *in,
                                        double *out, double *tmp, int n_vec, int n,
                                        const DevTerm *terms, int n_terms, double *dot_out,
                                        cudaStream_t st);
cudaError_t launch_apply_transfer(const double *T, const double *a, double *out, int n_vec,
                                  int n, cudaStream_t st);
int resident_lanes_per_group(int n);

// Streamed passes over n_vec vectors of 4^n doubles in global memory.
cudaError_t launch_fill(double *vec, int n, int n_vec, int init, const DevTerm *terms,
                        int n_terms, cudaStream_t st);
cudaError_t launch_stream_wire(double *vec, int n, int n_vec, const DevPass &p, const DevOp *ops,
                               const DevMap3 *maps, int inverse, cudaStream_t st);
cudaError_t launch_stream_cliff(const double *src, double *dst, int n, int n_vec,
                                const DevPass &p, const DevOp *ops, int inverse, cudaStream_t st);
cudaError_t launch_xfree_sum(const double *vec, int n, int n_vec, double *out, cudaStream_t st);
// *out = <a, b> over the 4^n entries, fixed order; partial: 256 doubles of scratch.
cudaError_t launch_dot(const double *a, const double *b, int n, double *partial, double *out,
                       cudaStream_t st);
// P_TAB: dst = the Clifford map whose tableau is *tab applied as a signed gather (n <= 12).
cudaError_t launch_stream_tab(const double *src, double *dst, int n, int n_vec,
                              const DevTab *tab, cudaStream_t st);

// Several consecutive wire passes on at most kTileWires wires fused into one
// streamed launch: each CTA loads a tile (all 4^|Q| slots of the wires Q times
// some of the lowest other index bits) into shared memory, applies the passes
// in order and writes it back.
constexpr int kTileWires = 4;
constexpr int kTileMaxPasses = 8;
constexpr int kTileMaxBits = 12;        // 4096 doubles = 32 KiB of shared memory
constexpr int kTileStagedOps = 96;      // ops of a group staged in shared memory (3 KiB)

struct BitRuns {                        // deposit of a packed integer into index bits
    uint8_t n;
    uint8_t src[16], dst[16], len[16];
};

struct TileGroup {
    int32_t n_pass;
    int32_t tile_bits;                  // log2 entries per tile
    int32_t rest_bits;                  // 2n - tile_bits: log2 tiles per vector
    int32_t inverse;
    uint8_t lz[kTileMaxPasses], lx[kTileMaxPasses];   // tile-local bits of each pass's wire
    uint16_t n_ops[kTileMaxPasses];
    uint8_t n_rot[kTileMaxPasses];      // rotations of each pass (adjoint groups)
    uint32_t first[kTileMaxPasses];
    BitRuns tile_runs;                  // local entry -> global index bits
    BitRuns rest_runs;                  // tile id -> global index bits
    // A Clifford gather folded into the tile loads (a P_CLIFF pass that
    // precedes the group): entry i is read from pull(i) of the source, signed.
    int32_t pull_n;                     // ops of that pass (0: plain load)
    uint32_t pull_first;
    int32_t pull_inverse;
};

// src == dst unless the group carries a folded Clifford gather (then the
// result goes to dst, a different buffer).
cudaError_t launch_stream_tile(const double *src, double *dst, int n, int n_vec,
                               const TileGroup &tg, const DevOp *ops, const DevMap3 *maps,
                               cudaStream_t st);

// Adjoint gradient, shared-memory resident (n <= kMaxResidentAdjoint).
cudaError_t launch_adjoint_split(int n, const AdjointSplitArgs &a, cudaStream_t s);
cudaError_t launch_adjoint_stream(int n, const AdjointStreamArgs &a, cudaStream_t st);

// Streamed adjoint pieces.
int adjoint_stream_blocks(int n);
// One wire pass of the adjoint on (lambda, rho): backward (forward = 0: the
// dot at the post-gate pair, then the inverse gate) or forward (the gate, then
// the dot); partials[gate][block], adjoint_stream_blocks(n) blocks.
cudaError_t launch_adjoint_wire(double *lam, double *rho, int n, const DevPass &p,
                                const DevOp *ops, double *partials, int forward,
                                cudaStream_t st);
// Tile-fused reverse sweep on the contiguous pair (lambda, rho) for n <=
// kAdjTileMaxN: tiles of 2^kAdjTileBits entries, one per CTA and one group per
// thread, grid = adjoint_stream_blocks(n); partials[gate][block] as
// launch_adjoint_wire.
constexpr int kAdjTileMaxN = 8;
constexpr int kAdjTileBits = 9;
size_t adjoint_tile_smem(int tile_bits, int n_rot);   // n_rot: rotations of the group
cudaError_t launch_adjoint_tile(const double *src_pair, double *dst_pair, int n,
                                const TileGroup &tg, const DevOp *ops, double *partials,
                                cudaStream_t st);
cudaError_t launch_reduce_partials(const double *partials, int n_rot, int n_blocks,
                                   double *grad_rot, cudaStream_t st);
cudaError_t launch_gather_grads(const double *grad_rot, const int32_t *param_ptr,
                                const int32_t *param_rot, int n_params, double *grads,
                                cudaStream_t st);

// ---------------------------------------------------------------- sparse term lists (k_sparse.cu)

constexpr int kSpMaxBlocks = 608;        // 4 CTAs per SM on 152 SMs

struct SpGate {                          // one Clifford gate of a run, already inverted for
    uint8_t op, q0, q1, pad;             // backward runs (S <-> S^dagger)
};

struct SpTab {                           // tableau entry: image of X_q or Z_q, its sign
    uint64_t key;
    uint32_t neg;
    uint32_t pad;
};

// A run's tableau regrouped by chunks of 4 qubits (8 generators): per chunk
// the ordered products of all 256 subsets of its generator images.
constexpr int kSpChunkQubits = 4;
constexpr int kSpChunks = 8;             // 32 qubits
constexpr int kSpChunkEntries = kSpChunks * 256;
struct SpChunk {                         // x, z of the product string, phase exponent (mod 4)
    uint32_t x, z, e, pad;
};

struct SpSlot {                          // a table slot: key and list position (-1 free)
    uint64_t key;
    int32_t pos;
    int32_t pad;
};

struct SpRotArgs {
    const uint64_t *keys;                // input list (keys z | x << n, coefficients)
    const double *vals;
    uint64_t *keys_out;                  // output list (the other buffer)
    double *vals_out;
    int64_t *counts;                     // counts[step] = order before step
    int32_t *flags;                      // [0] stop code (1 overflow, 2 threshold), [1] step
    int32_t step, n, q, axis;            // axis 0/1/2 = R_x/R_y/R_z
    const double *cs;
    int32_t param, inverse;
    SpSlot *table;                       // open-addressing table (one 16-byte slot per probe)
    int32_t log_h;
    int32_t *slot_of;                    // per term: its table slot
    int32_t *partner;                    // per term: position of its partner, -1 absent
    int64_t *blk;                        // per block: emitted terms, then their offsets
    int32_t *err;                        // set when a table probe runs out (never expected)
    int64_t cap;                         // list capacity
    int64_t threshold;                   // stop above this order (0: never)
    int64_t bound;                       // host bound on counts[step] (sizes the grid)
};

cudaError_t launch_sp_cliff(uint64_t *keys, double *vals, int64_t *counts, const int32_t *flags,
                            int step, int n, const SpGate *gates, int n_gates, int64_t bound,
                            cudaStream_t st);
cudaError_t launch_sp_rotation(const SpRotArgs &a, cudaStream_t st);
// cs[2 p] = cos(thetas[p]), cs[2 p + 1] = sin(thetas[p]) for every slot
cudaError_t launch_sp_cos_sin(const double *thetas, int64_t n_params, double *cs,
                              cudaStream_t st);
// tabs: 64 entries per run (2n used); runs [r] = gates [run_first[r], + run_count[r]);
// chunks: kSpChunkEntries per run, built from tabs
cudaError_t launch_sp_tableau(const SpGate *gates, const int32_t *run_first,
                              const int32_t *run_count, int n_runs, int n, SpTab *tabs,
                              SpChunk *chunks, cudaStream_t st);
// chunks: the run's kSpChunkEntries entries
cudaError_t launch_sp_cliff_tab(uint64_t *keys, double *vals, int64_t *counts,
                                const int32_t *flags, int step, int n, const SpChunk *chunks,
                                int64_t bound, cudaStream_t st);
cudaError_t launch_sp_xfree(const uint64_t *keys, const double *vals, const int64_t *counts,
                            int step, int n, double *partial, double *out, cudaStream_t st);
cudaError_t launch_sp_to_terms(const uint64_t *keys, const double *vals, const int64_t *counts,
                               int step, DevTerm *out, int64_t bound, cudaStream_t st);

}  // namespace stab

struct stab_ctx;
namespace stab {
// <0^n| U^dagger O U |0^n> for the loaded circuit, O given as nt deduplicated
// device terms (stab_api.cpp); blocks until the value is on the host.
int expect_device_terms(stab_ctx *c, const DevTerm *terms, int64_t nt, double *out);
}  // namespace stab
