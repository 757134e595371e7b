// stab_internal.h -- device program format shared by the host planner and the
// CUDA kernels of the library (not part of the public interface).
//
// A loaded circuit becomes a list of passes (Sec. III-A "dividing"): a P_WIRE
// pass applies the run of single-qubit gates of one wire inside a block of
// consecutive non-CX gates (the paper's U_{k,j}); a P_CLIFF pass applies a run
// of two-qubit Clifford gates (the paper's V_k) as one signed permutation of
// the index space.  Each pass refers to a slice of the op array.
#pragma once

#include <cstdint>

namespace stab {

enum OpKind : uint8_t {
    K_PERM = 0,  // single-qubit Clifford: signed permutation of the (X, Y, Z) slots
    K_ROT = 1,   // single-qubit rotation, lifting form (three shears)
    K_MAP3 = 2,  // composed single-qubit run: 3x3 orthogonal map on (X, Y, Z)
    K_CX = 3,    // CNOT(q -> q1)
    K_CZ = 4,    // CZ(q, q1)
};

// P_TAB: a long run of Clifford gates of any kind (streamed plans only),
// applied as one signed gather through the run's tableau (DevTab).
enum PassType : uint8_t { P_WIRE = 0, P_CLIFF = 1, P_TAB = 2 };

// Rotation axes.  Within the 4-slot group (I, X, Y, Z) of one wire a rotation
// about axis a mixes the pair (u, v) below as u' = c u - s v, v' = s u + c v
// (Table I rows R_x, R_y, R_z).
enum Axis : uint8_t { AX_X = 0, AX_Y = 1, AX_Z = 2 };

struct DevOp {          // 32 bytes
    uint8_t kind;       // OpKind
    uint8_t q;          // wire; control of CX; first qubit of CZ
    uint8_t q1;         // target of CX; second qubit of CZ
    uint8_t axis;       // K_ROT: Axis
    int32_t param;      // K_ROT: angle slot; K_MAP3: index into the map array
    int32_t gate;       // K_ROT: gradient slot (rotation ordinal); else -1
    uint16_t perm;      // K_PERM: forward code (see perm_code in device_ops.cuh);
                        // K_ROT: 1 when the reduced angle carries a factor R(pi) (set on device)
    uint16_t perm_inv;  // K_PERM: inverse code
    double t;           // K_ROT: -tan(phi / 2) of the reduced angle phi (set on device)
    double s;           // K_ROT: sin(phi) (set on device)
};
static_assert(sizeof(DevOp) == 32, "DevOp layout");

struct DevPass {        // 8 bytes
    uint8_t type;       // PassType
    uint8_t q;          // P_WIRE: wire
    uint16_t n_ops;
    uint32_t first;     // first op
};
static_assert(sizeof(DevPass) == 8, "DevPass layout");

struct DevMap3 {        // 80 bytes; m is composed on device from the run's gates
    double m[9];        // row-major on (X, Y, Z): new = m * old
    int32_t first;      // first entry in the map-gate index array
    int32_t count;      // number of gates in the run
};
static_assert(sizeof(DevMap3) == 80, "DevMap3 layout");

// Device-side raw gate (same layout as the public stab_gate).
struct RawGate {
    uint8_t op, q0, q1, flags;
    int32_t param;
};

enum InitMode : int32_t {
    INIT_GENERATOR = 0,  // block b starts as Z_b (generator of |0^n>)
    INIT_TERMS = 1,      // sum of observable terms
    INIT_RHO0 = 2,       // 1 on every string of I and Z (2^n |0><0| in the Pauli basis)
    INIT_LOAD = 3,       // copy from a device vector
};

// Tableau of a Clifford map V on n <= 12 qubits: the images V X_q V^dagger
// (entry q) and V Z_q V^dagger (entry n + q), each a signed string with x / z
// masks; sign bit j of `neg` is entry j's sign.  A P_TAB pass (first = k)
// refers to tabs[2k] = the run's inverse U^dagger (forward gathers) and
// tabs[2k + 1] = the run U (inverse gathers).
struct DevTab {         // 200 bytes
    uint32_t x[24];
    uint32_t z[24];
    uint32_t neg;
    uint32_t pad;
};
static_assert(sizeof(DevTab) == 200, "DevTab layout");

struct Program {
    const DevPass *passes;
    const DevOp *ops;
    const DevMap3 *maps;
    const DevTab *tabs;
    int32_t n_passes;
    int32_t n_ops;
};

// ---------------------------------------------------------------- streams
//
// The shared-memory-resident kernels read a forward-only instruction stream
// of 32-byte records, packed by the host into chunks of kChunkRecs records
// that the kernel stages into shared memory with bulk copies.  A pass never
// straddles a chunk.  Runs of two-qubit Clifford gates are not separate
// passes: their records (R_CX, R_CZ) precede the next wire pass and are
// applied while that pass reads its inputs (each entry is pulled through the
// permutation).  The backward stream lists passes, pulls and ops in the order
// the inverse circuit needs them, with rotations and maps flagged inverse, so
// kernels never walk a stream backward.
constexpr int kChunkRecs = 128;            // 4 KiB per chunk

enum RecKind : uint8_t {
    R_END = 0,    // end of the program
    R_NEXT = 1,   // the rest of this chunk is unused: continue with the next chunk
    R_PASS = 2,   // wire pass on qubit q: param = number of pull records, gate = op records
    R_CX = 3,     // pull record CX(q -> q1)
    R_CZ = 4,     // pull record CZ(q, q1)
    R_ROT = 5,    // rotation (axis, param = angle slot, gate = gradient slot)
    R_PERM = 6,   // signed permutation of (X, Y, Z); code = permutation code
    R_MAP3 = 7,   // composed 3x3 map, param = index of the run; 3 R_DATA records follow
    R_DATA = 8,   // raw storage of the 9 matrix entries of the preceding R_MAP3
};

struct Rec {            // 32 bytes
    uint8_t kind;       // RecKind
    uint8_t q, q1;      // qubits
    uint8_t axis;       // R_ROT: Axis
    int32_t param;
    int32_t gate;
    uint16_t code;      // R_PERM: permutation code; R_ROT: 1 when a factor R(pi) applies (device)
    uint16_t inv;       // R_ROT / R_MAP3: 1 = apply the inverse (set by the host)
    double t, s;        // R_ROT: shear coefficients (device)
};
static_assert(sizeof(Rec) == 32, "Rec layout");

// R_PASS header, code field: the pass's pull records equal those of the
// stream's previous pull pass (a repeated Clifford run, as in layered
// circuits).  A hint: a kernel that has pulled through that previous pass in
// the same layout may reuse its source index and sign; any other reads the
// records as usual.
constexpr uint16_t kPullRepeat = 1;

struct DevTerm {         // deduplicated observable term: index in the device layout
    double coeff;
    uint64_t idx;
};

}  // namespace stab
