// planner.h -- host-side validation, encoding and pass planning.
//
// Dividing (Sec. III-A): the gate list is cut into maximal blocks of
// single-qubit gates (the paper's U_k) and of two-qubit Clifford gates (V_k).
// Inside a U_k block, the gates of each wire form the run U_{k,j}; gates on
// different wires commute, so each run becomes one P_WIRE pass.  A run with
// more than three rotations is composed into one 3x3 map (the paper's
// LUT_non-CX entry, composed on the device from the angles); shorter runs keep
// their rotations (three FMAs per pair each, fewer than the nine of a map)
// with adjacent Clifford gates folded into signed permutations.  Each V_k
// block becomes one P_CLIFF pass.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/stab.h"
#include "stab_internal.h"

namespace stab {

enum PlanMode {
    PLAN_FUSED = 0,  // runs with more than three rotations become one 3x3 map
    PLAN_GRAD = 1,   // no maps (every rotation kept for its gradient), <= kRotPerGradPass per pass
    PLAN_PLAIN = 2,  // one pass per gate
    PLAN_ROWS = 3,   // every wire run becomes one 3x3 map (latency-optimised resident kernel)
    PLAN_PLAIN_ROWS = 4,  // one pass per gate, every single-qubit gate a 3x3 map
};

struct HostPlan {
    std::vector<DevPass> passes;
    std::vector<DevOp> ops;
    std::vector<DevMap3> maps;
    std::vector<int32_t> map_gate_idx;
    std::vector<RawGate> raw;            // copy of the gate list (map composition reads it)
    std::vector<int32_t> param_ptr;      // CSR: angle slot -> rotation ordinals (PLAN_GRAD only)
    std::vector<int32_t> param_rot;
    std::vector<int32_t> rot_ordinal;    // planning scratch: gate -> rotation ordinal, or -1
    int32_t n_rot = 0;
    int64_t n_params = 0;
    PlanMode mode = PLAN_FUSED;
    std::vector<DevTab> tabs;            // P_TAB passes (two per pass)
};

// Returns STAB_OK or an error code; msg receives a description on error.
int validate_gates(int n, const stab_gate *gates, int64_t m, int64_t n_params, std::string *msg);
int validate_thetas(const double *thetas, int64_t n_params);

// Builds the pass list.  gates must be valid.
// tableaus: long Clifford runs become P_TAB passes (streamed plans; the
// resident instruction streams and the batch kernel do not read them).
// chunked: long gate lists are planned in parallel chunks (same result).
void build_plan(int n, const stab_gate *gates, int64_t m, int64_t n_params, PlanMode mode,
                HostPlan *out, bool tableaus = false, bool chunked = true);

// Tableau of the Clifford gates [i0, i1) applied in order (inverse: the
// inverse map, the inverse gates in reverse order).
void clifford_tableau(int n, const stab_gate *gates, int64_t i0, int64_t i1, bool inverse,
                      DevTab *out);

// Instruction stream of a plan for the resident kernels (see stab_internal.h):
// forward (backward = false) or for the inverse circuit (backward = true).
// With k1 >= 0 only passes [k0, k1) of the plan (walked backward when
// backward is set).  enc, when given, receives the positions of the R_ROT and
// R_MAP3 records (the records the device encodes from the angles).  With last
// = false the records are the first piece of a longer stream: pending pulls
// are applied in an identity pass and the last chunk closes with R_NEXT, so
// the next piece starts on a chunk boundary.
void build_stream(const HostPlan &plan, bool backward, std::vector<Rec> *out, int k0 = 0,
                  int k1 = -1, std::vector<int32_t> *enc = nullptr, bool last = true);

// Signed permutation codes of the single-qubit Clifford opcodes on (X, Y, Z).
uint32_t clifford_perm_code(int op);
uint32_t perm_compose(uint32_t first, uint32_t then);   // apply first, then then
uint32_t perm_inverse(uint32_t code);
constexpr uint32_t kPermIdentity = 0u | (1u << 3) | (2u << 6);

// Observable terms -> deduplicated device terms (index z | x << n).
int encode_terms(int n, const stab_term *O, int64_t n_terms, std::vector<DevTerm> *out);

}  // namespace stab
