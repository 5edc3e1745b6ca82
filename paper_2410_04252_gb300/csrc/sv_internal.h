// Internal structures shared by the planner, the kernels and the C ABI.
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/sv.h"

namespace sv {

constexpr int kMaxQubits = 40;
constexpr int kMaxSpan = 10;         // coset dimension limit of an EVC / H|psi> pass
constexpr int kMaxRunBits = 7;       // longest contiguous run of a coset pass (2^7 amplitudes)
constexpr int kMaxPassStrings = 384; // strings per EVC pass (shared-memory accumulators and constants)
constexpr int kMaxPassOps = 256;       // gates per shared-memory pass
constexpr int kMaxGroupStrings = 256; // distinct Z masks sharing one X/Y mask in one group

// ---------------------------------------------------------------- planning --

// One schedulable operator: a gate (QSU) or a Pauli string (EVC).
struct Op {
    int32_t kind = 0, nq = 0;
    int32_t q[4] = {-1, -1, -1, -1};
    int32_t param = -1, mat = -1;
    uint64_t tmask = 0;   // logical targets T(op)
};

// A tile of Sec. IV: operators applied under one qubit mapping.
struct Tile {
    int32_t begin = 0, end = 0;      // range of the schedule (order)
    uint64_t local_mask = 0;         // logical local set Q_L
    std::vector<int32_t> pairs;      // QR before the tile: (local phys, global phys) pairs
    std::vector<int32_t> l2p;        // layout in force during the tile
    uint64_t intra_mask = 0;         // hierarchical tiling: logical intra set Q_intra (Alg. 4/5)
};

// Device-side gate of a pass: kind, targets as TILE-LOCAL bit positions.  A
// target t >= kOutTarget is outside the staged tile (only diagonal gates on
// global qubits under the diagonal exemption): physical bit t - kOutTarget,
// constant over a tile.
constexpr int kOutTarget = 64;
struct DevOp {
    int32_t kind;
    int8_t t[4];
    int32_t gate;     // index in the caller's gate list (coefficient / gradient slot)
    int32_t mat;      // complex offset into the matrix array, or -1
};

// One shared-memory pass of K-GATE / K-ADJ.
struct GatePass {
    int32_t tile = 0;
    int32_t k = 0, nlow = 0;          // staged bits, of which the nlow lowest are contiguous
    uint64_t bits = 0;                // physical staged bits
    int32_t op_begin = 0, op_end = 0; // into QsuPlan::ops
    int32_t ph_begin = -1, ph_end = -1;  // register phases (register-blocked passes), else -1
    int32_t db_begin = 0, db_end = 0;    // diagonal blocks of the pass (register-blocked passes)
    int32_t st_begin = 0, st_end = 0;    // steps of the pass's phases
    int32_t area = 0;                    // bytes of the pass's diagonal-block data (shared memory)
    int32_t mem_begin = 0, mem_end = 0;  // the pass's diagonal-block members (QsuPlan::dmembers)
};

// A run of consecutive diagonal operations (RZ, CZ) inside one register
// phase, applied as one diagonal operator.  Two kinds:
//  * register block (kind 0): RZ / CZ on register bits and CZs between a
//    register and a thread bit; the factor of register amplitude v of a
//    thread is a table entry T[v][zm], zm = the register bits on which the
//    thread's register-thread CZs put a Z (a per-thread constant);
//  * thread block (kind 1): RZ / CZ on thread bits only; one complex factor
//    per thread for all its amplitudes.  Such gates commute with everything
//    else in the phase, so all of a phase's go into one thread block.
// Every member op carries mat = -2 - (block index).  smem: byte offset of
// the block's data in the kernels' block area (tables and per-thread data).
struct DiagBlock {
    int32_t op_begin, op_end;     // member ops (consecutive in QsuPlan::ops)
    int32_t m_begin, m_end;       // into QsuPlan::dmembers
    uint32_t rmask;               // register tile bits of the phase
    int32_t kind;                 // 0 register block, 1 thread block
    int32_t smem;
    uint32_t lanes;               // the phase's lane bits (Phase::lanes)
};
enum { SV_DM_REG_RZ = 0, SV_DM_THR_RZ = 1, SV_DM_REG_CZ = 2, SV_DM_THR_CZ = 3, SV_DM_MIX_CZ = 4 };
struct DiagMember {
    int32_t type;     // SV_DM_*
    int32_t a, b;     // register index (0..r-1) or tile bit, per type; MIX_CZ: a register, b tile bit
    int32_t op;       // index into QsuPlan::ops (coefficient and gradient slot)
};
constexpr int kMaxPassDiag = 24;       // diagonal blocks per register-blocked pass
constexpr int kRegThreads = 512;       // CTA size of register-blocked passes (r = k - 9)

// A register phase of a register-blocked pass: each thread holds the
// amplitudes spanned by the tile bits in rmask; ops [op_begin, op_end) are
// applied in registers (non-diagonal gates on rmask bits, diagonal gates on
// any bits).
struct Phase {
    uint32_t rmask;
    int32_t op_begin, op_end;
    int32_t st_begin, st_end;   // steps of the phase (QsuPlan::steps)
    uint32_t lanes;             // tile bits held by the lane bits of the thread index (phase_lanes)
};

// A step of a register phase, executed as one unit by the register-blocked
// kernels.  ROT: RY gates on distinct register bits (they commute), ops
// [op_begin, op_end) ordered by register bit, a = the register-bit mask.
// DIAG: a diagonal block (a = its index in QsuPlan::dblocks), ops = its
// members.  OP: one operation (a = op_begin), applied by the generic code.
enum { SV_STEP_ROT = 0, SV_STEP_DIAG = 1, SV_STEP_OP = 2 };
// The shared-memory slot of tile index i in the register-blocked passes: a
// linear (XOR) swizzle of the low 4 bits by bits 4..11, so that slot(a | b)
// = slot(a) ^ slot(b) for disjoint a, b.
#ifdef __CUDACC__
#define SV_HD __host__ __device__
#else
#define SV_HD
#endif
SV_HD inline uint32_t swz_slot(uint32_t i) { return i ^ (((i >> 4) ^ (i >> 8)) & 15u); }
// Shared memory of a register-blocked pass of k staged bits (512 threads,
// amplitudes of amp bytes): the block area needs at most this much beyond
// the tiles, tables and accumulators, and each block takes
// diag_block_bytes() of it.
constexpr int kRegSmemLimit = 226 * 1024;
constexpr int kAdjSlotStride = kRegThreads / 32 + 1;   // adjoint gradient slots per op (one per warp, padded)
inline int diag_block_bytes(int kind, int k, int amp) {
    const int V = 1 << (k - 9);
    return kind == 0 ? V * V * amp + 512 : 512 * amp;
}
inline int reg_pass_fixed_bytes(int k, int nlow, int nops, int nsteps, int nphases, int amp) {
    // adjoint (the larger): psi and lambda tiles, high offsets, (c, s) per op,
    // steps, block headers, per-phase thread bases and register offsets,
    // per-warp gradient slots, the RY factor per step, alignment
    return 2 * (1 << k) * amp + 8 * (1 << (k - nlow)) + nops * amp + 16 * nsteps + 32 * kMaxPassDiag +
           16 * nops + nphases * (2 * kRegThreads + 8) + nops * kAdjSlotStride * 8 + 8 * (nsteps + 1) + 272;
}
struct RegStep {
    int32_t type, a;
    int32_t op_begin, op_end;
};

struct QsuPlan {
    int n = 0, g = 0, nL = 0;
    std::vector<int32_t> order;       // schedule g at tile granularity
    std::vector<Tile> tiles;
    std::vector<GatePass> passes;
    std::vector<DevOp> ops;           // pass operations, pass by pass, in execution order
    std::vector<Phase> phases;        // register phases of register-blocked passes
    std::vector<RegStep> steps;       // steps of the register phases
    std::vector<DiagBlock> dblocks;   // diagonal blocks of register phases
    std::vector<DiagMember> dmembers;
    std::vector<int32_t> init_l2p, final_l2p;
    int32_t nqr() const {
        int32_t c = 0;
        for (auto &t : tiles) c += t.pairs.empty() ? 0 : 1;
        return c;
    }
};

// EVC / H|psi>: strings grouped by physical X/Y mask, groups packed into
// coset passes (see kernels).
struct EvcString {
    uint64_t z;        // physical Z/Y mask
    int32_t nY;        // |x & z| mod 4
    uint32_t bz;       // bit j = parity(basis_j & z) for the pass's span basis
    double coef;       // summed coefficient of the merged terms
};
struct EvcGroup {
    uint64_t x;        // physical X/Y mask
    uint32_t X;        // partner offset inside the coset tile: (c << kl) | (x & (2^kl - 1))
    int32_t s_begin, s_end;   // strings (slots)
};
struct CosetPass {
    int32_t kl = 0, m = 0;
    uint64_t basis[kMaxSpan] = {};    // span vectors over bits >= kl, reduced
    int32_t pivot[kMaxSpan] = {};
    int32_t g_begin = 0, g_end = 0;   // groups
    int32_t s_begin = 0, s_end = 0;   // strings (slots), contiguous
};

struct EvcPlan {
    int n = 0, g = 0, nL = 0;
    std::vector<int32_t> order;       // term order at tile granularity
    std::vector<Tile> tiles;
    std::vector<int32_t> tile_pass_begin, tile_pass_end;
    std::vector<char> tile_wide;      // 1: strings wider than n_L, pairs cross chunks
    std::vector<CosetPass> passes;
    std::vector<EvcGroup> groups;
    std::vector<EvcString> strings;   // slots
    std::vector<int32_t> term_slot;   // per input term
    std::vector<int32_t> init_l2p, final_l2p;
    int32_t nqr() const {
        int32_t c = 0;
        for (auto &t : tiles) c += t.pairs.empty() ? 0 : 1;
        return c;
    }
};

struct PlanOptions {
    int tile_bits = 12, low_bits = 5;
    int evc_low_bits = 7, evc_span = 6;
    bool pad_highest = true;
    int fuse_max = 0;            // gate operations per gate pass (0 = as many as fit)
    int hier_intra = -1;         // >= 0: hierarchical tiling (Alg. 4/5) with this many intra qubits
    int max_diag = kMaxPassDiag; // diagonal blocks per register-blocked pass (shared-memory budget)
    int amp_bytes = 8;           // 8 complex64, 16 complex128 (shared-memory budget of the blocks)
    bool reg_pairs = true;       // Givens / double excitations may run in register phases
    bool diag_exempt = false;    // QSU: diagonal gates (RZ, CZ) never ask for a QR (per-chunk phases)
    // One greedy step of Alg. 6 done elsewhere (on the device): given the
    // distinct X/Y supports xs with remaining weights w, return the rank of
    // the first global set (lexicographic order) of maximal count and that
    // count.  Empty: the host search with incrementally maintained counts.
    std::function<std::string(const std::vector<uint64_t> &xs, const std::vector<int32_t> &w, int n, int nG,
                              int64_t &rank, int64_t &count)>
        alg6_step;
};

// Returns an empty string on success, else the error message.
std::string validate_gates(int n, const sv_gate *gates, size_t m, size_t np, size_t nmats);
std::string plan_qsu(int n, int g, const sv_gate *gates, size_t m, bool lazy,
                     const PlanOptions &o, const std::vector<int32_t> &l2p_init, QsuPlan &out);
std::string plan_evc(int n, int g, const sv_pauli *p, const double *coeffs, size_t nterms,
                     bool lazy, const PlanOptions &o, const std::vector<int32_t> &l2p_init,
                     EvcPlan &out);
// H|psi> grouping: one tile, no QR, cosets over all n bits.
std::string plan_hpsi(int n, const sv_pauli *p, const double *coeffs, size_t nterms,
                      const PlanOptions &o, const std::vector<int32_t> &l2p, EvcPlan &out);
// Write a bit permutation from layout `from` to layout `to` as at most two
// sets of disjoint physical bit swaps (every permutation is a product of two
// involutions).
void permutation_swaps(const std::vector<int32_t> &from, const std::vector<int32_t> &to,
                       std::vector<std::vector<int32_t>> &swap_sets);

uint64_t hash_bytes(const void *p, size_t n, uint64_t h = 1469598103934665603ull);

// Thread-local message returned by sv_last_error().
void set_last_error(const std::string &m);

}  // namespace sv
